// Fused nodal-DG step kernels for sm_103a (FP32 CUDA-core path).
//
// One CTA owns a contiguous block of EB elements.  Per step it
//   1. stages the block's fields q^m [EB][Nf][Np], geometry records and
//      connectivity in shared memory with 1-D TMA bulk copies
//      (cp.async.bulk + mbarrier, bounded wait), together with the operator
//      blob [Dr Ds Dt LIFT] when it fits;
//   2. computes, element-wise, the GEMM inputs in shared memory with the
//      element index fastest (columns): the fields / geometric combinations
//      the volume term needs, and the Fscale-weighted penalty terms at the
//      4 Nfp face nodes (trace gather: own node via the face mask, neighbour
//      node via neighbour face + one of 6 face rotations; neighbours inside
//      the block are read from shared memory, others from global/L2);
//   3. each thread owns a tile of 4 output nodes x TN elements and
//      accumulates every operator product for that tile in registers
//      (Section 3.2: six Np x Np products + the merged LIFT product for the
//      acoustic model, eighteen + LIFT for the elastic model), streaming the
//      operator rows as float4 from shared memory (or L1) and the element
//      columns as float2/float;
//   4. combines the reference-direction results with the geometric factors
//      and does the AB3 update (Eq. updateScheme) straight from registers:
//      q^{m+1} = q^m + dt (a1 r^m + a2 r^{m-1} + a3 r^{m-2}); r^m overwrites
//      r^{m-2} in place (each value is read before it is written by the same
//      thread), and q^{m+1} goes to the other buffer of a ping-pong pair
//      because neighbours still read q^m.
//
// The RHS (Eq. dgLocalRhs) in the form used here:
//   acoustic: r_p   = sum_d D_d w_d + LIFT (Fscale dp),  w_d = -kappa sum_c g_cd v_c
//             r_v_c = -(1/rho) sum_d g_cd (D_d p) + LIFT (Fscale dv_c)
//   elastic:  r_v_i = sum_d D_d s_id + LIFT (Fscale p_v,i), s_id = (1/rho) sum_m g_md sigma_im
//             r_sig_ij = lambda delta_ij div v + mu (dv_i/dx_j + dv_j/dx_i) + LIFT (Fscale P_sig,ij),
//             dv_i/dx_j = sum_d g_jd (D_d v_i)
// with g_cd = dr_d/dx_c and the penalty terms of Section 2.1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_args.h"

namespace dgk {

template <int N>
struct Sz {
  static constexpr int Np = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int Nfp = (N + 1) * (N + 2) / 2;
  static constexpr int NFN = 4 * Nfp;
  static constexpr int Mpad = (Np + 3) & ~3;
  static constexpr int RT = Mpad / 4;
  static constexpr int KD = 3 * Np + NFN;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, "
      "p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after ~2^31 clock cycles (about a second) and
// reports through the error word.  Returns false on expiry.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1ll << 31)) {
      if (err) atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

template <int TN>
struct VecT;
template <>
struct VecT<1> {
  __device__ __forceinline__ static void load(const float* p, float* o) { o[0] = p[0]; }
};
template <>
struct VecT<2> {
  __device__ __forceinline__ static void load(const float* p, float* o) {
    float2 v = *reinterpret_cast<const float2*>(p);
    o[0] = v.x;
    o[1] = v.y;
  }
};
template <>
struct VecT<4> {
  __device__ __forceinline__ static void load(const float* p, float* o) {
    float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
};

template <bool SMEM>
__device__ __forceinline__ float4 load_op(const float* p) {
  if constexpr (SMEM) return *reinterpret_cast<const float4*>(p);
  else return __ldg(reinterpret_cast<const float4*>(p));
}

__device__ __forceinline__ void fma4(float acc[4], const float4& a, float x) {
  acc[0] = fmaf(a.x, x, acc[0]);
  acc[1] = fmaf(a.y, x, acc[1]);
  acc[2] = fmaf(a.z, x, acc[2]);
  acc[3] = fmaf(a.w, x, acc[3]);
}

__device__ __forceinline__ constexpr float ref_normal(int f, int i) {
  return (f == 0) ? (i == 2 ? -1.f : 0.f)
       : (f == 1) ? (i == 1 ? -1.f : 0.f)
       : (f == 2) ? 1.f
                  : (i == 0 ? -1.f : 0.f);
}

// ---------------------------------------------------------------- smem plan
template <int MODEL, int N, int EB, bool OPS_SMEM>
struct Plan {
  using S = Sz<N>;
  static constexpr int Nf = MODEL == 0 ? 4 : 9;
  static constexpr int nQ = EB * Nf * S::Np;
  // GEMM inputs, column (element) fastest
  static constexpr int nXvol = (MODEL == 0 ? 4 : 12) * S::Np * EB;   // acoustic p,w0..2 ; elastic v0..2, s00..s22
  static constexpr int nXsur = Nf * S::NFN * EB;                     // penalties per field
  static constexpr int nOps = OPS_SMEM ? S::KD * S::Mpad : 0;
  static constexpr int oQ = 0;
  static constexpr int oXvol = oQ + nQ;
  static constexpr int oXsur = oXvol + nXvol;
  static constexpr int oOps = oXsur + nXsur;
  static constexpr int oGeo = oOps + nOps;
  static constexpr int oFn = oGeo + EB * kGeo;          // [EB][4][4] n, Fscale
  static constexpr int oNbr = oFn + EB * 16;            // int4 [EB]
  static constexpr int oCode = oNbr + EB * 4;           // uint32 [EB]
  static constexpr int oFtab = oCode + EB;              // int [10][Nfp]
  static constexpr int oBar = ((oFtab + 10 * S::Nfp) + 3) & ~3;  // 16-byte aligned mbarrier
  static constexpr int nFloats = oBar + 4;
  static constexpr size_t bytes = size_t(nFloats) * 4;
};

// ---------------------------------------------------------------- kernel
template <int MODEL, int N, int EB, int TN, int NT, bool OPS_SMEM>
__global__ void __launch_bounds__(NT) dg_step_kernel(const StepArgs a) {
  using S = Sz<N>;
  using P = Plan<MODEL, N, EB, OPS_SMEM>;
  constexpr int Np = S::Np, Nfp = S::Nfp, NFN = S::NFN, Mpad = S::Mpad, RT = S::RT;
  constexpr int Nf = P::Nf;
  constexpr int CT = EB / TN;
  static_assert(EB % TN == 0, "EB must be a multiple of TN");
  static_assert(EB % 4 == 0, "EB must be a multiple of 4 (TMA 16-byte granularity)");
  static_assert(RT * CT <= NT, "one output tile per thread");

  extern __shared__ __align__(16) float smem[];
  float* sQ = smem + P::oQ;
  float* sXv = smem + P::oXvol;
  float* sXs = smem + P::oXsur;
  const float* sOps = OPS_SMEM ? smem + P::oOps : a.ops;
  float* sGeo = smem + P::oGeo;
  float* sFn = smem + P::oFn;
  int4* sNbr = reinterpret_cast<int4*>(smem + P::oNbr);
  uint32_t* sCode = reinterpret_cast<uint32_t*>(smem + P::oCode);
  int* sFtab = reinterpret_cast<int*>(smem + P::oFtab);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + P::oBar);

  const int tid = threadIdx.x;
  const int k0 = blockIdx.x * EB;

  // -------- stage 1: TMA bulk loads
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0) {
    const uint32_t bq = uint32_t(EB * Nf * Np * 4), bg = uint32_t(EB * kGeo * 4);
    const uint32_t bn = uint32_t(EB * 16), bc = uint32_t(EB * 4);
    const uint32_t bo = OPS_SMEM ? uint32_t(S::KD * Mpad * 4) : 0u;
    mbar_arrive_expect_tx(bar, bq + bg + bn + bc + bo);
    tma_bulk_g2s(sQ, a.q + size_t(k0) * Nf * Np, bq, bar);
    tma_bulk_g2s(sGeo, a.geo + size_t(k0) * kGeo, bg, bar);
    tma_bulk_g2s(sNbr, a.nbr + k0, bn, bar);
    tma_bulk_g2s(sCode, a.code + k0, bc, bar);
    if (OPS_SMEM) tma_bulk_g2s(smem + P::oOps, a.ops, bo, bar);
  }
  for (int i = tid; i < 10 * Nfp; i += NT) sFtab[i] = a.ftab[i];
  if (!mbar_wait_bounded(bar, 0, a.err)) {
    // the copies may still be in flight: wait once more (bounded) before leaving
    mbar_wait_bounded(bar, 0, nullptr);
    return;
  }
  __syncthreads();

  // -------- stage 2a: face normals and Fscale  (n = g N_f / |g N_f|)
  for (int it = tid; it < EB * 4; it += NT) {
    const int e = it >> 2, f = it & 3;
    const float* gk = sGeo + e * kGeo;
    float nv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      nv[i] = gk[3 * i] * ref_normal(f, 0) + gk[3 * i + 1] * ref_normal(f, 1) + gk[3 * i + 2] * ref_normal(f, 2);
    const float fs = sqrtf(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    const float inv = 1.0f / fs;
    float* o = sFn + it * 4;
    o[0] = nv[0] * inv;
    o[1] = nv[1] * inv;
    o[2] = nv[2] * inv;
    o[3] = fs;
  }
  // -------- stage 2b: volume inputs
  for (int it = tid; it < EB * Np; it += NT) {
    const int e = it % EB, j = it / EB;  // e fastest: conflict-free column writes
    const float* gk = sGeo + e * kGeo;
    const float* qe = sQ + e * Nf * Np;
    if constexpr (MODEL == 0) {
      const float kap = gk[9];
      const float v0 = qe[Np + j], v1 = qe[2 * Np + j], v2 = qe[3 * Np + j];
      sXv[(0 * Np + j) * EB + e] = qe[j];
#pragma unroll
      for (int d = 0; d < 3; ++d)
        sXv[((1 + d) * Np + j) * EB + e] = -kap * (gk[d] * v0 + gk[3 + d] * v1 + gk[6 + d] * v2);
    } else {
      const float rinv = gk[11];
      float sg[3][3];
      sg[0][0] = qe[3 * Np + j]; sg[1][1] = qe[4 * Np + j]; sg[2][2] = qe[5 * Np + j];
      sg[0][1] = sg[1][0] = qe[6 * Np + j];
      sg[0][2] = sg[2][0] = qe[7 * Np + j];
      sg[1][2] = sg[2][1] = qe[8 * Np + j];
#pragma unroll
      for (int c = 0; c < 3; ++c) sXv[(c * Np + j) * EB + e] = qe[c * Np + j];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d)
          sXv[((3 + 3 * c + d) * Np + j) * EB + e] =
              rinv * (gk[d] * sg[c][0] + gk[3 + d] * sg[c][1] + gk[6 + d] * sg[c][2]);
    }
  }
  __syncthreads();  // sFn ready for the flux stage

  // -------- stage 2c: traces and penalty terms at the 4 Nfp face nodes
  for (int it = tid; it < EB * NFN; it += NT) {
    const int e = it % EB, fm = it / EB;
    const int f = fm / Nfp, m = fm - f * Nfp;
    const int nM = sFtab[f * Nfp + m];
    const float* qe = sQ + e * Nf * Np;
    const float* fn = sFn + (e * 4 + f) * 4;
    const float nx = fn[0], ny = fn[1], nz = fn[2], fs = fn[3];
    const uint32_t cw = (sCode[e] >> (8 * f)) & 0xffu;
    const int kn = (f == 0) ? sNbr[e].x : (f == 1) ? sNbr[e].y : (f == 2) ? sNbr[e].z : sNbr[e].w;
    const bool bnd = (cw & 0x80u) || kn < 0;
    float qP[Nf];
    float qM[Nf];
#pragma unroll
    for (int c = 0; c < Nf; ++c) qM[c] = qe[c * Np + nM];
    const float* gM = sGeo + e * kGeo;
    float zP0 = 0.f, zP1 = 0.f;
    if (!bnd) {
      const int f2 = int(cw & 3u), rot = int((cw >> 2) & 7u);
      const int nP = sFtab[f2 * Nfp + sFtab[4 * Nfp + rot * Nfp + m]];
      const int le = kn - k0;
      if (le >= 0 && le < EB) {
        const float* qn = sQ + le * Nf * Np;
#pragma unroll
        for (int c = 0; c < Nf; ++c) qP[c] = qn[c * Np + nP];
        zP0 = sGeo[le * kGeo + (MODEL == 0 ? 11 : 12)];
        if (MODEL == 1) zP1 = sGeo[le * kGeo + 13];
      } else {
        const float* qn = a.q + size_t(kn) * Nf * Np;
#pragma unroll
        for (int c = 0; c < Nf; ++c) qP[c] = __ldg(qn + c * Np + nP);
        zP0 = __ldg(a.geo + size_t(kn) * kGeo + (MODEL == 0 ? 11 : 12));
        if (MODEL == 1) zP1 = __ldg(a.geo + size_t(kn) * kGeo + 13);
      }
    }
    if constexpr (MODEL == 0) {
      const float kap = gM[9], rinv = gM[10], ZM = gM[11], cM = gM[12];
      if (bnd) {  // rigid wall: p+ = p-, v+ = v- - 2 (v-.n) n
        const float vn = qM[1] * nx + qM[2] * ny + qM[3] * nz;
        qP[0] = qM[0];
        qP[1] = qM[1] - 2.f * vn * nx;
        qP[2] = qM[2] - 2.f * vn * ny;
        qP[3] = qM[3] - 2.f * vn * nz;
        zP0 = ZM;
      }
      const float jp = 0.5f * (qP[0] - qM[0]);
      const float jvn = 0.5f * ((qP[1] - qM[1]) * nx + (qP[2] - qM[2]) * ny + (qP[3] - qM[3]) * nz);
      float dp, sv;  // dv = sv * n
      if (a.flux == 0) {
        const float kc = 2.f / (ZM + zP0);
        const float ac = jp - zP0 * jvn;
        dp = kap * kc * ac;
        sv = -cM * kc * ac;
      } else {
        dp = -kap * jvn;
        sv = -rinv * jp;
      }
      float* X = sXs + fm * EB + e;
      X[0] = fs * dp;
      X[NFN * EB] = fs * sv * nx;
      X[2 * NFN * EB] = fs * sv * ny;
      X[3 * NFN * EB] = fs * sv * nz;
    } else {
      const float lam = gM[9], mu = gM[10], rinv = gM[11], ZpM = gM[12], ZsM = gM[13], cpM = gM[14],
                  csM = gM[15];
      if (bnd) {
        const float sv = (a.bc == 0) ? 1.f : -1.f;  // free: v+ = v-, sigma+ = -sigma-
#pragma unroll
        for (int c = 0; c < 3; ++c) qP[c] = sv * qM[c];
#pragma unroll
        for (int c = 3; c < 9; ++c) qP[c] = -sv * qM[c];
        zP0 = ZpM;
        zP1 = ZsM;
      }
      const float n[3] = {nx, ny, nz};
      float jv[3], jt[3];
      const float ds[6] = {qP[3] - qM[3], qP[4] - qM[4], qP[5] - qM[5],
                           qP[6] - qM[6], qP[7] - qM[7], qP[8] - qM[8]};
      // [[sigma n]] = (sigma+ - sigma-) n / 2 ; order sxx syy szz sxy sxz syz
      jt[0] = 0.5f * (ds[0] * nx + ds[3] * ny + ds[4] * nz);
      jt[1] = 0.5f * (ds[3] * nx + ds[1] * ny + ds[5] * nz);
      jt[2] = 0.5f * (ds[4] * nx + ds[5] * ny + ds[2] * nz);
#pragma unroll
      for (int c = 0; c < 3; ++c) jv[c] = 0.5f * (qP[c] - qM[c]);
      float pv[3], dv[3];  // p_v and the velocity jump that P_sigma = C:sym(n (x) dv) uses
      if (a.flux == 0) {
        const float jsnn = jt[0] * nx + jt[1] * ny + jt[2] * nz;
        const float jvn = jv[0] * nx + jv[1] * ny + jv[2] * nz;
        const float ap = jsnn + zP0 * jvn;
        const float as = jsnn + zP1 * jvn;
        const float kp = 2.f / (ZpM + zP0), ks = 2.f / (ZsM + zP1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float asv = jt[c] + zP1 * jv[c];
          const float tang = asv - as * n[c];
          dv[c] = kp * ap * n[c] + ks * tang;
          pv[c] = kp * ap * cpM * n[c] + ks * csM * tang;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          dv[c] = jv[c];
          pv[c] = rinv * jt[c];
        }
      }
      // P_sigma = lambda (n.dv) I + 2 mu sym(n (x) dv)
      const float ndv = nx * dv[0] + ny * dv[1] + nz * dv[2];
      float* X = sXs + fm * EB + e;
      X[0 * NFN * EB] = fs * pv[0];
      X[1 * NFN * EB] = fs * pv[1];
      X[2 * NFN * EB] = fs * pv[2];
      X[3 * NFN * EB] = fs * (lam * ndv + 2.f * mu * nx * dv[0]);
      X[4 * NFN * EB] = fs * (lam * ndv + 2.f * mu * ny * dv[1]);
      X[5 * NFN * EB] = fs * (lam * ndv + 2.f * mu * nz * dv[2]);
      X[6 * NFN * EB] = fs * (mu * (nx * dv[1] + ny * dv[0]));
      X[7 * NFN * EB] = fs * (mu * (nx * dv[2] + nz * dv[0]));
      X[8 * NFN * EB] = fs * (mu * (ny * dv[2] + nz * dv[1]));
    }
  }
  __syncthreads();

  // -------- stage 3: register-tiled operator products
  if (tid >= RT * CT) return;
  const int rt = tid % RT, ct = tid / RT;
  const int i0 = 4 * rt, e0 = TN * ct;
  const float* A = sOps + i0;

  if constexpr (MODEL == 0) {
    float G[3][TN][4], R[TN][4], L[3][TN][4];
#pragma unroll
    for (int t = 0; t < TN; ++t)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        R[t][u] = 0.f;
#pragma unroll
        for (int d = 0; d < 3; ++d) G[d][t][u] = L[d][t][u] = 0.f;
      }
    // volume: G_d = D_d p ;  R = sum_d D_d w_d
#pragma unroll 2
    for (int j = 0; j < Np; ++j) {
      const float4 a0 = load_op<OPS_SMEM>(A + (0 * Np + j) * Mpad);
      const float4 a1 = load_op<OPS_SMEM>(A + (1 * Np + j) * Mpad);
      const float4 a2 = load_op<OPS_SMEM>(A + (2 * Np + j) * Mpad);
      float xp[TN], x0[TN], x1[TN], x2[TN];
      VecT<TN>::load(sXv + (0 * Np + j) * EB + e0, xp);
      VecT<TN>::load(sXv + (1 * Np + j) * EB + e0, x0);
      VecT<TN>::load(sXv + (2 * Np + j) * EB + e0, x1);
      VecT<TN>::load(sXv + (3 * Np + j) * EB + e0, x2);
#pragma unroll
      for (int t = 0; t < TN; ++t) {
        fma4(G[0][t], a0, xp[t]);
        fma4(G[1][t], a1, xp[t]);
        fma4(G[2][t], a2, xp[t]);
        fma4(R[t], a0, x0[t]);
        fma4(R[t], a1, x1[t]);
        fma4(R[t], a2, x2[t]);
      }
    }
    // surface: merged LIFT
#pragma unroll 2
    for (int c = 0; c < NFN; ++c) {
      const float4 l = load_op<OPS_SMEM>(A + (3 * Np + c) * Mpad);
      float pp[TN], p0[TN], p1[TN], p2[TN];
      VecT<TN>::load(sXs + (0 * NFN + c) * EB + e0, pp);
      VecT<TN>::load(sXs + (1 * NFN + c) * EB + e0, p0);
      VecT<TN>::load(sXs + (2 * NFN + c) * EB + e0, p1);
      VecT<TN>::load(sXs + (3 * NFN + c) * EB + e0, p2);
#pragma unroll
      for (int t = 0; t < TN; ++t) {
        fma4(R[t], l, pp[t]);
        fma4(L[0][t], l, p0[t]);
        fma4(L[1][t], l, p1[t]);
        fma4(L[2][t], l, p2[t]);
      }
    }
    // epilogue: geometric combination + source + AB3 / store
#pragma unroll
    for (int t = 0; t < TN; ++t) {
      const int e = e0 + t;
      const int k = k0 + e;
      if (k >= a.K) continue;
      const float* gk = sGeo + e * kGeo;
      const float rinv = gk[10];
      const bool src = (k == a.src_elem) && a.srcvec;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u;
        if (i >= Np) continue;
        float r[4];
        r[0] = R[t][u];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          r[1 + c] = L[c][t][u] - rinv * (gk[3 * c] * G[0][t][u] + gk[3 * c + 1] * G[1][t][u] +
                                          gk[3 * c + 2] * G[2][t][u]);
        if (src) {
#pragma unroll
          for (int c = 0; c < 4; ++c) r[c] = fmaf(a.src_amp, __ldg(a.srcvec + c * Np + i), r[c]);
        }
        const size_t base = size_t(k) * Nf * Np + i;
        if (a.mode == 0) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const size_t idx = base + c * Np;
            const float qv = sQ[e * Nf * Np + c * Np + i];
            const float acc = a.a1 * r[c] + a.a2 * a.r1[idx] + a.a3 * a.r2[idx];
            a.qn[idx] = fmaf(a.dt, acc, qv);
            a.r2[idx] = r[c];
          }
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) a.rout[base + c * Np] = r[c];
        }
      }
    }
  } else {
    // elastic: U_cd = D_d v_c ; Rv_c = sum_d D_d s_cd
    float U[3][3][TN][4], Rv[3][TN][4];
#pragma unroll
    for (int t = 0; t < TN; ++t)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Rv[c][t][u] = 0.f;
#pragma unroll
          for (int d = 0; d < 3; ++d) U[c][d][t][u] = 0.f;
        }
#pragma unroll 1
    for (int j = 0; j < Np; ++j) {
      float4 ad[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) ad[d] = load_op<OPS_SMEM>(A + (d * Np + j) * Mpad);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float xv[TN];
        VecT<TN>::load(sXv + (c * Np + j) * EB + e0, xv);
#pragma unroll
        for (int t = 0; t < TN; ++t)
#pragma unroll
          for (int d = 0; d < 3; ++d) fma4(U[c][d][t], ad[d], xv[t]);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          float xs[TN];
          VecT<TN>::load(sXv + ((3 + 3 * c + d) * Np + j) * EB + e0, xs);
#pragma unroll
          for (int t = 0; t < TN; ++t) fma4(Rv[c][t], ad[d], xs[t]);
        }
      }
    }
    // stress volume terms from the velocity gradient
    float Rs[6][TN][4];
#pragma unroll
    for (int t = 0; t < TN; ++t) {
      const float* gk = sGeo + (e0 + t) * kGeo;
      const float lam = gk[9], mu = gk[10];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float gv[3][3];  // gv[c][x] = d v_c / d x_x = sum_d g[x][d] U[c][d]
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int x = 0; x < 3; ++x)
            gv[c][x] = gk[3 * x] * U[c][0][t][u] + gk[3 * x + 1] * U[c][1][t][u] + gk[3 * x + 2] * U[c][2][t][u];
        const float div = gv[0][0] + gv[1][1] + gv[2][2];
        Rs[0][t][u] = lam * div + 2.f * mu * gv[0][0];
        Rs[1][t][u] = lam * div + 2.f * mu * gv[1][1];
        Rs[2][t][u] = lam * div + 2.f * mu * gv[2][2];
        Rs[3][t][u] = mu * (gv[0][1] + gv[1][0]);
        Rs[4][t][u] = mu * (gv[0][2] + gv[2][0]);
        Rs[5][t][u] = mu * (gv[1][2] + gv[2][1]);
      }
    }
#pragma unroll 1
    for (int c = 0; c < NFN; ++c) {
      const float4 l = load_op<OPS_SMEM>(A + (3 * Np + c) * Mpad);
#pragma unroll
      for (int fld = 0; fld < 3; ++fld) {
        float p[TN];
        VecT<TN>::load(sXs + (fld * NFN + c) * EB + e0, p);
#pragma unroll
        for (int t = 0; t < TN; ++t) fma4(Rv[fld][t], l, p[t]);
      }
#pragma unroll
      for (int fld = 0; fld < 6; ++fld) {
        float p[TN];
        VecT<TN>::load(sXs + ((3 + fld) * NFN + c) * EB + e0, p);
#pragma unroll
        for (int t = 0; t < TN; ++t) fma4(Rs[fld][t], l, p[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < TN; ++t) {
      const int e = e0 + t;
      const int k = k0 + e;
      if (k >= a.K) continue;
      const bool src = (k == a.src_elem) && a.srcvec;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u;
        if (i >= Np) continue;
        float r[9];
#pragma unroll
        for (int c = 0; c < 3; ++c) r[c] = Rv[c][t][u];
#pragma unroll
        for (int c = 0; c < 6; ++c) r[3 + c] = Rs[c][t][u];
        if (src) {
#pragma unroll
          for (int c = 0; c < 9; ++c) r[c] = fmaf(a.src_amp, __ldg(a.srcvec + c * Np + i), r[c]);
        }
        const size_t base = size_t(k) * Nf * Np + i;
        if (a.mode == 0) {
#pragma unroll
          for (int c = 0; c < 9; ++c) {
            const size_t idx = base + c * Np;
            const float qv = sQ[e * Nf * Np + c * Np + i];
            const float acc = a.a1 * r[c] + a.a2 * a.r1[idx] + a.a3 * a.r2[idx];
            a.qn[idx] = fmaf(a.dt, acc, qv);
            a.r2[idx] = r[c];
          }
        } else {
#pragma unroll
          for (int c = 0; c < 9; ++c) a.rout[base + c * Np] = r[c];
        }
      }
    }
  }
}

}  // namespace dgk
