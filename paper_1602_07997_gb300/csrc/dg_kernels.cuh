// Fused nodal-DG step kernels for sm_103a (FP32 CUDA-core path).
//
// Persistent CTAs walk blocks of EB consecutive elements (block b, b + grid,
// ...).  Per block:
//   1. its fields q^m [EB][Nf][Np], element records and neighbour words were
//      bulk-copied into shared memory stage s during the previous block
//      (1-D TMA: cp.async.bulk + mbarrier, bounded wait); the copy of the
//      next block into stage s^1, and of this block's AB3 history r^{m-1},
//      r^{m-2} into shared memory, are issued now and land while it computes;
//   2. face normals and Fscale = |g N_f| from the inverse metric;
//   3. element-wise GEMM inputs in shared memory, element index fastest:
//      volume inputs (acoustic p and w_d = -kappa sum_c g_cd v_c; elastic v_c
//      and s_cd = (1/rho) sum_m g_md sigma_cm) and the Fscale-weighted
//      penalty terms at the 4 Nfp face nodes (own trace via the face mask,
//      neighbour trace via the neighbour's face mask and one of the 6 face
//      rotations; neighbours in the block come from shared memory, the
//      others from global memory, several face nodes per thread in flight);
//   4. each thread owns tiles of 4 output nodes x TN elements and
//      accumulates every operator product of its tile in registers
//      (Section 3.2: 6 Np x Np products + the merged LIFT product for the
//      acoustic model, 18 + LIFT for the elastic model), operator rows as
//      float4 from shared memory (or L1 when the blob exceeds the budget);
//   5. epilogue from registers: geometric combination, point source, and the
//      AB3 update (Eq. updateScheme) q^{m+1} = q^m + dt (a1 r^m + a2 r^{m-1}
//      + a3 r^{m-2}); r^m overwrites r^{m-2} in global memory (read before
//      written, same thread), q^{m+1} goes to the other ping-pong buffer
//      because neighbours still read q^m.
//
// RHS (Eq. dgLocalRhs) in the form computed here (g_cd = dr_d/dx_c):
//   acoustic: r_p   = sum_d D_d w_d + LIFT (Fscale dp)
//             r_v_c = -(1/rho) sum_d g_cd (D_d p) + LIFT (Fscale dv_c)
//   elastic:  r_v_c = sum_d D_d s_cd + LIFT (Fscale p_v,c)
//             r_sig_ij = lambda delta_ij div v + mu (dv_i/dx_j + dv_j/dx_i)
//                        + LIFT (Fscale P_sig,ij),  dv_i/dx_j = sum_d g_jd (D_d v_i)
// with the penalty terms of Section 2.1.
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
template <int MODEL, int N, int EB, bool OPS_SMEM, bool R_SMEM>
struct Plan {
  using S = Sz<N>;
  static constexpr int Nf = MODEL == 0 ? 4 : 9;
  static constexpr int REC = Rec<MODEL>::size;
  static constexpr int nQ = EB * Nf * S::Np;
  static constexpr int nStage = nQ + EB * REC + EB * 4;  // q, records, neighbour words
  static constexpr int nR = R_SMEM ? 2 * nQ : 0;
  static constexpr int nXvol = (MODEL == 0 ? 4 : 12) * S::Np * EB;
  static constexpr int nXsur = Nf * S::NFN * EB;
  static constexpr int nOps = OPS_SMEM ? S::KD * S::Mpad : 0;
  static constexpr int oStage0 = 0;
  static constexpr int oStage1 = oStage0 + nStage;
  static constexpr int oR = oStage1 + nStage;
  static constexpr int oXvol = oR + nR;
  static constexpr int oXsur = oXvol + nXvol;
  static constexpr int oOps = oXsur + nXsur;
  static constexpr int oFn = oOps + nOps;                 // [EB][4][4] n, Fscale
  static constexpr int oFtab = oFn + EB * 16;              // int [10][Nfp]
  static constexpr int oBar = ((oFtab + 10 * S::Nfp) + 3) & ~3;
  static constexpr int nFloats = oBar + 8;                 // 3 mbarriers
  static constexpr size_t bytes = size_t(nFloats) * 4;
  // offsets inside a stage
  static constexpr int sQ = 0, sRec = nQ, sNbr = nQ + EB * REC;
  static_assert((nQ % 4) == 0 && ((EB * REC) % 4) == 0, "16-byte aligned stage pieces");
};

// ---------------------------------------------------------------- kernel
template <int MODEL, int N, int EB, int TN, int NT, bool OPS_SMEM, bool R_SMEM>
__global__ void __launch_bounds__(NT) dg_step_kernel(const StepArgs a) {
  using S = Sz<N>;
  using P = Plan<MODEL, N, EB, OPS_SMEM, R_SMEM>;
  constexpr int Np = S::Np, Nfp = S::Nfp, NFN = S::NFN, Mpad = S::Mpad, RT = S::RT;
  constexpr int Nf = P::Nf, REC = P::REC;
  constexpr int CT = EB / TN;
  constexpr int NTILE = RT * CT;
  static_assert(EB % TN == 0, "EB must be a multiple of TN");
  static_assert(EB % 4 == 0, "EB must be a multiple of 4 (TMA 16-byte granularity)");

  extern __shared__ __align__(16) float smem[];
  float* sR = smem + P::oR;
  float* sXv = smem + P::oXvol;
  float* sXs = smem + P::oXsur;
  const float* sOps = OPS_SMEM ? smem + P::oOps : a.ops;
  float* sFn = smem + P::oFn;
  int* sFtab = reinterpret_cast<int*>(smem + P::oFtab);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P::oBar);

  const int tid = threadIdx.x;
  const int nblk = (a.K + EB - 1) / EB;
  const int G = gridDim.x;
  constexpr uint32_t kStageBytes = uint32_t((P::nQ + EB * REC + EB * 4) * 4);
  constexpr uint32_t kQBytes = uint32_t(P::nQ * 4);

  auto issue_stage = [&](int b, int s, bool with_ops) {
    float* st = smem + (s ? P::oStage1 : P::oStage0);
    const int k0 = b * EB;
    const uint32_t bo = (OPS_SMEM && with_ops) ? uint32_t(S::KD * Mpad * 4) : 0u;
    mbar_arrive_expect_tx(&bars[s], kStageBytes + bo);
    tma_bulk_g2s(st + P::sQ, a.q + size_t(k0) * Nf * Np, kQBytes, &bars[s]);
    tma_bulk_g2s(st + P::sRec, a.rec + size_t(k0) * REC, uint32_t(EB * REC * 4), &bars[s]);
    tma_bulk_g2s(st + P::sNbr, a.nbr + k0, uint32_t(EB * 16), &bars[s]);
    if (OPS_SMEM && with_ops) tma_bulk_g2s(smem + P::oOps, a.ops, bo, &bars[s]);
  };

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid == 0 && (int)blockIdx.x < nblk) issue_stage(blockIdx.x, 0, true);
  for (int i = tid; i < 10 * Nfp; i += NT) sFtab[i] = a.ftab[i];

  int it = 0;
  for (int b = blockIdx.x; b < nblk; b += G, ++it) {
    const int s = it & 1;
    const int k0 = b * EB;
    bool ok = mbar_wait_bounded(&bars[s], uint32_t((it >> 1) & 1), a.err);
    if (!__syncthreads_and(ok)) {
      mbar_wait_bounded(&bars[s], uint32_t((it >> 1) & 1), nullptr);
      return;
    }
    // everyone is past the previous block: stage s^1, the history buffer and X are free
    const float* sQ = smem + (s ? P::oStage1 : P::oStage0) + P::sQ;
    const float* sRec = smem + (s ? P::oStage1 : P::oStage0) + P::sRec;
    const int4* sNbr = reinterpret_cast<const int4*>(smem + (s ? P::oStage1 : P::oStage0) + P::sNbr);
    if (tid == 0) {
      if (b + G < nblk) issue_stage(b + G, s ^ 1, false);
      if (R_SMEM && a.mode == 0) {
        mbar_arrive_expect_tx(&bars[2], 2 * kQBytes);
        tma_bulk_g2s(sR, a.r1 + size_t(k0) * Nf * Np, kQBytes, &bars[2]);
        tma_bulk_g2s(sR + P::nQ, a.r2 + size_t(k0) * Nf * Np, kQBytes, &bars[2]);
      }
    }

    // -------- face normals and Fscale (n = g N_f / |g N_f|)
    for (int i = tid; i < EB * 4; i += NT) {
      const int e = i >> 2, f = i & 3;
      const float* gk = sRec + e * REC;
      float nv[3];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        nv[c] = gk[3 * c] * ref_normal(f, 0) + gk[3 * c + 1] * ref_normal(f, 1) + gk[3 * c + 2] * ref_normal(f, 2);
      const float fs = sqrtf(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
      const float inv = 1.0f / fs;
      float4 o = make_float4(nv[0] * inv, nv[1] * inv, nv[2] * inv, fs);
      *reinterpret_cast<float4*>(sFn + i * 4) = o;
    }
    // -------- volume inputs
    for (int i = tid; i < EB * Np; i += NT) {
      const int e = i % EB, j = i / EB;
      const float* gk = sRec + e * REC;
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
    __syncthreads();  // sFn ready

    // -------- traces and penalty terms at the 4 Nfp face nodes
    constexpr int BATCH = MODEL == 0 ? 4 : 2;
    for (int base = tid; base < EB * NFN; base += NT * BATCH) {
      float qP[BATCH][Nf];
      int nMv[BATCH], bndv[BATCH];
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int i = base + u * NT;
        bndv[u] = 1;
        nMv[u] = 0;
        if (i >= EB * NFN) continue;
        const int e = i % EB, fm = i / EB;
        const int f = fm / Nfp, m = fm - f * Nfp;
        nMv[u] = sFtab[f * Nfp + m];
        const int4 nb = sNbr[e];
        const int w = (f == 0) ? nb.x : (f == 1) ? nb.y : (f == 2) ? nb.z : nb.w;
        if (w < 0) continue;
        bndv[u] = 0;
        const int kn = w >> kNbrShift, rot = (w >> 2) & 7, f2 = w & 3;
        const int nP = sFtab[f2 * Nfp + sFtab[4 * Nfp + rot * Nfp + m]];
        const int le = kn - k0;
        if (le >= 0 && le < EB) {
          const float* qn = sQ + le * Nf * Np;
#pragma unroll
          for (int c = 0; c < Nf; ++c) qP[u][c] = qn[c * Np + nP];
        } else {
          const float* qn = a.q + size_t(kn) * Nf * Np;
#pragma unroll
          for (int c = 0; c < Nf; ++c) qP[u][c] = __ldg(qn + c * Np + nP);
        }
      }
#pragma unroll
      for (int u = 0; u < BATCH; ++u) {
        const int i = base + u * NT;
        if (i >= EB * NFN) continue;
        const int e = i % EB, fm = i / EB;
        const int f = fm / Nfp;
        const int nM = nMv[u];
        const bool bnd = bndv[u] != 0;
        const float* qe = sQ + e * Nf * Np;
        const float4 fn = *reinterpret_cast<const float4*>(sFn + (e * 4 + f) * 4);
        const float nx = fn.x, ny = fn.y, nz = fn.z, fs = fn.w;
        const float* gM = sRec + e * REC;
        float qM[Nf];
#pragma unroll
        for (int c = 0; c < Nf; ++c) qM[c] = qe[c * Np + nM];
        float* X = sXs + fm * EB + e;
        if constexpr (MODEL == 0) {
          const float kap = gM[9], rinv = gM[10], ZM = gM[11], zP = gM[12 + f];
          float pP, vP0, vP1, vP2;
          if (bnd) {  // rigid wall: p+ = p-, v+ = v- - 2 (v-.n) n
            const float vn = qM[1] * nx + qM[2] * ny + qM[3] * nz;
            pP = qM[0];
            vP0 = qM[1] - 2.f * vn * nx;
            vP1 = qM[2] - 2.f * vn * ny;
            vP2 = qM[3] - 2.f * vn * nz;
          } else {
            pP = qP[u][0]; vP0 = qP[u][1]; vP1 = qP[u][2]; vP2 = qP[u][3];
          }
          const float jp = 0.5f * (pP - qM[0]);
          const float jvn = 0.5f * ((vP0 - qM[1]) * nx + (vP1 - qM[2]) * ny + (vP2 - qM[3]) * nz);
          float dp, sv;  // dv = sv * n
          if (a.flux == 0) {
            const float kc = 2.f / (ZM + zP);
            const float ac = jp - zP * jvn;
            dp = kap * kc * ac;
            sv = -(ZM * rinv) * kc * ac;  // c^- = Z^- / rho^-
          } else {
            dp = -kap * jvn;
            sv = -rinv * jp;
          }
          X[0] = fs * dp;
          X[NFN * EB] = fs * sv * nx;
          X[2 * NFN * EB] = fs * sv * ny;
          X[3 * NFN * EB] = fs * sv * nz;
        } else {
          const float lam = gM[9], mu = gM[10], rinv = gM[11], ZpM = gM[12], ZsM = gM[13], cpM = gM[14],
                      csM = gM[15], zP0 = gM[16 + f], zP1 = gM[20 + f];
          float vP[3], sPd[6];
          if (bnd) {
            const float sv = (a.bc == 0) ? 1.f : -1.f;  // free: v+ = v-, sigma+ = -sigma-
#pragma unroll
            for (int c = 0; c < 3; ++c) vP[c] = sv * qM[c];
#pragma unroll
            for (int c = 0; c < 6; ++c) sPd[c] = -sv * qM[3 + c];
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) vP[c] = qP[u][c];
#pragma unroll
            for (int c = 0; c < 6; ++c) sPd[c] = qP[u][3 + c];
          }
          const float n[3] = {nx, ny, nz};
          float ds[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) ds[c] = sPd[c] - qM[3 + c];
          float jt[3], jv[3];  // [[sigma n]], [[v]]  (sxx syy szz sxy sxz syz)
          jt[0] = 0.5f * (ds[0] * nx + ds[3] * ny + ds[4] * nz);
          jt[1] = 0.5f * (ds[3] * nx + ds[1] * ny + ds[5] * nz);
          jt[2] = 0.5f * (ds[4] * nx + ds[5] * ny + ds[2] * nz);
#pragma unroll
          for (int c = 0; c < 3; ++c) jv[c] = 0.5f * (vP[c] - qM[c]);
          float pv[3], dv[3];  // p_v and the velocity jump with P_sigma = C:sym(n (x) dv)
          if (a.flux == 0) {
            const float jsnn = jt[0] * nx + jt[1] * ny + jt[2] * nz;
            const float jvn = jv[0] * nx + jv[1] * ny + jv[2] * nz;
            const float ap = jsnn + zP0 * jvn;
            const float as = jsnn + zP1 * jvn;
            const float kp = 2.f / (ZpM + zP0), ks = 2.f / (ZsM + zP1);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float tang = (jt[c] + zP1 * jv[c]) - as * n[c];
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
          const float ndv = nx * dv[0] + ny * dv[1] + nz * dv[2];
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
    }
    __syncthreads();
    if (R_SMEM && a.mode == 0) {
      bool okr = mbar_wait_bounded(&bars[2], uint32_t(it & 1), a.err);
      if (!__syncthreads_and(okr)) {
        mbar_wait_bounded(&bars[2], uint32_t(it & 1), nullptr);
        return;
      }
    }

    // -------- register-tiled operator products + epilogue
    for (int tile = tid; tile < NTILE; tile += NT) {
      const int rt = tile % RT, ct = tile / RT;
      const int i0 = 4 * rt, e0 = TN * ct;
      const float* A = sOps + i0;
      if constexpr (MODEL == 0) {
        float G[3][TN][4], R[TN][4], L[3][TN][4];
#pragma unroll
        for (int t = 0; t < TN; ++t)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            R[t][v] = 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) G[d][t][v] = L[d][t][v] = 0.f;
          }
#pragma unroll 4
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
#pragma unroll 4
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
#pragma unroll
        for (int t = 0; t < TN; ++t) {
          const int e = e0 + t;
          const int k = k0 + e;
          if (k >= a.K) continue;
          const float* gk = sRec + e * REC;
          const float rinv = gk[10];
          const bool src = (k == a.src_elem) && a.srcvec;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int i = i0 + v;
            if (i >= Np) continue;
            float r[4];
            r[0] = R[t][v];
#pragma unroll
            for (int c = 0; c < 3; ++c)
              r[1 + c] = L[c][t][v] - rinv * (gk[3 * c] * G[0][t][v] + gk[3 * c + 1] * G[1][t][v] +
                                              gk[3 * c + 2] * G[2][t][v]);
            if (src) {
#pragma unroll
              for (int c = 0; c < 4; ++c) r[c] = fmaf(a.src_amp, __ldg(a.srcvec + c * Np + i), r[c]);
            }
            const size_t base = size_t(k) * Nf * Np + i;
            if (a.mode == 0) {
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const int li = e * Nf * Np + c * Np + i;
                const float r1v = R_SMEM ? sR[li] : __ldg(a.r1 + base + c * Np);
                const float r2v = R_SMEM ? sR[P::nQ + li] : a.r2[base + c * Np];
                const float acc = a.a1 * r[c] + a.a2 * r1v + a.a3 * r2v;
                a.qn[base + c * Np] = fmaf(a.dt, acc, sQ[li]);
                a.r2[base + c * Np] = r[c];
              }
            } else {
#pragma unroll
              for (int c = 0; c < 4; ++c) a.rout[base + c * Np] = r[c];
            }
          }
        }
      } else {
        float U[3][3][TN][4], Rv[3][TN][4];
#pragma unroll
        for (int t = 0; t < TN; ++t)
#pragma unroll
          for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              Rv[c][t][v] = 0.f;
#pragma unroll
              for (int d = 0; d < 3; ++d) U[c][d][t][v] = 0.f;
            }
#pragma unroll 2
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
        float Rs[6][TN][4];
#pragma unroll
        for (int t = 0; t < TN; ++t) {
          const float* gk = sRec + (e0 + t) * REC;
          const float lam = gk[9], mu = gk[10];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            float gv[3][3];  // gv[c][x] = d v_c / d x_x = sum_d g[x][d] U[c][d]
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
              for (int x = 0; x < 3; ++x)
                gv[c][x] = gk[3 * x] * U[c][0][t][v] + gk[3 * x + 1] * U[c][1][t][v] + gk[3 * x + 2] * U[c][2][t][v];
            const float div = gv[0][0] + gv[1][1] + gv[2][2];
            Rs[0][t][v] = lam * div + 2.f * mu * gv[0][0];
            Rs[1][t][v] = lam * div + 2.f * mu * gv[1][1];
            Rs[2][t][v] = lam * div + 2.f * mu * gv[2][2];
            Rs[3][t][v] = mu * (gv[0][1] + gv[1][0]);
            Rs[4][t][v] = mu * (gv[0][2] + gv[2][0]);
            Rs[5][t][v] = mu * (gv[1][2] + gv[2][1]);
          }
        }
#pragma unroll 2
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
          for (int v = 0; v < 4; ++v) {
            const int i = i0 + v;
            if (i >= Np) continue;
            float r[9];
#pragma unroll
            for (int c = 0; c < 3; ++c) r[c] = Rv[c][t][v];
#pragma unroll
            for (int c = 0; c < 6; ++c) r[3 + c] = Rs[c][t][v];
            if (src) {
#pragma unroll
              for (int c = 0; c < 9; ++c) r[c] = fmaf(a.src_amp, __ldg(a.srcvec + c * Np + i), r[c]);
            }
            const size_t base = size_t(k) * Nf * Np + i;
            if (a.mode == 0) {
#pragma unroll
              for (int c = 0; c < 9; ++c) {
                const int li = e * Nf * Np + c * Np + i;
                const float r1v = R_SMEM ? sR[li] : __ldg(a.r1 + base + c * Np);
                const float r2v = R_SMEM ? sR[P::nQ + li] : a.r2[base + c * Np];
                const float acc = a.a1 * r[c] + a.a2 * r1v + a.a3 * r2v;
                a.qn[base + c * Np] = fmaf(a.dt, acc, sQ[li]);
                a.r2[base + c * Np] = r[c];
              }
            } else {
#pragma unroll
              for (int c = 0; c < 9; ++c) a.rout[base + c * Np] = r[c];
            }
          }
        }
      }
    }
  }
}

}  // namespace dgk
