// Fused nodal-DG step kernels for sm_103a (FP32 CUDA-core path).
//
// Persistent CTAs walk blocks of EB consecutive elements (block b, b + grid,
// ...).  Per block:
//   1. its fields q^m [EB][Nf][Np], element records and neighbour words were
//      bulk-copied into shared memory stage s during the previous block
//      (1-D TMA: cp.async.bulk + mbarrier, bounded wait); the copy of the
//      next block into stage s^1, and of this block's AB3 history r^{m-1},
//      r^{m-2} into shared memory, are issued now and land while it computes;
//      the traces of the neighbours outside the block arrived during the
//      previous block (4-byte cp.async per face node and field, or, HALO,
//      the whole neighbour by one bulk copy per element face);
//   2. per element face: normal and Fscale = |g N_f| from the inverse metric
//      and, acoustic, the penalty coefficients and the neighbour's source;
//   3. element-wise GEMM inputs in shared memory, element index fastest:
//      volume inputs (acoustic p and w_d = -kappa sum_c g_cd v_c; elastic v_c
//      and s_cd = (1/rho) sum_m g_md sigma_cm) and the Fscale-weighted
//      penalty terms at the 4 Nfp face nodes (own trace via the face mask,
//      neighbour trace via the neighbour's face mask and one of the 6 face
//      rotations; neighbours in the block come from shared memory, the
//      others from the gathered traces); acoustic: two surface streams, the
//      pressure penalty and psi (the velocity penalty is psi n_f);
//   4. each thread owns a tile of 4 output nodes x TN elements (element
//      index fastest across lanes) and accumulates every operator product of
//      its tile in registers
//      (Section 3.2: 6 Np x Np products + the merged LIFT product for the
//      acoustic model, 18 + LIFT for the elastic model), operator rows as
//      float4 from shared memory (or L1 when the blob exceeds the budget);
//   5. epilogue from registers: geometric combination (acoustic: the velocity
//      lift sum_f n_f LIFT_f psi), point source, and the AB3 update (Eq.
//      updateScheme) q^{m+1} = q^m + dt (a1 r^m + a2 r^{m-1} + a3 r^{m-2})
//      over the block staged in shared memory; r^m overwrites r^{m-2},
//      q^{m+1} goes to the other ping-pong buffer because neighbours still
//      read q^m.
// The split step's front half (SPLIT > 0) runs 1-3 and writes the GEMM
// inputs to global memory (FP32: straight from the loops of 2-3, DIRECT;
// tensor cores: BF16 pieces in the tcgen05 operand layout).
//
#pragma once

#include <cuda_bf16.h>
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

// K chunk of a split-step GEMM tile at which the tile's AB3 inputs are
// prefetched into L2: six chunks before the epilogue (or the first chunk).
__host__ __device__ constexpr int ab3_prefetch_chunk(int nch) { return nch > 6 ? nch - 6 : 0; }

// Rows per element of the FP32 split step's GEMM input X: NV volume inputs
// per node, NXS surface streams per face node (acoustic: the pressure penalty
// and psi, the magnitude of the velocity penalty psi n_f; elastic: Fscale p_v
// and Fscale dv, of which the 9 penalties are made with the face normal and
// the Lame coefficients), then the 4 x 3 face-normal components.
template <int MODEL, int N>
struct XRows {
  static constexpr int NV = MODEL == 0 ? 4 : 12;
  static constexpr int NXS = MODEL == 0 ? 2 : 6;
  static constexpr int KXM = NV * Sz<N>::Np + NXS * Sz<N>::NFN;
  static constexpr int KX = KXM + 12;
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
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// raise the transaction count of the current phase without arriving
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
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
// Bounded wait: gives up after `limit` clock cycles (0 = the default 2^31,
// about a second) and sets bit 0 of the error word.  limit < 0 gives up at
// once without looking at the barrier (a test hook: every first wait of a
// kernel expires).  Returns false on expiry.  Drains after an expiry always
// use the default limit.
constexpr long long kWaitLimit = 1ll << 31;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err,
                                                  long long limit = kWaitLimit) {
  if (limit < 0) {
    if (err) atomicOr(err, 1);
    return false;
  }
  const long long lim = limit > 0 ? limit : kWaitLimit;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > lim) {
      if (err) atomicOr(err, 1);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void tma_bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
constexpr int round4(int x) { return (x + 3) & ~3; }

// FACT (acoustic, FP32 paths): the surface inputs are two streams per face
// node, the pressure penalty and the magnitude psi of the velocity penalty
// psi n_f (n_f is constant on a face of a straight-sided tetrahedron), plus
// per-face penalty coefficients and neighbour sources.
// DIRECT (FP32 split front half): the GEMM inputs go straight from the
// compute loops to X in global memory, no staging buffers.  HALO (acoustic
// fused step): the neighbours outside the block arrive whole, one bulk copy
// of Nf Np floats per (element, face) slot, instead of their face-node traces.
template <int MODEL, int N, int EB, bool OPS_SMEM, bool R_SMEM, bool FACT = false, bool DIRECT = false,
          bool HALO = false>
struct Plan {
  using S = Sz<N>;
  static constexpr int Nf = MODEL == 0 ? 4 : 9;
  static constexpr int REC = Rec<MODEL>::size;
  static constexpr int EBP = EB + 1;                      // odd row stride of element-fastest arrays
  static constexpr int nQ = EB * Nf * S::Np;
  // element stride of q in the stage: DIRECT reads it element-fastest across
  // lanes, so a stride that is a multiple of 8 words gets 4 words of padding
  // (8 consecutive elements then start in 8 different 4-bank groups) and the
  // elements are copied one by one
  static constexpr int QPAD = (DIRECT && (Nf * S::Np) % 8 == 0) ? 4 : 0;
  static constexpr int QS = Nf * S::Np + QPAD;
  static constexpr int nStage = round4(EB * QS + EB * REC) + EB * 4;  // q, records, neighbour words
  static constexpr int sQ = 0, sRec = EB * QS, sNbr = round4(EB * QS + EB * REC);
  static constexpr int nR = R_SMEM ? 2 * nQ : 0;
  static constexpr int nXvol = DIRECT ? 0 : (MODEL == 0 ? 4 : 12) * S::Np * EBP;
  static constexpr int nXsur = DIRECT ? 0 : (FACT ? 2 : Nf) * S::NFN * EBP;
  // halo slot stride: Nf Np floats, + 4 when that is a multiple of 8 words
  // (the 4 slots of an element then start in different bank groups)
  static constexpr int HS = Nf * S::Np + ((Nf * S::Np) % 8 == 0 ? 4 : 0);
  static constexpr int nT = HALO ? 4 * EB * HS              // halo slots [EB][4][HS]
                                : Nf * S::NFN * EBP;      // neighbour traces [Nf][4Nfp][EBP]
  // per-face arrays [4][EBF]: the odd row stride keeps the 4 faces of an
  // element in different banks when lanes run over face nodes
  static constexpr int EBF = EB + 1;
  static constexpr int nOps = OPS_SMEM ? S::KD * S::Mpad : 0;
  static constexpr int oStage0 = 0;
  static constexpr int oStage1 = oStage0 + nStage;
  static constexpr int oR = oStage1 + nStage;
  static constexpr int oXvol = round4(oR + nR);
  static constexpr int oXsur = round4(oXvol + nXvol);
  static constexpr int oT0 = round4(oXsur + nXsur);
  // one trace buffer: every path gathers the next block's traces after the
  // barrier that follows this block's last read of them
  static constexpr int oT1 = oT0;
  static constexpr int oOps = round4(oT1 + nT);
  static constexpr int oFn = round4(oOps + nOps);          // [4][EBF] float4: n, Fscale
  static constexpr int oNt = oFn + EBF * 16;               // [4 x 3][EBP]: normals, element fastest (FACT)
  static constexpr int oCo = round4(oNt + (FACT ? 12 * EBP : 0));  // [4][EBF] float4: penalty coefficients (FACT)
  static constexpr int oFi = oCo + (FACT ? EBF * 16 : 0);  // [4][EBF] int2: neighbour source (FACT)
  static constexpr int oFtab = oFi + (FACT ? EBF * 8 : 0); // int [10][Nfp]
  static constexpr int oPtab = oFtab + 10 * S::Nfp;        // int [4][6][Nfp]: neighbour node (FACT)
  static constexpr int oBar = round4(oPtab + (FACT ? 24 * S::Nfp : 0));
  static constexpr int nFloats = oBar + 10;                // 5 mbarriers
  static constexpr size_t bytes = size_t(nFloats) * 4;
  static_assert(DIRECT || nXvol >= Nf * S::Np * EBP, "the RHS of a block is staged in the volume-input buffer");
};

// Split step for the tensor cores: the front half leaves its GEMM inputs as
// NSPLIT BF16 pieces, already in the tcgen05 operand layout.  Per column tile
// of NE elements, chunk c of 16 input indices (volume chunks c < NKD: the NV
// volume input vectors at nodes 16c..16c+15; lift chunks: the Nf penalty
// vectors at face nodes 16(c - NKD)..) is one contiguous block
// [piece][vector][NE/8 element groups][2 K halves][8 elements][8 values]
// (no-swizzle K-major core matrices of 8 rows x 16 bytes), zero beyond Np or
// 4 Nfp, so that one bulk copy moves a chunk.
template <int MODEL, int N, int NSPLIT>
struct TcX {
  using S = Sz<N>;
  static constexpr int Np = S::Np, NFN = S::NFN;
  static constexpr int Nf = MODEL == 0 ? 4 : 9;
  static constexpr int NV = MODEL == 0 ? 4 : 12;
  // elements per column tile (the MMA N): each operator piece in shared memory
  // serves NE elements; acoustic N >= 7 takes 64 (7 x 64 TMEM columns, one
  // accumulator), below 32 (two accumulators alternate)
  static constexpr int NE = MODEL == 0 ? (N >= 7 ? 64 : 32) : 16;
  static constexpr int NKD = (Np + 15) / 16, NKL = (NFN + 15) / 16;
  static constexpr int BV = NE * 16 * 2;           // one piece of one vector of one chunk
  static constexpr int CD = NSPLIT * NV * BV;      // bytes of a volume chunk
  static constexpr int CL = NSPLIT * Nf * BV;      // bytes of a lift chunk
  static constexpr size_t TILE = size_t(NKD) * CD + size_t(NKL) * CL;
  __host__ __device__ static constexpr size_t chunk_off(int c) {
    return c < NKD ? size_t(c) * CD : size_t(NKD) * CD + size_t(c - NKD) * CL;
  }
};

// BF16 pieces of 8 values, two at a time: x_0 = bf16(x), x_1 = bf16(x - x_0),
// x_2 = bf16(x - x_0 - x_1) (round to nearest even; the remainders are exact
// in FP32); out[h] holds piece h of the 8 values, value 0 in the low half.
template <int NSPLIT>
__device__ __forceinline__ void bf16_pieces8(const float* x, uint4* out) {
  float r[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) r[t] = x[t];
#pragma unroll
  for (int h = 0; h < NSPLIT; ++h) {
    uint32_t w[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const __nv_bfloat162 b = __floats2bfloat162_rn(r[2 * p], r[2 * p + 1]);
      w[p] = *reinterpret_cast<const uint32_t*>(&b);
      if (h + 1 < NSPLIT) {
        const float2 f = __bfloat1622float2(b);
        r[2 * p] -= f.x;
        r[2 * p + 1] -= f.y;
      }
    }
    out[h] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Outward unit normal and Fscale = |g N_f| of face f of an element with
// inverse metric g (row-major g[c][d] = dr_d/dx_c): n = g N_f / |g N_f|.
__device__ __forceinline__ float4 face_normal(const float* g, int f) {
  float nv[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    nv[c] = g[3 * c] * ref_normal(f, 0) + g[3 * c + 1] * ref_normal(f, 1) + g[3 * c + 2] * ref_normal(f, 2);
  const float fs = sqrtf(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
  const float inv = 1.0f / fs;
  return make_float4(nv[0] * inv, nv[1] * inv, nv[2] * inv, fs);
}

// Fscale-weighted penalty terms at one face node (Section 2.1): the numerical
// flux across the face minus the own trace's flux, for the upwind (flux = 0)
// or centred (flux = 1) flux, with the mirror ghost state on the outer
// boundary (acoustic rigid wall; elastic bc = 0 traction-free, 1 rigid).
//   gM: the element's record; f: its face; qM, qP: own and neighbour traces
//   (qP unused on the boundary); fn = (n_x, n_y, n_z, Fscale) of the face.
//   pen[Nf]: acoustic (dp, dv_x, dv_y, dv_z), elastic (p_v[3], P_sigma[6]).
//   pvdv (elastic, optional): instead of pen, (Fscale p_v, Fscale dv) -- the
//   stress penalty is lambda (n.dv) I + mu (n dv^T + dv n^T), times Fscale
template <int MODEL>
__device__ __forceinline__ void face_penalty(const float* gM, int f, bool bnd, const float* qM, const float* qPv,
                                             const float4 fn, int flux, int bc, float* pen,
                                             float* pvdv = nullptr) {
  const float nx = fn.x, ny = fn.y, nz = fn.z, fs = fn.w;
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
      pP = qPv[0]; vP0 = qPv[1]; vP1 = qPv[2]; vP2 = qPv[3];
    }
    const float jp = 0.5f * (pP - qM[0]);
    const float jvn = 0.5f * ((vP0 - qM[1]) * nx + (vP1 - qM[2]) * ny + (vP2 - qM[3]) * nz);
    float dp, sv;  // dv = sv * n
    if (flux == 0) {
      const float kc = 2.f / (ZM + zP);
      const float ac = jp - zP * jvn;
      dp = kap * kc * ac;
      sv = -(ZM * rinv) * kc * ac;  // c^- = Z^- / rho^-
    } else {
      dp = -kap * jvn;
      sv = -rinv * jp;
    }
    pen[0] = fs * dp;
    pen[1] = fs * sv * nx;
    pen[2] = fs * sv * ny;
    pen[3] = fs * sv * nz;
  } else {
    const float lam = gM[9], mu = gM[10], rinv = gM[11], ZpM = gM[12], ZsM = gM[13], cpM = gM[14],
                csM = gM[15], zP0 = gM[16 + f], zP1 = gM[20 + f];
    float vP[3], sPd[6];
    if (bnd) {
      const float sv = (bc == 0) ? 1.f : -1.f;  // free: v+ = v-, sigma+ = -sigma-
#pragma unroll
      for (int c = 0; c < 3; ++c) vP[c] = sv * qM[c];
#pragma unroll
      for (int c = 0; c < 6; ++c) sPd[c] = -sv * qM[3 + c];
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) vP[c] = qPv[c];
#pragma unroll
      for (int c = 0; c < 6; ++c) sPd[c] = qPv[3 + c];
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
    if (flux == 0) {
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
    if (pvdv) {  // the two vectors the 9 penalties are made of, Fscale included
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pvdv[c] = fs * pv[c];
        pvdv[3 + c] = fs * dv[c];
      }
      return;
    }
    const float ndv = nx * dv[0] + ny * dv[1] + nz * dv[2];
    pen[0] = fs * pv[0];
    pen[1] = fs * pv[1];
    pen[2] = fs * pv[2];
    pen[3] = fs * (lam * ndv + 2.f * mu * nx * dv[0]);
    pen[4] = fs * (lam * ndv + 2.f * mu * ny * dv[1]);
    pen[5] = fs * (lam * ndv + 2.f * mu * nz * dv[2]);
    pen[6] = fs * (mu * (nx * dv[1] + ny * dv[0]));
    pen[7] = fs * (mu * (nx * dv[2] + nz * dv[0]));
    pen[8] = fs * (mu * (ny * dv[2] + nz * dv[1]));
  }
}

// ---------------------------------------------------------------- block providers
// A provider maps a global block index to the arguments of the solve it
// belongs to and to its local block index; operators, face tables, error word
// and mode are common to every block of one launch.
struct SingleSolve {
  const StepArgs& a;
  int EB;
  __device__ int nblocks() const { return (a.K + EB - 1) / EB; }
  __device__ void get(int b, StepArgs& A, int& lb) const {
    A = a;
    lb = b;
  }
  __device__ const float* ops() const { return a.ops; }
  __device__ const int* ftab() const { return a.ftab; }
  __device__ int* err() const { return a.err; }
  __device__ int mode() const { return a.mode; }
  __device__ long long limit() const { return a.wait_limit; }
};

// Step arguments of one solve of a batch, from its device-side state.
__device__ __forceinline__ void solve_args(const BatchArgs& B, const SolveDev& d, StepArgs& A) {
  {
    const int qc = d.qcur, r1s = d.r1slot;
    A.q = d.q[qc];
    A.qn = d.q[1 - qc];
    A.r1 = d.r[r1s];
    A.r2 = d.r[1 - r1s];
    A.rout = nullptr;
    A.rec = d.rec;
    A.nbr = d.nbr;
    A.ops = B.ops;
    A.ftab = B.ftab;
    A.srcvec = d.src_elem >= 0 ? d.srcvec : nullptr;
    A.src_elem = d.src_elem;
    A.src_amp = (d.src_elem >= 0 && d.step < d.namp) ? d.amp[d.step] : 0.0f;
    A.K = d.K;
    A.mode = 0;
    A.flux = d.flux;
    A.bc = d.bc;
    A.dt = d.dt;
    if (d.have == 0) { A.a1 = 1.f; A.a2 = 0.f; A.a3 = 0.f; }
    else if (d.have == 1) { A.a1 = 1.5f; A.a2 = -0.5f; A.a3 = 0.f; }
    else { A.a1 = 23.f / 12.f; A.a2 = -16.f / 12.f; A.a3 = 5.f / 12.f; }
    A.err = B.err;
    A.wait_limit = B.wait_limit;
    A.xg = d.xg;
    A.ops2 = B.ops2;
    A.opstc = nullptr;
  }
}

struct SolveBatch {
  const BatchArgs& B;
  __device__ int nblocks() const { return B.total_blocks; }
  __device__ void get(int b, StepArgs& A, int& lb) const {
    const int lo = __ldg(B.block_solve + b);  // solve of global block b
    lb = b - __ldg(B.block_start + lo);
    solve_args(B, B.solves[lo], A);
  }
  __device__ const float* ops() const { return B.ops; }
  __device__ const int* ftab() const { return B.ftab; }
  __device__ int* err() const { return B.err; }
  __device__ int mode() const { return 0; }
  __device__ long long limit() const { return B.wait_limit; }
};

// ---------------------------------------------------------------- kernel body
template <int MODEL, int N, int EB, int TN, int NT, bool OPS_SMEM, bool R_SMEM, int SPLIT, int XP, bool HALO,
          class Prov>
__device__ __forceinline__ void step_body(const Prov& prov) {
  using S = Sz<N>;
  constexpr bool FACT = MODEL == 0 && XP == 0;  // every acoustic path but the tensor-core one
  constexpr bool DIRECT = SPLIT > 0 && XP == 0;  // FP32 split front half: X written from the loops
  static_assert(!HALO || (FACT && SPLIT == 0), "whole-neighbour halos in the acoustic fused step");
  using P = Plan<MODEL, N, EB, OPS_SMEM, R_SMEM, FACT, DIRECT, HALO>;
  constexpr int Np = S::Np, Nfp = S::Nfp, NFN = S::NFN, Mpad = S::Mpad, RT = S::RT;
  constexpr int Nf = P::Nf, REC = P::REC, EBP = P::EBP;
  constexpr int NTILE = RT * (EB / TN);  // tiles of 4 output nodes x TN elements
  static_assert(EB % 4 == 0, "EB must be a multiple of 4 (16-byte TMA pieces)");
  static_assert(EB % TN == 0, "EB must be a multiple of TN");
  static_assert(NTILE <= NT, "one output tile per thread");

  extern __shared__ __align__(16) float smem[];
  float* sR = smem + P::oR;
  float* sXv = smem + P::oXvol;
  float* sXs = smem + P::oXsur;
  const float* sOps = OPS_SMEM ? smem + P::oOps : prov.ops();
  int* const err = prov.err();
  const int mode = prov.mode();
  float* sFn = smem + P::oFn;
  int* sFtab = reinterpret_cast<int*>(smem + P::oFtab);
  float* sNt = smem + P::oNt;
  float4* sCo = reinterpret_cast<float4*>(smem + P::oCo);
  int2* sFi = reinterpret_cast<int2*>(smem + P::oFi);
  int* sPtab = reinterpret_cast<int*>(smem + P::oPtab);
  // DIRECT: address of GEMM input row `row` of element k in X[tile][row][NE]
  constexpr int XNE = SPLIT > 0 ? SPLIT : 1;
  auto xrow = [](const StepArgs& A, int row, int k) {
    return A.xg + (size_t(k / XNE) * XRows<MODEL, N>::KX + row) * XNE + (k % XNE);
  };
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + P::oBar);

  const int tid = threadIdx.x;
  const int nblk = prov.nblocks();
  const int G = gridDim.x;
  constexpr uint32_t kQBytes = uint32_t(P::nQ * 4);
  constexpr uint32_t kRecBytes = uint32_t(EB * REC * 4);
  constexpr uint32_t kStageBytes = kQBytes + kRecBytes + uint32_t(EB * 16);

  // Copies in flight, for the drain after an expired wait: bit i of pmask is
  // set while barrier i (stages 0/1, history 2, halo buffers 3/4) has a phase
  // with copies issued and not yet seen complete, bit i of ppar is that
  // phase's parity.  The issue conditions are CTA-uniform, so every thread
  // keeps the same bits (cp.async gathers are drained per thread, bulk stores
  // by the thread that issued them).
  const long long lim = prov.limit();
  uint32_t pmask = 0, ppar = 0;
  auto pend_set = [&](int i, uint32_t par) {
    pmask |= 1u << i;
    ppar = (ppar & ~(1u << i)) | (par << i);
  };
  auto pend_clr = [&](int i) { pmask &= ~(1u << i); };
  auto drain = [&]() {
#pragma unroll
    for (int i = 0; i < 5; ++i)
      if (pmask & (1u << i)) mbar_wait_bounded(&bars[i], (ppar >> i) & 1u, nullptr);
    cp_async_wait_all();
    if (tid == 0) bulk_wait_all();
  };

  auto stage = [&](int s) { return smem + (s ? P::oStage1 : P::oStage0); };
  auto issue_stage = [&](const StepArgs& a, int lb, int s, bool with_ops) {
    float* st = stage(s);
    const int k0 = lb * EB;
    const uint32_t bo = (OPS_SMEM && with_ops) ? uint32_t(S::KD * Mpad * 4) : 0u;
    mbar_arrive_expect_tx(&bars[s], kStageBytes + bo);
    if constexpr (P::QPAD == 0) {
      tma_bulk_g2s(st + P::sQ, a.q + size_t(k0) * Nf * Np, kQBytes, &bars[s]);
    } else {
      for (int e = 0; e < EB; ++e)
        tma_bulk_g2s(st + P::sQ + e * P::QS, a.q + size_t(k0 + e) * Nf * Np, uint32_t(Nf * Np * 4), &bars[s]);
    }
    tma_bulk_g2s(st + P::sRec, a.rec + size_t(k0) * REC, kRecBytes, &bars[s]);
    tma_bulk_g2s(st + P::sNbr, a.nbr + k0, uint32_t(EB * 16), &bars[s]);
    if (OPS_SMEM && with_ops) tma_bulk_g2s(smem + P::oOps, a.ops, bo, &bars[s]);
    if (!R_SMEM && SPLIT == 0 && a.mode == 0) {
      // the block's AB3 history into L2 (it is read from global memory in the update pass)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.r1 + size_t(k0) * Nf * Np), "r"(kQBytes)
                   : "memory");
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.r2 + size_t(k0) * Nf * Np), "r"(kQBytes)
                   : "memory");
    }
  };
  // neighbour traces of block b that live outside it: 4-byte async copies
  // (cp.async) into trace buffer s, layout [Nf][4 Nfp][EBP], face node fastest;
  // HALO: the whole neighbour, one bulk copy per (element, face) slot of
  // buffer s, every thread arriving once on its barrier after registering
  // the bytes of its own copies
  auto issue_gathers = [&](const StepArgs& a, int lb, int s) {
    const int k0 = lb * EB;
    const int4* nb_s = reinterpret_cast<const int4*>(stage(s) + P::sNbr);
    float* T = smem + (s ? P::oT1 : P::oT0);
    if constexpr (HALO) {
      constexpr uint32_t kElem = uint32_t(Nf * Np * 4);
      for (int i = tid; i < EB * 4; i += NT) {
        const int e = i >> 2, f = i & 3;
        const int4 nb = nb_s[e];
        const int w = (f == 0) ? nb.x : (f == 1) ? nb.y : (f == 2) ? nb.z : nb.w;
        if (w < 0) continue;
        const int kn = w >> kNbrShift;
        const int le = kn - k0;
        if (le >= 0 && le < EB) continue;
        mbar_expect_tx(&bars[3 + s], kElem);
        tma_bulk_g2s(T + i * P::HS, a.q + size_t(kn) * Nf * Np, kElem, &bars[3 + s]);
      }
      mbar_arrive(&bars[3 + s]);
      return;
    }
    for (int i = tid; i < EB * NFN; i += NT) {
      const int fm = i % NFN, e = i / NFN;
      const int f = fm / Nfp, m = fm - f * Nfp;
      const int4 nb = nb_s[e];
      const int w = (f == 0) ? nb.x : (f == 1) ? nb.y : (f == 2) ? nb.z : nb.w;
      if (w < 0) continue;
      const int kn = w >> kNbrShift;
      const int le = kn - k0;
      if (le >= 0 && le < EB) continue;
      const int rot = (w >> 2) & 7, f2 = w & 3;
      const int nP = FACT ? sPtab[(f2 * 6 + rot) * Nfp + m] : sFtab[f2 * Nfp + sFtab[4 * Nfp + rot * Nfp + m]];
      const float* src = a.q + size_t(kn) * Nf * Np + nP;
#pragma unroll
      for (int c = 0; c < Nf; ++c) cp_async4(T + (c * NFN + fm) * EBP + e, src + c * Np);
    }
    cp_async_commit();
  };

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    mbar_init(&bars[3], NT);  // halo buffers: one arrival per thread
    mbar_init(&bars[4], NT);
    fence_barrier_init();
  }
  __syncthreads();
  // arguments of the block being processed (cur) and of the next one (nxt)
  StepArgs nxt_a;
  int nxt_lb = 0;
  if ((int)blockIdx.x < nblk) prov.get(blockIdx.x, nxt_a, nxt_lb);
  if (tid == 0 && (int)blockIdx.x < nblk) issue_stage(nxt_a, nxt_lb, 0, true);
  if ((int)blockIdx.x < nblk) pend_set(0, 0u);
  for (int i = tid; i < 10 * Nfp; i += NT) sFtab[i] = prov.ftab()[i];
  __syncthreads();
  if constexpr (FACT) {
    // neighbour volume node of own face node m across a face seen as the
    // neighbour's face f2 under rotation rot: ptab[(f2 * 6 + rot) Nfp + m]
    for (int i = tid; i < 24 * Nfp; i += NT) {
      const int m = i % Nfp, fr = i / Nfp;
      sPtab[i] = sFtab[(fr / 6) * Nfp + sFtab[4 * Nfp + (fr % 6) * Nfp + m]];
    }
  }
  if ((int)blockIdx.x < nblk) {
    if (!__syncthreads_and(mbar_wait_bounded(&bars[0], 0u, err, lim))) {
      drain();
      return;
    }
    pend_clr(0);
    issue_gathers(nxt_a, nxt_lb, 0);
    if constexpr (HALO) pend_set(3, 0u);
  }

  int it = 0;
  for (int b = blockIdx.x; b < nblk; b += G, ++it) {
    const int s = it & 1;
    const StepArgs a = nxt_a;
    const int lb = nxt_lb;
    const int k0 = lb * EB;
    if (b + G < nblk) prov.get(b + G, nxt_a, nxt_lb);
    bool ok = mbar_wait_bounded(&bars[s], uint32_t((it >> 1) & 1), err, lim);
    if constexpr (HALO) ok = mbar_wait_bounded(&bars[3 + s], uint32_t((it >> 1) & 1), err, lim) && ok;
    else cp_async_wait_all();  // this block's neighbour traces
    if (!__syncthreads_and(ok)) {
      drain();
      return;
    }
    pend_clr(s);
    if constexpr (HALO) pend_clr(3 + s);
    // everyone is past the previous block: stage s^1, sR, the inputs and trace buffer s^1 are free
    const float* sQ = stage(s) + P::sQ;
    const float* sRec = stage(s) + P::sRec;
    const int4* sNbr = reinterpret_cast<const int4*>(stage(s) + P::sNbr);
    const float* sT = smem + (s ? P::oT1 : P::oT0);
    if (tid == 0) {
      if (b + G < nblk) issue_stage(nxt_a, nxt_lb, s ^ 1, false);
      if (R_SMEM && mode == 0) {
        if (it > 0) bulk_wait_read();  // the previous block's outputs have left sR
        mbar_arrive_expect_tx(&bars[2], 2 * kQBytes);
        tma_bulk_g2s(sR, a.r1 + size_t(k0) * Nf * Np, kQBytes, &bars[2]);
        tma_bulk_g2s(sR + P::nQ, a.r2 + size_t(k0) * Nf * Np, kQBytes, &bars[2]);
      }
    }
    const uint32_t pnext = uint32_t(((it + 1) >> 1) & 1);  // phase of stage s^1 for the next block
    if (b + G < nblk) pend_set(s ^ 1, pnext);
    if (R_SMEM && mode == 0) pend_set(2, uint32_t(it & 1));

    // -------- face normals and Fscale (n = g N_f / |g N_f|); the per-face
    // arrays are face-major, entry f EBF + e (element-fastest lanes read
    // consecutive entries)
    for (int i = tid; i < EB * 4; i += NT) {
      const int e = i % EB, f = i / EB;
      const float4 fn = face_normal(sRec + e * REC, f);
      const int fe = f * P::EBF + e;
      *reinterpret_cast<float4*>(sFn + fe * 4) = fn;
      if constexpr (DIRECT) {  // the face normals are GEMM inputs too
        constexpr int KXM = XRows<MODEL, N>::KXM;
        *xrow(a, KXM + 3 * f + 0, k0 + e) = fn.x;
        *xrow(a, KXM + 3 * f + 1, k0 + e) = fn.y;
        *xrow(a, KXM + 3 * f + 2, k0 + e) = fn.z;
      }
      if constexpr (FACT) {
        sNt[(3 * f + 0) * EBP + e] = fn.x;
        sNt[(3 * f + 1) * EBP + e] = fn.y;
        sNt[(3 * f + 2) * EBP + e] = fn.z;

        // penalty coefficients of the face, pen_p = A jp + B jvn and
        // psi = C jp + D jvn with jp = [[p]]/2, jvn = [[v]].n/2 (Fscale folded
        // in), and where the neighbour trace comes from: -1 outer boundary,
        // >= 0 the neighbour's fields in this block, -2 the gathered traces
        const float* gk = sRec + e * REC;
        const float fs = fn.w, kap = gk[9], rinv = gk[10], ZM = gk[11], zP = gk[12 + f];
        float4 co;
        if (a.flux == 0) {
          const float kc = 2.f / (ZM + zP);
          co.x = fs * kap * kc;
          co.y = -co.x * zP;
          co.z = -fs * (ZM * rinv) * kc;
          co.w = -co.z * zP;
        } else {
          co = make_float4(0.f, -fs * kap, -fs * rinv, 0.f);
        }
        sCo[fe] = co;
        const int4 nb = sNbr[e];
        const int w = (f == 0) ? nb.x : (f == 1) ? nb.y : (f == 2) ? nb.z : nb.w;
        int2 fi = make_int2(-1, 0);
        if (w >= 0) {
          const int le = (w >> kNbrShift) - k0;
          fi.x = (le >= 0 && le < EB) ? le * P::QS : -2;
          fi.y = ((w & 3) * 6 + ((w >> 2) & 7)) * Nfp;
        }
        sFi[fe] = fi;
      }
    }
    // -------- volume inputs (node index fastest: conflict-free reads of q;
    // DIRECT: element index fastest, each row of X gets EB consecutive words)
    for (int i = tid; i < EB * Np; i += NT) {
      const int j = DIRECT ? i / EB : i % Np, e = DIRECT ? i % EB : i / Np;
      const float* gk = sRec + e * REC;
      const float* qe = sQ + e * P::QS;
      // volume input v at node j of element e
      auto put = [&](int v, float x) {
        if constexpr (DIRECT) *xrow(a, v * Np + j, k0 + e) = x;
        else sXv[(v * Np + j) * EBP + e] = x;
      };
      if constexpr (MODEL == 0) {
        const float kap = gk[9];
        const float v0 = qe[Np + j], v1 = qe[2 * Np + j], v2 = qe[3 * Np + j];
        put(0, qe[j]);
#pragma unroll
        for (int d = 0; d < 3; ++d) put(1 + d, -kap * (gk[d] * v0 + gk[3 + d] * v1 + gk[6 + d] * v2));
      } else {
        const float rinv = gk[11];
        float sg[3][3];
        sg[0][0] = qe[3 * Np + j]; sg[1][1] = qe[4 * Np + j]; sg[2][2] = qe[5 * Np + j];
        sg[0][1] = sg[1][0] = qe[6 * Np + j];
        sg[0][2] = sg[2][0] = qe[7 * Np + j];
        sg[1][2] = sg[2][1] = qe[8 * Np + j];
#pragma unroll
        for (int c = 0; c < 3; ++c) put(c, qe[c * Np + j]);
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d)
            put(3 + 3 * c + d, rinv * (gk[d] * sg[c][0] + gk[3 + d] * sg[c][1] + gk[6 + d] * sg[c][2]));
      }
    }
    __syncthreads();  // sFn ready

    // -------- traces and penalty terms at the 4 Nfp face nodes (face node fastest)
    constexpr int NVX = XRows<MODEL, N>::NV;  // DIRECT: the surface rows of X follow NVX Np volume rows
    if constexpr (FACT) {
      constexpr int XS = NFN * EBP;
      for (int i = tid; i < EB * NFN; i += NT) {
        const int fm = DIRECT ? i / EB : i % NFN, e = DIRECT ? i % EB : i / NFN;
        const int f = fm / Nfp, m = fm - f * Nfp;
        const int fe = f * P::EBF + e;  // per-face arrays
        const int fi = e * 4 + f;   // halo slot
        const int2 src = sFi[fe];
        const float4 fn = *reinterpret_cast<const float4*>(sFn + fe * 4);
        const float4 co = sCo[fe];
        const int nM = sFtab[f * Nfp + m];
        const float* qe = sQ + e * P::QS + nM;
        const float pM = qe[0], vM0 = qe[Np], vM1 = qe[2 * Np], vM2 = qe[3 * Np];
        float jp, jvn;
        if (src.x == -1) {  // rigid wall: p+ = p-, v+ = v- - 2 (v-.n) n
          jp = 0.f;
          jvn = -(vM0 * fn.x + vM1 * fn.y + vM2 * fn.z);
        } else {
          float pP, vP0, vP1, vP2;
          if (src.x >= 0) {
            const float* qn = sQ + src.x + sPtab[src.y + m];
            pP = qn[0]; vP0 = qn[Np]; vP1 = qn[2 * Np]; vP2 = qn[3 * Np];
          } else if constexpr (HALO) {
            const float* qn = sT + fi * P::HS + sPtab[src.y + m];
            pP = qn[0]; vP0 = qn[Np]; vP1 = qn[2 * Np]; vP2 = qn[3 * Np];
          } else {
            const float* T = sT + fm * EBP + e;
            pP = T[0]; vP0 = T[XS]; vP1 = T[2 * XS]; vP2 = T[3 * XS];
          }
          jp = 0.5f * (pP - pM);
          jvn = 0.5f * ((vP0 - vM0) * fn.x + (vP1 - vM1) * fn.y + (vP2 - vM2) * fn.z);
        }
        const float pp = co.x * jp + co.y * jvn, ps = co.z * jp + co.w * jvn;
        if constexpr (DIRECT) {
          *xrow(a, NVX * Np + fm, k0 + e) = pp;
          *xrow(a, NVX * Np + NFN + fm, k0 + e) = ps;
        } else {
          float* X = sXs + fm * EBP + e;
          X[0] = pp;
          X[XS] = ps;
        }
      }
    } else
    for (int i = tid; i < EB * NFN; i += NT) {
      const int fm = DIRECT ? i / EB : i % NFN, e = DIRECT ? i % EB : i / NFN;
      const int f = fm / Nfp, m = fm - f * Nfp;
      const int nM = sFtab[f * Nfp + m];
      const int4 nb = sNbr[e];
      const int w = (f == 0) ? nb.x : (f == 1) ? nb.y : (f == 2) ? nb.z : nb.w;
      const bool bnd = w < 0;
      float qPv[Nf];
      if (!bnd) {
        const int kn = w >> kNbrShift;
        const int le = kn - k0;
        if (le >= 0 && le < EB) {
          const int rot = (w >> 2) & 7, f2 = w & 3;
          const int nP = sFtab[f2 * Nfp + sFtab[4 * Nfp + rot * Nfp + m]];
          const float* qn = sQ + le * P::QS;
#pragma unroll
          for (int c = 0; c < Nf; ++c) qPv[c] = qn[c * Np + nP];
        } else {
#pragma unroll
          for (int c = 0; c < Nf; ++c) qPv[c] = sT[(c * NFN + fm) * EBP + e];
        }
      }
      const float* qe = sQ + e * P::QS;
      const float4 fn = *reinterpret_cast<const float4*>(sFn + (f * P::EBF + e) * 4);
      const float* gM = sRec + e * REC;
      float qM[Nf];
#pragma unroll
      for (int c = 0; c < Nf; ++c) qM[c] = qe[c * Np + nM];
      float pen[Nf];
      if constexpr (DIRECT) {  // elastic: the 6 streams Fscale p_v, Fscale dv
        static_assert(MODEL == 1 && XRows<MODEL, N>::NXS == 6, "elastic surface streams of X");
        float pd[6];
        face_penalty<MODEL>(gM, f, bnd, qM, qPv, fn, a.flux, a.bc, pen, pd);
#pragma unroll
        for (int c = 0; c < 6; ++c) *xrow(a, NVX * Np + c * NFN + fm, k0 + e) = pd[c];
      } else {
        face_penalty<MODEL>(gM, f, bnd, qM, qPv, fn, a.flux, a.bc, pen);
        float* X = sXs + fm * EBP + e;
        constexpr int XS = NFN * EBP;
#pragma unroll
        for (int c = 0; c < Nf; ++c) X[c * XS] = pen[c];
      }
    }
    if constexpr (DIRECT) {
      // every GEMM input of the block is in X: start the next block's
      // neighbour gathers and move on
      static_assert(SPLIT % 4 == 0 && (SPLIT % EB == 0 || EB % SPLIT == 0), "element blocks inside column tiles");
      // (after a barrier: the gathers overwrite the trace buffer this block
      // has just read; the decision is CTA-wide)
      {
        const bool okn = b + G < nblk ? mbar_wait_bounded(&bars[s ^ 1], pnext, err, lim) : true;
        if (!__syncthreads_and(okn)) {
          drain();
          return;
        }
      }
      if (b + G < nblk) {
        pend_clr(s ^ 1);
        issue_gathers(nxt_a, nxt_lb, s ^ 1);
      }
      continue;
    }
    // the next block's stage was issued at the top of this block: once it has
    // landed, start its neighbour gathers so that they overlap the products
    // (a CTA-wide decision: halo copies need every thread's arrival)
    {
      const bool okn = b + G < nblk ? mbar_wait_bounded(&bars[s ^ 1], pnext, err, lim) : true;
      if (!__syncthreads_and(okn)) {
        drain();
        return;
      }
    }
    if (b + G < nblk) {
      pend_clr(s ^ 1);
      issue_gathers(nxt_a, nxt_lb, s ^ 1);
      if constexpr (HALO) pend_set(3 + (s ^ 1), pnext);
    }

    if constexpr (SPLIT > 0 && XP > 0) {
      // split step for the tensor cores, front half: every 8 input indices of
      // one element become XP BF16 pieces of 16 bytes in the chunk layout of TcX
      using TX = TcX<MODEL, N, XP>;
      static_assert(TX::NE == SPLIT, "column tile of the tensor-core kernel");
      constexpr int NV = TX::NV, NKD = TX::NKD, NKL = TX::NKL, NE = TX::NE;
      constexpr int NRG = 2 * (NV * NKD + Nf * NKL);  // groups of 8 input indices per element
      uint8_t* xb = reinterpret_cast<uint8_t*>(a.xg);
      for (int i = tid; i < EB * NRG; i += NT) {
        const int e = i % EB, rg = i / EB;
        const bool vol = rg < 2 * NV * NKD;
        const int r2 = vol ? rg : rg - 2 * NV * NKD;
        const int per = vol ? 2 * NKD : 2 * NKL;
        const int vv = r2 / per, w = r2 - vv * per;
        const int cl = w >> 1, kh = w & 1;  // chunk within its kind, K half
        const int i0 = cl * 16 + kh * 8;    // first node (volume) or face node (lift)
        const int lim = vol ? Np : NFN;
        const float* src = vol ? sXv + (vv * Np) * EBP + e : sXs + (vv * NFN) * EBP + e;
        float x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = (i0 + t < lim) ? src[(i0 + t) * EBP] : 0.f;
        uint4 pc[XP];
        bf16_pieces8<XP>(x, pc);
        const int k = k0 + e;
        const int el = k % NE;
        const int nvs = vol ? NV : Nf;
        uint8_t* dst = xb + size_t(k / NE) * TX::TILE + TX::chunk_off(vol ? cl : NKD + cl) +
                       size_t(vv * (NE / 8) + (el >> 3)) * 256 + kh * 128 + (el & 7) * 16;
#pragma unroll
        for (int h = 0; h < XP; ++h)
          *reinterpret_cast<uint4*>(dst + size_t(h) * nvs * TX::BV) = pc[h];
      }
      continue;
    }

    // -------- register-tiled operator products (one tile of 4 nodes x TN elements per thread)
    float r[TN][Nf][4];
    const bool has_tile = tid < NTILE;
    // element index fastest across lanes: a warp shares each operator row
    // segment (one broadcast wavefront) and reads consecutive input columns
    constexpr int CT = EB / TN;
    const int e0 = (tid % CT) * TN, rt = tid / CT;
    const int i0 = 4 * rt;
    if (has_tile) {
      const float* A = sOps + i0;
      if constexpr (MODEL == 0) {
        // L: LIFT of the three velocity penalties (split step) or, FACT, of
        // psi face by face (L[f]; the velocity lift is sum_f n_f L[f])
        constexpr int NL = FACT ? 4 : 3;
        float G3[3][TN][4], R[TN][4], L[NL][TN][4];
#pragma unroll
        for (int t = 0; t < TN; ++t)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            R[t][v] = 0.f;
#pragma unroll
            for (int d = 0; d < 3; ++d) G3[d][t][v] = 0.f;
#pragma unroll
            for (int d = 0; d < NL; ++d) L[d][t][v] = 0.f;
          }
#pragma unroll 4
        for (int j = 0; j < Np; ++j) {
          const float4 a0 = load_op<OPS_SMEM>(A + (0 * Np + j) * Mpad);
          const float4 a1 = load_op<OPS_SMEM>(A + (1 * Np + j) * Mpad);
          const float4 a2 = load_op<OPS_SMEM>(A + (2 * Np + j) * Mpad);
#pragma unroll
          for (int t = 0; t < TN; ++t) {
            const float xp = sXv[(0 * Np + j) * EBP + e0 + t];
            const float x0 = sXv[(1 * Np + j) * EBP + e0 + t];
            const float x1 = sXv[(2 * Np + j) * EBP + e0 + t];
            const float x2 = sXv[(3 * Np + j) * EBP + e0 + t];
            fma4(G3[0][t], a0, xp);
            fma4(G3[1][t], a1, xp);
            fma4(G3[2][t], a2, xp);
            fma4(R[t], a0, x0);
            fma4(R[t], a1, x1);
            fma4(R[t], a2, x2);
          }
        }
        if constexpr (FACT) {
#pragma unroll
          for (int f = 0; f < 4; ++f) {
#pragma unroll 4
            for (int m = 0; m < Nfp; ++m) {
              const int c = f * Nfp + m;
              const float4 l = load_op<OPS_SMEM>(A + (3 * Np + c) * Mpad);
#pragma unroll
              for (int t = 0; t < TN; ++t) {
                fma4(R[t], l, sXs[c * EBP + e0 + t]);
                fma4(L[f][t], l, sXs[(NFN + c) * EBP + e0 + t]);
              }
            }
          }
        } else {
#pragma unroll 4
          for (int c = 0; c < NFN; ++c) {
            const float4 l = load_op<OPS_SMEM>(A + (3 * Np + c) * Mpad);
#pragma unroll
            for (int t = 0; t < TN; ++t) {
              fma4(R[t], l, sXs[(0 * NFN + c) * EBP + e0 + t]);
              fma4(L[0][t], l, sXs[(1 * NFN + c) * EBP + e0 + t]);
              fma4(L[1][t], l, sXs[(2 * NFN + c) * EBP + e0 + t]);
              fma4(L[2][t], l, sXs[(3 * NFN + c) * EBP + e0 + t]);
            }
          }
        }
#pragma unroll
        for (int t = 0; t < TN; ++t) {
          const float* gk = sRec + (e0 + t) * REC;
          const float rinv = gk[10];
          float lv[3][4];
          if constexpr (FACT) {
            float nf[4][3];  // face normals of the element, element fastest in shared memory
#pragma unroll
            for (int f = 0; f < 4; ++f)
#pragma unroll
              for (int c = 0; c < 3; ++c) nf[f][c] = sNt[(3 * f + c) * EBP + e0 + t];
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
              for (int v = 0; v < 4; ++v)
                lv[c][v] = nf[0][c] * L[0][t][v] + nf[1][c] * L[1][t][v] + nf[2][c] * L[2][t][v] +
                           nf[3][c] * L[NL - 1][t][v];
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
              for (int v = 0; v < 4; ++v) lv[c][v] = L[c][t][v];
          }
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            r[t][0][v] = R[t][v];
#pragma unroll
            for (int c = 0; c < 3; ++c)
              r[t][1 + c][v] = lv[c][v] - rinv * (gk[3 * c] * G3[0][t][v] + gk[3 * c + 1] * G3[1][t][v] +
                                                  gk[3 * c + 2] * G3[2][t][v]);
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
          for (int t = 0; t < TN; ++t)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              const float xv = sXv[(c * Np + j) * EBP + e0 + t];
#pragma unroll
              for (int d = 0; d < 3; ++d) fma4(U[c][d][t], ad[d], xv);
#pragma unroll
              for (int d = 0; d < 3; ++d) fma4(Rv[c][t], ad[d], sXv[((3 + 3 * c + d) * Np + j) * EBP + e0 + t]);
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
          for (int t = 0; t < TN; ++t) {
#pragma unroll
            for (int fld = 0; fld < 3; ++fld) fma4(Rv[fld][t], l, sXs[(fld * NFN + c) * EBP + e0 + t]);
#pragma unroll
            for (int fld = 0; fld < 6; ++fld) fma4(Rs[fld][t], l, sXs[((3 + fld) * NFN + c) * EBP + e0 + t]);
          }
        }
#pragma unroll
        for (int t = 0; t < TN; ++t)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
#pragma unroll
            for (int c = 0; c < 3; ++c) r[t][c][v] = Rv[c][t][v];
#pragma unroll
            for (int c = 0; c < 6; ++c) r[t][3 + c][v] = Rs[c][t][v];
          }
      }
#pragma unroll
      for (int t = 0; t < TN; ++t) {
        const int k = k0 + e0 + t;
        if (k == a.src_elem && a.srcvec) {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (i0 + v < Np)
#pragma unroll
              for (int c = 0; c < Nf; ++c) r[t][c][v] = fmaf(a.src_amp, __ldg(a.srcvec + c * Np + i0 + v), r[t][c][v]);
        }
      }
    }

    if (mode != 0) {  // RHS only: straight to the caller's buffer
#pragma unroll
      for (int t = 0; t < TN; ++t) {
        const int k = k0 + e0 + t;
        if (has_tile && k < a.K) {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (i0 + v < Np)
#pragma unroll
              for (int c = 0; c < Nf; ++c) a.rout[size_t(k) * Nf * Np + c * Np + i0 + v] = r[t][c][v];
        }
      }
      continue;
    }

    // -------- AB3 update: the block's RHS goes to the (now free) volume-input
    // buffer as [Nf Np][EBP] (element fastest: the tile stores are free of
    // bank conflicts); one flat pass over [EB][Nf][Np] then updates the block
    __syncthreads();  // every tile has finished reading the GEMM inputs
    float* sRhs = sXv;
    if (has_tile) {
#pragma unroll
      for (int t = 0; t < TN; ++t)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (i0 + v < Np)
#pragma unroll
            for (int c = 0; c < Nf; ++c) sRhs[(c * Np + i0 + v) * EBP + e0 + t] = r[t][c][v];
    }
    // the 4 RHS values of float4 i of the block's [EB][Nf][Np] fields
    auto rhs4 = [&](int i) {
      constexpr int NQ = Nf * Np;
      float o[4];
      if constexpr (NQ % 4 == 0) {
        const int e = (4 * i) / NQ, r0 = 4 * i - e * NQ;
#pragma unroll
        for (int u = 0; u < 4; ++u) o[u] = sRhs[(r0 + u) * EBP + e];
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int l = 4 * i + u, e = l / NQ;
          o[u] = sRhs[(l - e * NQ) * EBP + e];
        }
      }
      return make_float4(o[0], o[1], o[2], o[3]);
    };
    bool okr = true;
    if constexpr (R_SMEM) okr = mbar_wait_bounded(&bars[2], uint32_t(it & 1), err, lim);  // history landed
    if (!__syncthreads_and(okr)) {
      drain();
      return;
    }
    if constexpr (R_SMEM) pend_clr(2);
    const float a1 = a.a1, a2 = a.a2, a3 = a.a3, dt = a.dt;
    if constexpr (R_SMEM) {
      // q^{m+1} replaces r^{m-1} and r^m replaces r^{m-2} in sR, then both are bulk-stored
      for (int i = tid; i < P::nQ / 4; i += NT) {
        const float4 q4 = reinterpret_cast<const float4*>(sQ)[i];
        const float4 r4 = rhs4(i);
        float4* h1 = reinterpret_cast<float4*>(sR) + i;
        float4* h2 = reinterpret_cast<float4*>(sR + P::nQ) + i;
        const float4 p1 = *h1, p2 = *h2;
        *h1 = make_float4(fmaf(dt, a1 * r4.x + a2 * p1.x + a3 * p2.x, q4.x),
                          fmaf(dt, a1 * r4.y + a2 * p1.y + a3 * p2.y, q4.y),
                          fmaf(dt, a1 * r4.z + a2 * p1.z + a3 * p2.z, q4.z),
                          fmaf(dt, a1 * r4.w + a2 * p1.w + a3 * p2.w, q4.w));
        *h2 = r4;
      }
      fence_proxy_async_smem();
      __syncthreads();
      if (tid == 0) {
        tma_bulk_s2g(a.qn + size_t(k0) * Nf * Np, sR, kQBytes);
        tma_bulk_s2g(a.r2 + size_t(k0) * Nf * Np, sR + P::nQ, kQBytes);
        bulk_commit();
      }
    } else {
      // history from global memory (prefetched into L2 with the block's
      // stage): UB float4 per thread in flight, loads before stores
      const size_t g0 = size_t(k0) * Nf * Np / 4;
      const float4* gr1 = reinterpret_cast<const float4*>(a.r1) + g0;
      float4* gr2 = reinterpret_cast<float4*>(a.r2) + g0;
      float4* gqn = reinterpret_cast<float4*>(a.qn) + g0;
      constexpr int UB = 4;
      for (int i0 = tid; i0 < P::nQ / 4; i0 += NT * UB) {
        float4 p1[UB], p2[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int i = i0 + u * NT;
          if (i < P::nQ / 4) {
            p1[u] = __ldg(gr1 + i);
            p2[u] = gr2[i];
          }
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int i = i0 + u * NT;
          if (i < P::nQ / 4) {
            const float4 q4 = reinterpret_cast<const float4*>(sQ)[i];
            const float4 r4 = rhs4(i);
            gqn[i] = make_float4(fmaf(dt, a1 * r4.x + a2 * p1[u].x + a3 * p2[u].x, q4.x),
                                 fmaf(dt, a1 * r4.y + a2 * p1[u].y + a3 * p2[u].y, q4.y),
                                 fmaf(dt, a1 * r4.z + a2 * p1[u].z + a3 * p2[u].z, q4.z),
                                 fmaf(dt, a1 * r4.w + a2 * p1[u].w + a3 * p2[u].w, q4.w));
            gr2[i] = r4;
          }
        }
      }
    }
  }
  if (R_SMEM && tid == 0) bulk_wait_all();
}

// One solve per launch (dg_rhs / dg_step); SPLIT > 0: front half of the split
// step writing X in column tiles of SPLIT elements (FP32 rows, or XP BF16
// pieces in the tensor-core chunk layout when XP > 0).
template <int MODEL, int N, int EB, int TN, int NT, bool OPS_SMEM, bool R_SMEM, int SPLIT = 0, int XP = 0,
          bool HALO = false>
__global__ void __launch_bounds__(NT) dg_step_kernel(const StepArgs a) {
  SingleSolve p{a, EB};
  step_body<MODEL, N, EB, TN, NT, OPS_SMEM, R_SMEM, SPLIT, XP, HALO>(p);
}

// Every solve of a batch (same model and N) in one persistent launch; the
// per-solve step index, AB3 phase and buffer parity are read from device
// memory.  SPLIT > 0: front half of the batch's split step.
template <int MODEL, int N, int EB, int TN, int NT, bool OPS_SMEM, bool R_SMEM, int SPLIT = 0, bool HALO = false>
__global__ void __launch_bounds__(NT) dg_step_batched_kernel(const BatchArgs b) {
  SolveBatch p{b};
  step_body<MODEL, N, EB, TN, NT, OPS_SMEM, R_SMEM, SPLIT, 0, HALO>(p);
}

}  // namespace dgk
