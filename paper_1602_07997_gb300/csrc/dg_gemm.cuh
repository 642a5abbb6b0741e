// Split step, FP32 back half: operator products as a register-tiled GEMM over
// column tiles of elements.
//
// At high N the operator blob [Dr Ds Dt LIFT] no longer fits in shared
// memory next to a block of elements, so the fused kernel must stream it
// from L2 once per block of a few elements.  The split step instead
//   kernel A (the fused kernel's front half, SPLIT = NE): stages q, records
//     and neighbour traces as usual, computes the volume inputs, the surface
//     streams and the face normals, and writes them from its compute loops to
//     a global buffer X laid out in column tiles of NE elements:
//     X[tile][row][NE] (rows of XRows: the input indices of the products);
//   kernel B (this file; the autotuner times the designs):
//   design A: a CTA owns 32 output rows x NE elements, one thread 4 (or 8)
//     rows x TN elements of every product, double-buffered 16-deep K chunks,
//     and the combination and AB3 update in the epilogue;
//   design B: a CTA owns MT output rows x NE elements (or half of NE: HALF);
//     operator rows and X rows stream through shared memory in 16-deep K
//     chunks (16-byte cp.async, NS-stage ring, one barrier per chunk), every
//     operator row is reused by the CTA's elements and every X row by MT
//     rows.  One thread accumulates TM rows x TE elements.  The K loop runs
//     the volume chunks (D_r, D_s, D_t) and then the LIFT chunks; at the
//     boundary the accumulators of the pure derivative products are combined
//     with the element's geometric factors into the RHS components, and the
//     LIFT products accumulate onto them:
//       acoustic: G_d = D_d p and R = sum_d D_d w_d over the volume chunks;
//                 then T_c = -(1/rho) sum_d g_cd G_d; over the LIFT chunks
//                 r_p = R + LIFT P_p and, face by face, L_f = LIFT_f psi,
//                 which joins r_v,c = T_c + sum_f n_f,c L_f at each face end;
//       elastic:  U_cd = D_d v_c and Rv_c = sum_d D_d s_cd over the volume
//                 chunks; then the stress parts S (lambda div v + 2 mu dv_i/dx_i,
//                 mu (dv_i/dx_j + dv_j/dx_i)) from U; over the LIFT chunks
//                 r_v,c = Rv_c + LIFT (Fscale p_v,c) and, face by face,
//                 W_f = LIFT_f (Fscale dv), which joins the stress as
//                 lambda (n_f.W_f) I + mu (n_f W_f^T + W_f n_f^T).
//   design W: design B's narrow packed thread tile in a warp-specialised,
//     persistent CTA: a producer warp streams every chunk with 1-D bulk
//     copies into an mbarrier ring, the consumer warps (one row group each)
//     never meet a CTA-wide barrier in the K loop, and the CTA walks its
//     tiles so that the next tile's chunks land during the epilogue.
//   The epilogue stages one field at a time in shared memory and runs the
//   point source and the AB3 update (Eq. updateScheme) with coalesced accesses.
#pragma once

#include "dg_kernels.cuh"

namespace dgk {

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
template <int K>
__device__ __forceinline__ void cp_async_wait_n() {
  asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

// Two FP32 FMAs lane by lane, d = a b + c: one packed instruction
// (fma.rn.f32x2) when PK, else two scalar FMAs; the same rounding either way.
template <bool PK>
__device__ __forceinline__ float2 fma2(const float2 a, const float2 b, const float2 c) {
  if constexpr (PK) return __ffma2_rn(a, b, c);
  else return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 dup2(const float x) { return make_float2(x, x); }

// AB3 update (a.mode 0) or RHS store (mode 1) of U values: every load of the
// batch is issued before the first store, so that their latencies overlap.
template <int U>
__device__ __forceinline__ void ab3_batch(const StepArgs& a, const size_t* idx, const float* rv, const bool* on) {
  if (a.mode == 0) {
    float q[U], r1[U], r2[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      q[u] = on[u] ? __ldg(a.q + idx[u]) : 0.f;
      r1[u] = on[u] ? __ldg(a.r1 + idx[u]) : 0.f;
      r2[u] = on[u] ? a.r2[idx[u]] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (on[u]) {
        const float accv = a.a1 * rv[u] + a.a2 * r1[u] + a.a3 * r2[u];
        a.qn[idx[u]] = fmaf(a.dt, accv, q[u]);
        a.r2[idx[u]] = rv[u];
      }
  } else {
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (on[u]) a.rout[idx[u]] = rv[u];
  }
}

// The AB3 inputs of NE elements from element k0 into L2 while their products
// run (q, r^{m-1}, r^{m-2} are padded past K: a whole tile stays inside the
// allocation).  The GEMMs issue it a few K chunks before a tile's epilogue
// (ab3_prefetch_chunk): issued when the tile starts, the lines had left L2
// again by the time the epilogue read them (measured: no faster than no
// prefetch at all; 1-3 % faster steps at N = 5..8 issued late).
template <int Nf, int Np, int NE>
__device__ __forceinline__ void prefetch_tile_l2(const StepArgs& a, int k0) {
  const size_t e0 = size_t(k0) * Nf * Np;
  constexpr uint32_t bytes = uint32_t(NE * Nf * Np * 4);
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.q + e0), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.r1 + e0), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.r2 + e0), "r"(bytes) : "memory");
}

// Layout shared by the front half, both GEMM designs and the library route:
// X[tile][row][NE] (the KX rows of XRows per element) and the operator blob
// [3 Np + 4 Nfp][OPP] (row = input index, column = output node, OPP = Np
// rounded up to 32, enough for every design's row tiles).
template <int MODEL, int N>
struct SplitShape {
  using S = Sz<N>;
  static constexpr int Np = S::Np, NFN = S::NFN;
  static constexpr int Nf = MODEL == 0 ? 4 : 9;
  static constexpr int NV = XRows<MODEL, N>::NV;      // X rows per volume index j
  static constexpr int KX = XRows<MODEL, N>::KX;      // X rows per element
  static constexpr int NE = MODEL == 0 ? 64 : 32;      // elements per column tile
  static constexpr int OPP = (Np + 31) / 32 * 32;      // row pitch of the operator blob
  static constexpr size_t x_floats_per_tile = size_t(KX) * NE;
};

template <int MODEL, int N>
struct GemmA {
  using S = Sz<N>;
  static constexpr int Nf = MODEL == 0 ? 4 : 9;
  static constexpr int NV = XRows<MODEL, N>::NV;          // X rows per volume index j
  static constexpr int KX = XRows<MODEL, N>::KX;          // X rows per element
  static constexpr int NE = MODEL == 0 ? 64 : 32;         // elements per column tile
  static constexpr int TN = MODEL == 0 ? 2 : 1;           // elements per thread tile
  static constexpr int RQ = MODEL == 0 ? 1 : 2;           // row quads per thread tile (4 or 8 rows)
  static constexpr int MT = 32;                           // output rows per CTA
  static constexpr int MP2 = (S::Np + MT - 1) / MT * MT;  // padded rows of the split operator blob
  static constexpr int JC = 16;                           // volume indices per chunk
  static constexpr int CC = 16;                           // face-node indices per chunk
  static constexpr int NT = (MT / (4 * RQ)) * (NE / TN);  // threads per CTA
  static constexpr int NVC = (S::Np + JC - 1) / JC;       // volume chunks
  static constexpr int NLC = (S::NFN + CC - 1) / CC;      // lift chunks
  static constexpr int MINB = 1;                          // resident CTAs the registers are sized for
  static constexpr int MTILES_L = (S::Np + MT - 1) / MT;  // row tiles (launch grid: x column tiles)
  // per buffer: A rows (3 JC volume, CC lift) x MT, X rows (NV JC volume;
  // lift: 2 CC streams + 12 normal rows acoustic, Nf CC elastic) x NE
  static constexpr int nA = (3 * JC > CC ? 3 * JC : CC) * MT;
  static constexpr int LB = XRows<MODEL, N>::NXS * CC + 12;
  static constexpr int nB = (NV * JC > LB ? NV * JC : LB) * NE;
  static constexpr int NEP = NE + (TN == 2 ? 2 : 1);       // row stride of the staged RHS tile
  static constexpr int nOut = Nf * MT * NEP;              // RHS tile [Nf][MT][NEP], reuses the B buffers
  static constexpr int nBB = (2 * nB > nOut ? 2 * nB : nOut);
  static constexpr size_t smem = size_t(2 * nA + nBB) * 4;
  static constexpr size_t x_floats_per_tile = size_t(KX) * NE;
};

template <int MODEL, int N>
__device__ __forceinline__ void gemm_a_body(const StepArgs& a, const int mtile, const int ntile) {
  using S = Sz<N>;
  using SS = GemmA<MODEL, N>;
  constexpr int Np = S::Np, NFN = S::NFN, Nf = SS::Nf, NV = SS::NV, NE = SS::NE, TN = SS::TN, RQ = SS::RQ;
  constexpr int Nfp = S::Nfp, NXS = XRows<MODEL, N>::NXS, KXM = XRows<MODEL, N>::KXM;
  constexpr int RV = 4 * RQ;  // rows per thread
  constexpr int MT = SS::MT, MP2 = SplitShape<MODEL, N>::OPP, JC = SS::JC, CC = SS::CC, NT = SS::NT;
  constexpr int NVC = SS::NVC, NLC = SS::NLC, NCH = NVC + NLC;
  constexpr int REC = Rec<MODEL>::size;

  extern __shared__ __align__(16) float smem[];
  float* sA[2] = {smem, smem + SS::nA};
  float* sB[2] = {smem + 2 * SS::nA, smem + 2 * SS::nA + SS::nB};

  const int tid = threadIdx.x;
  const int row0 = mtile * MT;
  const float* X = a.xg + size_t(ntile) * SplitShape<MODEL, N>::x_floats_per_tile;
  const float* OP = a.ops2;  // [3 Np + NFN][MP2]
  if (tid == 0 && mtile == 0 && a.mode == 0) prefetch_tile_l2<Nf, Np, NE>(a, ntile * NE);

  // chunk c -> shared buffer (c & 1)
  auto issue = [&](int c) {
    float* A = sA[c & 1];
    float* B = sB[c & 1];
    if (c < NVC) {
      const int j0 = c * JC;
      const int nj = Np - j0 < JC ? Np - j0 : JC;
      // A rows d*Np + j, j in [j0, j0+nj): MT columns from row0
      for (int i = tid; i < 3 * nj * (MT / 4); i += NT) {
        const int q4 = i % (MT / 4), rr = i / (MT / 4);
        const int d = rr / nj, jj = rr - d * nj;
        cp_async16(A + (d * JC + jj) * MT + 4 * q4, OP + size_t(d * Np + j0 + jj) * MP2 + row0 + 4 * q4);
      }
      // X rows f*Np + j for f < NV
      for (int i = tid; i < NV * nj * (NE / 4); i += NT) {
        const int q4 = i % (NE / 4), rr = i / (NE / 4);
        const int f = rr / nj, jj = rr - f * nj;
        cp_async16(B + (f * JC + jj) * NE + 4 * q4, X + size_t(f * Np + j0 + jj) * NE + 4 * q4);
      }
    } else {
      const int c0 = (c - NVC) * CC;
      const int nc = NFN - c0 < CC ? NFN - c0 : CC;
      for (int i = tid; i < nc * (MT / 4); i += NT) {
        const int q4 = i % (MT / 4), cc = i / (MT / 4);
        cp_async16(A + cc * MT + 4 * q4, OP + size_t(3 * Np + c0 + cc) * MP2 + row0 + 4 * q4);
      }
      for (int i = tid; i < NXS * nc * (NE / 4); i += NT) {
        const int q4 = i % (NE / 4), rr = i / (NE / 4);
        const int f = rr / nc, cc = rr - f * nc;
        cp_async16(B + (f * CC + cc) * NE + 4 * q4, X + size_t(NV * Np + f * NFN + c0 + cc) * NE + 4 * q4);
      }
      // the face normals, after the streams
      for (int i = tid; i < 12 * (NE / 4); i += NT) {
        const int q4 = i % (NE / 4), r = i / (NE / 4);
        cp_async16(B + (NXS * CC + r) * NE + 4 * q4, X + size_t(KXM + r) * NE + 4 * q4);
      }
    }
    cp_async_commit();
  };

  // thread tile: rows il..il+RV-1 of this CTA's slice, elements e0..e0+TN-1 of the
  // column tile; lanes of a warp share the row tile (broadcast operator reads)
  // and walk the elements
  const int ct = tid % (NE / TN), rt = tid / (NE / TN);
  const int il = RV * rt, e0 = ct * TN;

  constexpr int NACC = MODEL == 0 ? 7 : 12;  // acoustic G0..2, R, L0..2; elastic U00..U22, Rv0..2
  float acc[NACC][TN][RV];
  float lf[TN][RV];  // acoustic: LIFT_f psi of the current face f
#pragma unroll
  for (int t = 0; t < TN; ++t)
#pragma unroll
    for (int v = 0; v < RV; ++v) lf[t][v] = 0.f;
#pragma unroll
  for (int x = 0; x < NACC; ++x)
#pragma unroll
    for (int t = 0; t < TN; ++t)
#pragma unroll
      for (int v = 0; v < RV; ++v) acc[x][t][v] = 0.f;
  float accS[MODEL == 0 ? 1 : 6][TN][RV];  // elastic LIFT P_sigma
  float W[MODEL == 0 ? 1 : 3][TN][RV];     // elastic LIFT_f (Fscale dv) of the current face f
#pragma unroll
  for (int x = 0; x < (MODEL == 0 ? 1 : 6); ++x)
#pragma unroll
    for (int t = 0; t < TN; ++t)
#pragma unroll
      for (int v = 0; v < RV; ++v) accS[x][t][v] = 0.f;
#pragma unroll
  for (int x = 0; x < (MODEL == 0 ? 1 : 3); ++x)
#pragma unroll
    for (int t = 0; t < TN; ++t)
#pragma unroll
      for (int v = 0; v < RV; ++v) W[x][t][v] = 0.f;

  issue(0);
  for (int c = 0; c < NCH; ++c) {
    if (c + 1 < NCH) {
      issue(c + 1);
      cp_async_wait_n<1>();
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    const float* A = sA[c & 1] + il;
    const float* B = sB[c & 1] + e0;
    if (c < NVC) {
      const int j0 = c * JC;
      const int nj = Np - j0 < JC ? Np - j0 : JC;
#pragma unroll 2
      for (int jj = 0; jj < nj; ++jj) {
        float4 ad[3][RQ];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int q = 0; q < RQ; ++q) ad[d][q] = *reinterpret_cast<const float4*>(A + (d * JC + jj) * MT + 4 * q);
        if constexpr (MODEL == 0) {
          float xpv[TN], x0v[TN], x1v[TN], x2v[TN];
          VecT<TN>::load(B + (0 * JC + jj) * NE, xpv);
          VecT<TN>::load(B + (1 * JC + jj) * NE, x0v);
          VecT<TN>::load(B + (2 * JC + jj) * NE, x1v);
          VecT<TN>::load(B + (3 * JC + jj) * NE, x2v);
#pragma unroll
          for (int t = 0; t < TN; ++t)
#pragma unroll
            for (int q = 0; q < RQ; ++q) {
              const float xp = xpv[t], x0 = x0v[t], x1 = x1v[t], x2 = x2v[t];
              fma4(&acc[0][t][4 * q], ad[0][q], xp);
              fma4(&acc[1][t][4 * q], ad[1][q], xp);
              fma4(&acc[2][t][4 * q], ad[2][q], xp);
              fma4(&acc[3][t][4 * q], ad[0][q], x0);
              fma4(&acc[3][t][4 * q], ad[1][q], x1);
              fma4(&acc[3][t][4 * q], ad[2][q], x2);
            }
        } else {
#pragma unroll
          for (int t = 0; t < TN; ++t)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
              const float xv = B[(cc * JC + jj) * NE + t];
              const float s0 = B[((3 + 3 * cc + 0) * JC + jj) * NE + t];
              const float s1 = B[((3 + 3 * cc + 1) * JC + jj) * NE + t];
              const float s2 = B[((3 + 3 * cc + 2) * JC + jj) * NE + t];
#pragma unroll
              for (int q = 0; q < RQ; ++q) {
                fma4(&acc[3 * cc + 0][t][4 * q], ad[0][q], xv);
                fma4(&acc[3 * cc + 1][t][4 * q], ad[1][q], xv);
                fma4(&acc[3 * cc + 2][t][4 * q], ad[2][q], xv);
                fma4(&acc[9 + cc][t][4 * q], ad[0][q], s0);
                fma4(&acc[9 + cc][t][4 * q], ad[1][q], s1);
                fma4(&acc[9 + cc][t][4 * q], ad[2][q], s2);
              }
            }
        }
      }
    } else {
      const int c0 = (c - NVC) * CC;
      const int nc = NFN - c0 < CC ? NFN - c0 : CC;
      if constexpr (MODEL == 0) {
        // P_p onto R; psi face by face onto lf, which joins the velocity
        // accumulators L_c as n_f,c lf once face f is complete
        int cc = 0;
        while (cc < nc) {
          const int f = (c0 + cc) / Nfp;
          const int fe = (f + 1) * Nfp - c0;  // end of face f, chunk-relative
          const int ce = fe < nc ? fe : nc;
#pragma unroll 2
          for (; cc < ce; ++cc) {
            float4 l[RQ];
#pragma unroll
            for (int q = 0; q < RQ; ++q) l[q] = *reinterpret_cast<const float4*>(A + cc * MT + 4 * q);
            float p0[TN], p1[TN];
            VecT<TN>::load(B + (0 * CC + cc) * NE, p0);
            VecT<TN>::load(B + (1 * CC + cc) * NE, p1);
#pragma unroll
            for (int t = 0; t < TN; ++t)
#pragma unroll
              for (int q = 0; q < RQ; ++q) {
                fma4(&acc[3][t][4 * q], l[q], p0[t]);
                fma4(&lf[t][4 * q], l[q], p1[t]);
              }
          }
          if (cc == fe) {
#pragma unroll
            for (int x = 0; x < 3; ++x) {
              float nv[TN];
              VecT<TN>::load(B + (2 * CC + 3 * f + x) * NE, nv);
#pragma unroll
              for (int t = 0; t < TN; ++t)
#pragma unroll
                for (int v = 0; v < RV; ++v) acc[4 + x][t][v] = fmaf(nv[t], lf[t][v], acc[4 + x][t][v]);
            }
#pragma unroll
            for (int t = 0; t < TN; ++t)
#pragma unroll
              for (int v = 0; v < RV; ++v) lf[t][v] = 0.f;
          }
        }
      } else {
        // Fscale p_v onto Rv; Fscale dv face by face onto W, which joins the
        // stress LIFT as lambda (n.W) I + mu (n W^T + W n^T) at the face end
        int cc = 0;
        while (cc < nc) {
          const int f = (c0 + cc) / Nfp;
          const int fe = (f + 1) * Nfp - c0;  // end of face f, chunk-relative
          const int ce = fe < nc ? fe : nc;
#pragma unroll 2
          for (; cc < ce; ++cc) {
            float4 l[RQ];
#pragma unroll
            for (int q = 0; q < RQ; ++q) l[q] = *reinterpret_cast<const float4*>(A + cc * MT + 4 * q);
#pragma unroll
            for (int t = 0; t < TN; ++t) {
#pragma unroll
              for (int x = 0; x < 3; ++x) {
                const float p = B[(x * CC + cc) * NE + t];
#pragma unroll
                for (int q = 0; q < RQ; ++q) fma4(&acc[9 + x][t][4 * q], l[q], p);
              }
#pragma unroll
              for (int x = 0; x < 3; ++x) {
                const float p = B[((3 + x) * CC + cc) * NE + t];
#pragma unroll
                for (int q = 0; q < RQ; ++q) fma4(&W[x][t][4 * q], l[q], p);
              }
            }
          }
          if (cc == fe) {
#pragma unroll
            for (int t = 0; t < TN; ++t) {
              const int k = ntile * NE + e0 + t;
              const float* gk = a.rec + size_t(k < a.K ? k : a.K - 1) * REC;
              const float lam = __ldg(gk + 9), mu = __ldg(gk + 10);
              const float nx = B[(NXS * CC + 3 * f + 0) * NE + t], ny = B[(NXS * CC + 3 * f + 1) * NE + t],
                          nz = B[(NXS * CC + 3 * f + 2) * NE + t];
#pragma unroll
              for (int v = 0; v < RV; ++v) {
                const float w0 = W[0][t][v], w1 = W[1][t][v], w2 = W[2][t][v];
                const float lnw = lam * (nx * w0 + ny * w1 + nz * w2);
                accS[0][t][v] += lnw + 2.f * mu * nx * w0;
                accS[1][t][v] += lnw + 2.f * mu * ny * w1;
                accS[2][t][v] += lnw + 2.f * mu * nz * w2;
                accS[3][t][v] += mu * (nx * w1 + ny * w0);
                accS[4][t][v] += mu * (nx * w2 + nz * w0);
                accS[5][t][v] += mu * (ny * w2 + nz * w1);
                W[0][t][v] = W[1][t][v] = W[2][t][v] = 0.f;
              }
            }
          }
        }
      }
    }
    __syncthreads();  // buffer (c & 1) is refilled by chunk c + 2
  }

  // -------- epilogue, part 1: geometric combination and source in registers;
  // the RHS tile goes to shared memory as [Nf][MT][NEP] (element fastest)
  float* sOut = smem + 2 * SS::nA;
  constexpr int NEP = SS::NEP;
#pragma unroll
  for (int t = 0; t < TN; ++t) {
    const int k = ntile * NE + e0 + t;
    const int kk = k < a.K ? k : a.K - 1;  // padding columns: any valid record
    const float* gk = a.rec + size_t(kk) * REC;
    float g[9];
#pragma unroll
    for (int x = 0; x < 9; ++x) g[x] = __ldg(gk + x);
    const bool src = (k == a.src_elem) && a.srcvec;
#pragma unroll
    for (int v = 0; v < RV; ++v) {
      const int i = row0 + il + v;
      float r[Nf];
      if constexpr (MODEL == 0) {
        const float rinv = __ldg(gk + 10);
        r[0] = acc[3][t][v];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
          r[1 + cc] = acc[4 + cc][t][v] -
                      rinv * (g[3 * cc] * acc[0][t][v] + g[3 * cc + 1] * acc[1][t][v] + g[3 * cc + 2] * acc[2][t][v]);
      } else {
        const float lam = __ldg(gk + 9), mu = __ldg(gk + 10);
        float gv[3][3];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
#pragma unroll
          for (int x = 0; x < 3; ++x)
            gv[cc][x] = g[3 * x] * acc[3 * cc][t][v] + g[3 * x + 1] * acc[3 * cc + 1][t][v] +
                        g[3 * x + 2] * acc[3 * cc + 2][t][v];
        const float div = gv[0][0] + gv[1][1] + gv[2][2];
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) r[cc] = acc[9 + cc][t][v];
        r[3] = lam * div + 2.f * mu * gv[0][0] + accS[0][t][v];
        r[4] = lam * div + 2.f * mu * gv[1][1] + accS[1][t][v];
        r[5] = lam * div + 2.f * mu * gv[2][2] + accS[2][t][v];
        r[6] = mu * (gv[0][1] + gv[1][0]) + accS[3][t][v];
        r[7] = mu * (gv[0][2] + gv[2][0]) + accS[4][t][v];
        r[8] = mu * (gv[1][2] + gv[2][1]) + accS[5][t][v];
      }
      if (src && i < Np) {
#pragma unroll
        for (int f = 0; f < Nf; ++f) r[f] = fmaf(a.src_amp, __ldg(a.srcvec + f * Np + i), r[f]);
      }
#pragma unroll
      for (int f = 0; f < Nf; ++f) sOut[(f * MT + il + v) * NEP + e0 + t] = r[f];
    }
  }
  __syncthreads();
  // part 2: coalesced AB3 update over (element, field, row), rows fastest,
  // 8 values per thread in flight
  const int rows = (Np - row0) < MT ? (Np - row0) : MT;
  const int total = NE * Nf * rows;
  constexpr int U = 8;
  for (int v0 = tid; v0 < total; v0 += NT * U) {
    size_t idx[U];
    float rv[U];
    bool on[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int v = v0 + u * NT;
      const int rr = v % rows, ef = v / rows;
      const int e = ef / Nf, f = ef - e * Nf;
      const int k = ntile * NE + e;
      on[u] = v < total && k < a.K;
      idx[u] = on[u] ? size_t(k) * Nf * Np + size_t(f) * Np + row0 + rr : 0;
      rv[u] = on[u] ? sOut[(f * MT + rr) * NEP + e] : 0.f;
    }
    ab3_batch<U>(a, idx, rv, on);
  }
}

// Register tile of design B's (and W's) operator products: TM rows x TE
// element columns of every accumulator, in pairs of consecutive rows (the
// operands of the packed FMAs).  The chunk walks read a stage in shared
// memory: A = operator rows [KC-deep chunk][MTS] from the thread's first row,
// B = X rows [vector][KC][NES] from the thread's first element.
template <int MODEL, int N, int TM, int TE, bool PK, int MTS, int NES>
struct ProdTile {
  static constexpr int Np = Sz<N>::Np, NFN = Sz<N>::NFN, Nfp = Sz<N>::Nfp;
  static constexpr int KC = 16;
  static constexpr int NXS = XRows<MODEL, N>::NXS;
  static constexpr int NACC = MODEL == 0 ? 4 : 12;
  static constexpr int REC = Rec<MODEL>::size;
  static constexpr int kTM = TM, kTE = TE;
  // acoustic: 0..2 G_d then T_c (velocity), 3 R then r_p; elastic: 0..8
  // U_cd then the stress components (0..5) and W (6..8), 9..11 Rv_c
  float2 acc2[NACC][TE][TM / 2];
  float2 lf2[MODEL == 0 ? TE : 1][TM / 2];  // acoustic: LIFT_f psi of the current face f
  float lamv[TE], muv[TE];                  // elastic: Lame coefficients of the element columns

  // row v of element column t of accumulator x
  __device__ __forceinline__ float& acc(int x, int t, int v) {
    return (v & 1) ? acc2[x][t][v >> 1].y : acc2[x][t][v >> 1].x;
  }
  // accumulator holding field f of the RHS once the K loop is done
  __device__ static constexpr int slot_of_field(int f) {
    return MODEL == 0 ? (f == 0 ? 3 : f - 1) : (f < 3 ? 9 + f : f - 3);
  }

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int x = 0; x < NACC; ++x)
#pragma unroll
      for (int t = 0; t < TE; ++t)
#pragma unroll
        for (int v = 0; v < TM / 2; ++v) acc2[x][t][v] = make_float2(0.f, 0.f);
#pragma unroll
    for (int t = 0; t < (MODEL == 0 ? TE : 1); ++t)
#pragma unroll
      for (int v = 0; v < TM / 2; ++v) lf2[t][v] = make_float2(0.f, 0.f);
  }

  __device__ __forceinline__ static void ldA(const float* p, float2* o) {  // TM rows as float4s, in row pairs
#pragma unroll
    for (int q = 0; q < TM / 4; ++q) {
      const float4 v = *reinterpret_cast<const float4*>(p + 4 * q);
      o[2 * q] = make_float2(v.x, v.y);
      o[2 * q + 1] = make_float2(v.z, v.w);
    }
  }
  __device__ __forceinline__ static void ldB(const float* p, float* o) {  // TE consecutive elements
    if constexpr (TE == 4) {
      const float4 v = *reinterpret_cast<const float4*>(p);
      o[0] = v.x;
      o[1] = v.y;
      o[2] = v.z;
      o[3] = v.w;
    } else if constexpr (TE == 2) {
      const float2 v = *reinterpret_cast<const float2*>(p);
      o[0] = v.x;
      o[1] = v.y;
    } else {
      o[0] = *p;
    }
  }

  // a volume chunk of nj indices j: acoustic G_d += D_d p, R += sum_d D_d w_d;
  // elastic U_cd += D_d v_c, Rv_c += sum_d D_d s_cd
  __device__ __forceinline__ void volume(const float* A, const float* B, const int nj) {
#pragma unroll 2
    for (int jj = 0; jj < nj; ++jj) {
      float2 ad[3][TM / 2];
#pragma unroll
      for (int d = 0; d < 3; ++d) ldA(A + (d * KC + jj) * MTS, ad[d]);
      if constexpr (MODEL == 0) {
        float xp[TE], xw[3][TE];
        ldB(B + (0 * KC + jj) * NES, xp);
#pragma unroll
        for (int d = 0; d < 3; ++d) ldB(B + ((1 + d) * KC + jj) * NES, xw[d]);
#pragma unroll
        for (int t = 0; t < TE; ++t) {
          const float2 p2 = dup2(xp[t]), w0 = dup2(xw[0][t]), w1 = dup2(xw[1][t]), w2 = dup2(xw[2][t]);
#pragma unroll
          for (int v = 0; v < TM / 2; ++v) {
            acc2[0][t][v] = fma2<PK>(ad[0][v], p2, acc2[0][t][v]);
            acc2[1][t][v] = fma2<PK>(ad[1][v], p2, acc2[1][t][v]);
            acc2[2][t][v] = fma2<PK>(ad[2][v], p2, acc2[2][t][v]);
            acc2[3][t][v] = fma2<PK>(ad[0][v], w0, acc2[3][t][v]);
            acc2[3][t][v] = fma2<PK>(ad[1][v], w1, acc2[3][t][v]);
            acc2[3][t][v] = fma2<PK>(ad[2][v], w2, acc2[3][t][v]);
          }
        }
      } else {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
          float xv[TE], xs[3][TE];
          ldB(B + (cc * KC + jj) * NES, xv);
#pragma unroll
          for (int d = 0; d < 3; ++d) ldB(B + ((3 + 3 * cc + d) * KC + jj) * NES, xs[d]);
#pragma unroll
          for (int t = 0; t < TE; ++t) {
            const float2 v2 = dup2(xv[t]), s0 = dup2(xs[0][t]), s1 = dup2(xs[1][t]), s2 = dup2(xs[2][t]);
#pragma unroll
            for (int v = 0; v < TM / 2; ++v) {
              acc2[3 * cc + 0][t][v] = fma2<PK>(ad[0][v], v2, acc2[3 * cc + 0][t][v]);
              acc2[3 * cc + 1][t][v] = fma2<PK>(ad[1][v], v2, acc2[3 * cc + 1][t][v]);
              acc2[3 * cc + 2][t][v] = fma2<PK>(ad[2][v], v2, acc2[3 * cc + 2][t][v]);
              acc2[9 + cc][t][v] = fma2<PK>(ad[0][v], s0, acc2[9 + cc][t][v]);
              acc2[9 + cc][t][v] = fma2<PK>(ad[1][v], s1, acc2[9 + cc][t][v]);
              acc2[9 + cc][t][v] = fma2<PK>(ad[2][v], s2, acc2[9 + cc][t][v]);
            }
          }
        }
      }
    }
  }

  // volume/LIFT boundary: the derivative products -> RHS components with the
  // geometric factors of element column t (element k0 + t)
  __device__ __forceinline__ void boundary(const StepArgs& a, const int k0) {
#pragma unroll
    for (int t = 0; t < TE; ++t) {
      const int k = k0 + t;
      const int kk = k < a.K ? k : a.K - 1;  // padding columns: any valid record
      const float* gk = a.rec + size_t(kk) * REC;
      float g[9];
#pragma unroll
      for (int x = 0; x < 9; ++x) g[x] = __ldg(gk + x);
      if constexpr (MODEL == 0) {
        const float rinv = __ldg(gk + 10);
#pragma unroll
        for (int v = 0; v < TM; ++v) {
          const float G0 = acc(0, t, v), G1 = acc(1, t, v), G2 = acc(2, t, v);
#pragma unroll
          for (int cc = 0; cc < 3; ++cc)
            acc(cc, t, v) = -rinv * (g[3 * cc] * G0 + g[3 * cc + 1] * G1 + g[3 * cc + 2] * G2);
        }
      } else {
        const float lam = __ldg(gk + 9), mu = __ldg(gk + 10);
        lamv[t] = lam;
        muv[t] = mu;
#pragma unroll
        for (int v = 0; v < TM; ++v) {
          float gv[3][3];
#pragma unroll
          for (int cc = 0; cc < 3; ++cc)
#pragma unroll
            for (int x = 0; x < 3; ++x)
              gv[cc][x] = g[3 * x] * acc(3 * cc, t, v) + g[3 * x + 1] * acc(3 * cc + 1, t, v) +
                          g[3 * x + 2] * acc(3 * cc + 2, t, v);
          const float div = gv[0][0] + gv[1][1] + gv[2][2];
          acc(0, t, v) = lam * div + 2.f * mu * gv[0][0];
          acc(1, t, v) = lam * div + 2.f * mu * gv[1][1];
          acc(2, t, v) = lam * div + 2.f * mu * gv[2][2];
          acc(3, t, v) = mu * (gv[0][1] + gv[1][0]);
          acc(4, t, v) = mu * (gv[0][2] + gv[2][0]);
          acc(5, t, v) = mu * (gv[1][2] + gv[2][1]);
          acc(6, t, v) = acc(7, t, v) = acc(8, t, v) = 0.f;  // W: LIFT_f dv of the current face
        }
      }
    }
  }

  // a LIFT chunk of nc face nodes from face node c0; the chunk's face normals
  // follow its streams in B (rows NXS KC + 3 f + c)
  __device__ __forceinline__ void lift(const float* A, const float* B, const int c0, const int nc) {
    if constexpr (MODEL == 0) {
      // P_p onto r_p; psi face by face onto lf, which joins the velocity
      // components as n_f,c lf once face f is complete
      int cc = 0;
      while (cc < nc) {
        const int f = (c0 + cc) / Nfp;
        const int fe = (f + 1) * Nfp - c0;  // end of face f, chunk-relative
        const int ce = fe < nc ? fe : nc;
#pragma unroll 2
        for (; cc < ce; ++cc) {
          float2 l[TM / 2];
          float pp[TE], ps[TE];
          ldA(A + cc * MTS, l);
          ldB(B + (0 * KC + cc) * NES, pp);
          ldB(B + (1 * KC + cc) * NES, ps);
#pragma unroll
          for (int t = 0; t < TE; ++t) {
            const float2 p2 = dup2(pp[t]), s2 = dup2(ps[t]);
#pragma unroll
            for (int v = 0; v < TM / 2; ++v) {
              acc2[3][t][v] = fma2<PK>(l[v], p2, acc2[3][t][v]);
              lf2[t][v] = fma2<PK>(l[v], s2, lf2[t][v]);
            }
          }
        }
        if (cc == fe) {
#pragma unroll
          for (int x = 0; x < 3; ++x) {
            float nv[TE];
            ldB(B + (NXS * KC + 3 * f + x) * NES, nv);
#pragma unroll
            for (int t = 0; t < TE; ++t) {
              const float2 n2 = dup2(nv[t]);
#pragma unroll
              for (int v = 0; v < TM / 2; ++v) acc2[x][t][v] = fma2<PK>(n2, lf2[t][v], acc2[x][t][v]);
            }
          }
#pragma unroll
          for (int t = 0; t < TE; ++t)
#pragma unroll
            for (int v = 0; v < TM / 2; ++v) lf2[t][v] = make_float2(0.f, 0.f);
        }
      }
    } else {
      // Fscale p_v onto Rv (accumulators 9..11); Fscale dv face by face
      // onto W (6..8), which joins the stress components as
      // lambda (n.W) I + mu (n W^T + W n^T) once face f is complete
      int cc = 0;
      while (cc < nc) {
        const int f = (c0 + cc) / Nfp;
        const int fe = (f + 1) * Nfp - c0;  // end of face f, chunk-relative
        const int ce = fe < nc ? fe : nc;
#pragma unroll 2
        for (; cc < ce; ++cc) {
          float2 l[TM / 2];
          ldA(A + cc * MTS, l);
#pragma unroll
          for (int x = 0; x < 6; ++x) {
            float pf[TE];
            ldB(B + (x * KC + cc) * NES, pf);
            const int slot = x < 3 ? 9 + x : 3 + x;
#pragma unroll
            for (int t = 0; t < TE; ++t) {
              const float2 p2 = dup2(pf[t]);
#pragma unroll
              for (int v = 0; v < TM / 2; ++v) acc2[slot][t][v] = fma2<PK>(l[v], p2, acc2[slot][t][v]);
            }
          }
        }
        if (cc == fe) {
          float nv[3][TE];
#pragma unroll
          for (int x = 0; x < 3; ++x) ldB(B + (NXS * KC + 3 * f + x) * NES, nv[x]);
#pragma unroll
          for (int t = 0; t < TE; ++t)
#pragma unroll
            for (int v = 0; v < TM; ++v) {
              const float w0 = acc(6, t, v), w1 = acc(7, t, v), w2 = acc(8, t, v);
              const float nx = nv[0][t], ny = nv[1][t], nz = nv[2][t];
              const float lnw = lamv[t] * (nx * w0 + ny * w1 + nz * w2), m2 = 2.f * muv[t];
              acc(0, t, v) += lnw + m2 * nx * w0;
              acc(1, t, v) += lnw + m2 * ny * w1;
              acc(2, t, v) += lnw + m2 * nz * w2;
              acc(3, t, v) += muv[t] * (nx * w1 + ny * w0);
              acc(4, t, v) += muv[t] * (nx * w2 + nz * w0);
              acc(5, t, v) += muv[t] * (ny * w2 + nz * w1);
              acc(6, t, v) = acc(7, t, v) = acc(8, t, v) = 0.f;
            }
        }
      }
    }
  }
};

// Epilogue of a product tile: one field at a time through shared memory
// sOut[MT][NEP] (rows il.. of the thread tile, element columns e0..), then the
// point source and the AB3 update (or the RHS store) with the tile's values
// spread over the NTH threads (index th) in element-major order, so that
// consecutive threads touch consecutive nodes.  sync() makes the staged field
// visible to, and later free from, every one of the NTH threads.
template <int MODEL, int N, int MT, int NE, int NEP, int NTH, class PT, class Sync>
__device__ __forceinline__ void tile_epilogue(const StepArgs& a, PT& pt, float* sOut, const int th, const int il,
                                              const int e0, const int row0, const int kbase, Sync sync) {
  constexpr int Np = Sz<N>::Np, Nf = MODEL == 0 ? 4 : 9;
  const int rows = (Np - row0) < MT ? (Np - row0) : MT;
#pragma unroll
  for (int f = 0; f < Nf; ++f) {
    const int slot = PT::slot_of_field(f);
#pragma unroll
    for (int t = 0; t < PT::kTE; ++t)
#pragma unroll
      for (int v = 0; v < PT::kTM; ++v)
        sOut[(il + v) * NEP + e0 + t] = pt.acc(slot, t, v);
    sync();
    constexpr int U = 8;  // values per thread in flight
    for (int p0 = th; p0 < NE * MT; p0 += NTH * U) {
      size_t idx[U];
      float rv[U];
      bool on[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int p = p0 + u * NTH;
        const int e = p / MT, rr = p - e * MT;
        const int k = kbase + e;
        on[u] = p < NE * MT && k < a.K && rr < rows;
        const int i = row0 + rr;
        float r = on[u] ? sOut[rr * NEP + e] : 0.f;
        if (on[u] && k == a.src_elem && a.srcvec) r = fmaf(a.src_amp, __ldg(a.srcvec + f * Np + i), r);
        rv[u] = r;
        idx[u] = on[u] ? size_t(k) * Nf * Np + size_t(f) * Np + i : 0;
      }
      ab3_batch<U>(a, idx, rv, on);
    }
    sync();
  }
}

// NARROW: elements per thread halved (fewer registers, two CTAs per SM).
// SMALL (narrow only): short row tiles that divide Np (almost) exactly and
// registers sized for two resident CTAs per SM.  HALF (narrow only): a CTA
// takes half of a column tile of X (32 acoustic elements), so that two CTAs
// fit per SM with the registers of the narrow design.
template <int MODEL, int N, bool NARROW = false, bool SMALL = false, bool HALF = false, bool PK = false,
          bool THIRD = false>
struct GemmB {
  using S = Sz<N>;
  static constexpr int Np = S::Np, NFN = S::NFN;
  static constexpr int Nf = MODEL == 0 ? 4 : 9;
  static constexpr int NV = XRows<MODEL, N>::NV;          // X rows per volume index j
  static constexpr int KX = XRows<MODEL, N>::KX;          // X rows per element
  static constexpr int NE = MODEL == 0 ? 64 : 32;         // elements per column tile of X
  static constexpr int NSUB = HALF ? 2 : 1;               // CTAs per column tile
  static constexpr int NEG = NE / NSUB;                   // elements per CTA
  static constexpr int TM = MODEL == 0 ? 8 : 4;           // rows per thread tile
  static constexpr int TE = (MODEL == 0 ? 4 : 2) / (NARROW ? 2 : 1);  // elements per thread tile
  // output rows per CTA (MT / TM even, so that the CTA is whole warps)
  static constexpr int MT_WIDE =
      MODEL == 0 ? (N <= 2 ? 16 : N == 3 ? 32 : N == 4 ? 48 : N == 5 ? 64 : N == 6 ? 96 : N == 7 ? 128 : 96)
                 : (N <= 3 ? 24 : N == 4 ? 40 : N == 5 ? 56 : N == 6 ? 48 : N == 7 ? 64 : 56);
  // narrow: a warp is one row group of 32 elements, so any multiple of TM
  // rows makes whole warps; row tiles close to Np / ceil(Np / MT_WIDE) waste
  // fewer padding rows (acoustic Np = 84, 120 at N = 6, 7; at N = 8 two tiles
  // of 88 rows measured 2 % slower than two of 96)
  static constexpr int MT_NARROW = MODEL == 0 ? (N == 6 ? 88 : N == 7 ? 120 : MT_WIDE)
                                              : (N == 6 ? 44 : N == 7 ? 60 : MT_WIDE);
  // (acoustic N = 5: one tile of exactly Np = 56 rows, 13 % faster than
  // 64-row tiles; three short tiles at N = 7, 8 re-read X and spill)
  static constexpr int MT_SMALL = MODEL == 0 && N == 5 ? 56 : MT_NARROW;
  // (HALF: 16 lanes per row group, so an even number of row groups: MT_WIDE)
  // THIRD (narrow): three row tiles of about Np / 3 rows (multiple of TM),
  // registers and shared memory sized for two resident CTAs per SM
  static constexpr int MT_THIRD = ((Np + 2) / 3 + TM - 1) / TM * TM;
  static constexpr int MT = THIRD ? MT_THIRD : SMALL ? MT_SMALL : (NARROW && !HALF) ? MT_NARROW : MT_WIDE;
  static constexpr int MINB = SMALL || HALF || THIRD ? 2 : 1;  // resident CTAs the registers are sized for
  static constexpr int MP2 = (Np + MT - 1) / MT * MT;     // padded rows of the split operator blob
  static constexpr int KC = 16;                           // K chunk (volume indices or face nodes)
  // cp.async stages: 4 for the acoustic tiles that have the SM to themselves,
  // 3 where two CTAs share it (SMALL, HALF) and for the elastic tiles (a
  // fourth stage cost elastic N = 3 a third of its resident CTAs)
  static constexpr int NS = (MODEL == 0 && !SMALL && !HALF && !THIRD) ? 4 : 3;
  static constexpr int NT = (MT / TM) * (NEG / TE);       // threads per CTA
  static constexpr int MTILES_R = (Np + MT - 1) / MT;     // row tiles
  static constexpr int MTILES_L = MTILES_R * NSUB;        // CTAs per column tile (launch grid: x column tiles)
  static constexpr int NVC = (Np + KC - 1) / KC;          // volume chunks
  static constexpr int NLC = (NFN + KC - 1) / KC;         // lift chunks
  // X rows of one chunk: NV KC (volume); lift: 2 KC streams + 12 normal
  // rows (acoustic), Nf KC (elastic)
  static constexpr int LB = XRows<MODEL, N>::NXS * KC + 12;
  static constexpr int nA = 3 * KC * MT;                  // operator rows of one stage
  static constexpr int nB = (NV * KC > LB ? NV * KC : LB) * NEG;  // X rows of one stage
  static constexpr int NEP = NEG + 1;                     // row stride of the staged RHS field
  static constexpr int nOut = MT * NEP;
  static constexpr int nStage = nA + nB;
  static constexpr size_t smem = size_t(NS * nStage > nOut ? NS * nStage : nOut) * 4;
  static constexpr size_t x_floats_per_tile = size_t(KX) * NE;
  static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
  static_assert(MT % 4 == 0 && NEG % 4 == 0 && TM % 4 == 0, "16-byte copies and loads");
  static_assert(!HALF || NARROW, "half column tiles with the narrow thread tile");
  static_assert(NS >= 2, "the copy of a chunk is issued after the barrier that retires its stage");
};

template <int MODEL, int N, bool NARROW = false, bool SMALL = false, bool HALF = false, bool PK = false,
          bool THIRD = false>
__device__ __forceinline__ void gemm_b_body(const StepArgs& a, const int mtile_l, const int ntile) {
  using SS = GemmB<MODEL, N, NARROW, SMALL, HALF, PK, THIRD>;
  // NE: elements of this CTA; XNE: row stride of X (elements per column tile)
  constexpr int Np = SS::Np, NFN = SS::NFN, Nf = SS::Nf, NV = SS::NV, NE = SS::NEG, TM = SS::TM, TE = SS::TE;
  constexpr int XNE = SS::NE;
  const int mtile = mtile_l % SS::MTILES_R, half = mtile_l / SS::MTILES_R;
  const int kbase = ntile * XNE + half * NE;  // first element of the CTA
  constexpr int NXS = XRows<MODEL, N>::NXS, KXM = XRows<MODEL, N>::KXM;
  constexpr int MT = SS::MT, MP2 = SplitShape<MODEL, N>::OPP, KC = SS::KC, NT = SS::NT, NS = SS::NS;
  constexpr int NVC = SS::NVC, NLC = SS::NLC, NCH = NVC + NLC;

  extern __shared__ __align__(16) float smem[];
  auto sA = [&](int s) { return smem + s * SS::nStage; };
  auto sB = [&](int s) { return smem + s * SS::nStage + SS::nA; };

  const int tid = threadIdx.x;
  const int row0 = mtile * MT;
  const float* X = a.xg + size_t(ntile) * SplitShape<MODEL, N>::x_floats_per_tile + half * NE;
  const float* OP = a.ops2;  // [3 Np + NFN][MP2]

  // chunk c -> stage c % NS: operator rows [KC][MT] (3 of them for a volume
  // chunk), X rows [vector][KC][NE]; rows past Np / 4 Nfp are neither copied
  // nor read
  auto issue = [&](int c) {
    if (c < NCH) {
      float* A = sA(c % NS);
      float* B = sB(c % NS);
      if (c < NVC) {
        const int j0 = c * KC;
        const int nj = Np - j0 < KC ? Np - j0 : KC;
        for (int i = tid; i < 3 * nj * (MT / 4); i += NT) {
          const int q4 = i % (MT / 4), rr = i / (MT / 4);
          const int d = rr / nj, jj = rr - d * nj;
          cp_async16(A + (d * KC + jj) * MT + 4 * q4, OP + size_t(d * Np + j0 + jj) * MP2 + row0 + 4 * q4);
        }
        for (int i = tid; i < NV * nj * (NE / 4); i += NT) {
          const int q4 = i % (NE / 4), rr = i / (NE / 4);
          const int f = rr / nj, jj = rr - f * nj;
          cp_async16(B + (f * KC + jj) * NE + 4 * q4, X + size_t(f * Np + j0 + jj) * XNE + 4 * q4);
        }
      } else {
        const int c0 = (c - NVC) * KC;
        const int nc = NFN - c0 < KC ? NFN - c0 : KC;
        for (int i = tid; i < nc * (MT / 4); i += NT) {
          const int q4 = i % (MT / 4), cc = i / (MT / 4);
          cp_async16(A + cc * MT + 4 * q4, OP + size_t(3 * Np + c0 + cc) * MP2 + row0 + 4 * q4);
        }
        for (int i = tid; i < NXS * nc * (NE / 4); i += NT) {
          const int q4 = i % (NE / 4), rr = i / (NE / 4);
          const int f = rr / nc, cc = rr - f * nc;
          cp_async16(B + (f * KC + cc) * NE + 4 * q4, X + size_t(NV * Np + f * NFN + c0 + cc) * XNE + 4 * q4);
        }
        // the face normals, after the streams
        for (int i = tid; i < 12 * (NE / 4); i += NT) {
          const int q4 = i % (NE / 4), r = i / (NE / 4);
          cp_async16(B + (NXS * KC + r) * NE + 4 * q4, X + size_t(KXM + r) * XNE + 4 * q4);
        }
      }
    }
    cp_async_commit();  // an empty group past the last chunk keeps the wait count uniform
  };

  // thread tile: rows il..il+TM-1 of the CTA's slice, elements e0..e0+TE-1;
  // the lanes of a warp span the elements (NE / TE of them: two row groups
  // per warp at TE = 4, one otherwise)
  constexpr int CT = NE / TE;
  const int ct = tid % CT, rt = tid / CT;
  const int il = TM * rt, e0 = TE * ct;
  ProdTile<MODEL, N, TM, TE, PK, MT, NE> pt;
  pt.zero();

#pragma unroll
  for (int s = 0; s < NS - 1; ++s) issue(s);
  // row groups wholly past Np (padding of the last row tile) skip the
  // products; they still copy and meet every barrier
  const bool rows_live = row0 + il < Np;
  for (int c = 0; c < NCH; ++c) {
    cp_async_wait_n<NS - 2>();  // chunk c has landed (chunks up to c + NS - 2 may be in flight)
    // ... for every thread; and every thread is done with chunk c - 1, whose
    // stage the next copy refills: one barrier per chunk
    __syncthreads();
    issue(c + NS - 1);
    // the tile's AB3 inputs into L2 a few chunks before the epilogue
    if (tid == 0 && c == ab3_prefetch_chunk(NCH) && mtile == 0 && a.mode == 0)
      prefetch_tile_l2<Nf, Np, NE>(a, kbase);
    const float* A = sA(c % NS) + il;
    const float* B = sB(c % NS) + e0;
    if (c < NVC) {
      const int nj = !rows_live ? 0 : Np - c * KC < KC ? Np - c * KC : KC;
      pt.volume(A, B, nj);
      if (c == NVC - 1) pt.boundary(a, kbase + e0);
    } else {
      const int c0 = (c - NVC) * KC;
      const int nc = !rows_live ? 0 : NFN - c0 < KC ? NFN - c0 : KC;
      pt.lift(A, B, c0, nc);
    }
  }
  cp_async_wait_n<0>();
  __syncthreads();

  // -------- epilogue: one field at a time through shared memory [MT][NEP]
  tile_epilogue<MODEL, N, MT, NE, SS::NEP, NT>(a, pt, smem, tid, il, e0, row0, kbase, [] { __syncthreads(); });
}


// Design V of the FP32 GEMM (V = 2: design B, V = 3: design B with half the
// elements per thread, V = 4: V = 3 with short row tiles and two CTAs per SM,
// V = 5: V = 3 with half a column tile per CTA and two CTAs per SM,
// otherwise design A).
template <int MODEL, int N, int V>
struct GemmOf {
  using T = GemmA<MODEL, N>;
  __device__ static void body(const StepArgs& a, int mtile, int ntile) { gemm_a_body<MODEL, N>(a, mtile, ntile); }
};
template <int MODEL, int N>
struct GemmOf<MODEL, N, 2> {
  using T = GemmB<MODEL, N>;
  __device__ static void body(const StepArgs& a, int mtile, int ntile) { gemm_b_body<MODEL, N>(a, mtile, ntile); }
};
template <int MODEL, int N>
struct GemmOf<MODEL, N, 3> {
  using T = GemmB<MODEL, N, true>;
  __device__ static void body(const StepArgs& a, int mtile, int ntile) { gemm_b_body<MODEL, N, true>(a, mtile, ntile); }
};
template <int MODEL, int N>
struct GemmOf<MODEL, N, 4> {
  using T = GemmB<MODEL, N, true, true>;
  __device__ static void body(const StepArgs& a, int mtile, int ntile) {
    gemm_b_body<MODEL, N, true, true>(a, mtile, ntile);
  }
};
template <int MODEL, int N>
struct GemmOf<MODEL, N, 5> {
  using T = GemmB<MODEL, N, true, false, true>;
  __device__ static void body(const StepArgs& a, int mtile, int ntile) {
    gemm_b_body<MODEL, N, true, false, true>(a, mtile, ntile);
  }
};

// V = 6..9: designs 2..5 with the packed two-lane FMA (fma.rn.f32x2) in
// the operator products -- half the FMA instructions, the same results.
template <int MODEL, int N>
struct GemmOf<MODEL, N, 6> {
  using T = GemmB<MODEL, N, false, false, false, true>;
  __device__ static void body(const StepArgs& a, int mtile, int ntile) {
    gemm_b_body<MODEL, N, false, false, false, true>(a, mtile, ntile);
  }
};
template <int MODEL, int N>
struct GemmOf<MODEL, N, 7> {
  using T = GemmB<MODEL, N, true, false, false, true>;
  __device__ static void body(const StepArgs& a, int mtile, int ntile) {
    gemm_b_body<MODEL, N, true, false, false, true>(a, mtile, ntile);
  }
};
template <int MODEL, int N>
struct GemmOf<MODEL, N, 8> {
  using T = GemmB<MODEL, N, true, true, false, true>;
  __device__ static void body(const StepArgs& a, int mtile, int ntile) {
    gemm_b_body<MODEL, N, true, true, false, true>(a, mtile, ntile);
  }
};
template <int MODEL, int N>
struct GemmOf<MODEL, N, 9> {
  using T = GemmB<MODEL, N, true, false, true, true>;
  __device__ static void body(const StepArgs& a, int mtile, int ntile) {
    gemm_b_body<MODEL, N, true, false, true, true>(a, mtile, ntile);
  }
};

// V = 10: design 3 with the packed FMA and three row tiles, two CTAs per SM (THIRD).
template <int MODEL, int N>
struct GemmOf<MODEL, N, 10> {
  using T = GemmB<MODEL, N, true, false, false, true, true>;
  __device__ static void body(const StepArgs& a, int mtile, int ntile) {
    gemm_b_body<MODEL, N, true, false, false, true, true>(a, mtile, ntile);
  }
};

// ---------------------------------------------------------------- design W
// Warp-specialised, persistent form of design B (narrow thread tile, packed
// FMA).  Warp 0 is the producer: per K chunk one 1-D bulk copy for each
// operator row slice (MT floats of a row of the blob) and one for each X row
// block (a vector's KC rows of the column tile, contiguous in X), all
// completing on the stage's full barrier.  Warps 1..NC are the consumers, warp
// w + 1 owning rows TM w .. TM w + TM - 1 of the CTA's MT rows for all NE
// elements of the column tile (TE per lane); each waits on the stage's full
// barrier, runs the chunk and arrives on its empty barrier.  There is no
// CTA-wide barrier in the K loop, and the CTA walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... so that the producer fills the ring with the
// next tile's chunks while the consumers run the epilogue (which syncs the
// consumer warps only, on named barriers).
//
// Failure handling: every wait is bounded.  A consumer warp whose wait expires
// stops; all consumer warps then leave the tile loop together at the vote
// before the next epilogue (so the named barriers always see every consumer),
// the producer stops at its next expired empty wait, and thread 0 waits for
// the copies still in flight before the CTA leaves.
template <int MODEL, int N, int NC, int NSTG, int MINB_, int TM_ = (MODEL == 0 ? 8 : 4)>
struct GemmW {
  using S = Sz<N>;
  static constexpr int Np = S::Np, NFN = S::NFN;
  static constexpr int Nf = MODEL == 0 ? 4 : 9;
  static constexpr int NV = XRows<MODEL, N>::NV, NXS = XRows<MODEL, N>::NXS, KXM = XRows<MODEL, N>::KXM;
  static constexpr int NE = MODEL == 0 ? 64 : 32;   // elements per column tile of X
  static constexpr int TM = TM_;                    // rows per consumer warp (multiple of 4)
  static constexpr int TE = NE / 32;                // elements per lane
  static constexpr int MT = NC * TM;                // output rows per CTA tile
  static constexpr int KC = 16;
  static constexpr int NS = NSTG;
  static constexpr int NT = 32 * (NC + 1);
  static constexpr int MINB = MINB_;
  static constexpr int MTILES_R = (Np + MT - 1) / MT;
  static constexpr int MTILES_L = MTILES_R;
  static constexpr int NVC = (Np + KC - 1) / KC;
  static constexpr int NLC = (NFN + KC - 1) / KC;
  static constexpr int nA = 3 * KC * MT;             // operator rows of one stage
  static constexpr int LB = NXS * KC + 12;           // X rows of a LIFT chunk (streams, normals)
  static constexpr int nB = (NV * KC > LB ? NV * KC : LB) * NE;
  static constexpr int nStage = nA + nB;
  static constexpr int NEP = NE + 1;                 // row stride of the staged RHS field
  static constexpr int nOut = MT * NEP;
  static constexpr int oOut = NS * nStage;
  static constexpr int oBar = (oOut + nOut + 3) / 4 * 4;
  static constexpr size_t smem = size_t(oBar) * 4 + size_t(2 * NS) * 8;
  static constexpr size_t x_floats_per_tile = size_t(XRows<MODEL, N>::KX) * NE;
  static_assert(MT % 4 == 0 && nA % 4 == 0 && nB % 4 == 0, "16-byte aligned copies and stages");
  static_assert(NV <= 32 && NXS < 32, "one X copy per producer lane");
  static_assert(NT <= 1024 && NS >= 2, "launch shape");
};

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// AND of p over the nthreads threads that meet at named barrier id
__device__ __forceinline__ bool named_bar_and(int id, int nthreads, bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.and.pred po, %2, %3, pi;\n\tselp.u32 %0, 1, 0, "
      "po;\n\t}"
      : "=r"(r)
      : "r"(uint32_t(p)), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

// Tiles of one solve: tile t = (row tile t % MTILES, column tile t / MTILES).
template <int MTILES, int NE>
struct WTilesOne {
  const StepArgs& a;
  __device__ int ntiles() const { return MTILES * ((a.K + NE - 1) / NE); }
  __device__ const StepArgs& tile(int t, int& mtile, int& ntile) {
    mtile = t % MTILES;
    ntile = t / MTILES;
    return a;
  }
  __device__ int* err() const { return a.err; }
  __device__ long long limit() const { return a.wait_limit; }
};
// Tiles of every solve of a batch: global tile -> (solve, local tile) through
// the batch's tile tables, the solve's arguments from its device-side state.
template <int MTILES>
struct WTilesBatch {
  const BatchArgs& b;
  StepArgs a;
  __device__ int ntiles() const { return b.total_tiles; }
  __device__ const StepArgs& tile(int t, int& mtile, int& ntile) {
    const int so = __ldg(b.tile_solve + t);
    const int lt = t - __ldg(b.tile_start + so);
    solve_args(b, b.solves[so], a);
    mtile = lt % MTILES;
    ntile = lt / MTILES;
    return a;
  }
  __device__ int* err() const { return b.err; }
  __device__ long long limit() const { return b.wait_limit; }
};

template <int MODEL, int N, int NC, int NSTG, int MINB, int TM_, class Prov>
__device__ __forceinline__ void gemm_w_body(Prov& prov) {
  using W = GemmW<MODEL, N, NC, NSTG, MINB, TM_>;
  constexpr int Np = W::Np, NFN = W::NFN, NV = W::NV, NXS = W::NXS, KXM = W::KXM;
  constexpr int NE = W::NE, TM = W::TM, TE = W::TE, MT = W::MT, KC = W::KC, NS = W::NS;
  constexpr int NVC = W::NVC, NCH = W::NVC + W::NLC, MTILES = W::MTILES_R;
  constexpr int MP2 = SplitShape<MODEL, N>::OPP;
  constexpr int NCT = 32 * NC;  // consumer threads
  static_assert(MTILES * MT <= MP2, "row tiles inside the operator pitch");

  extern __shared__ __align__(16) float smem[];
  auto sA = [&](int s) { return smem + s * W::nStage; };
  auto sB = [&](int s) { return smem + s * W::nStage + W::nA; };
  float* sOut = smem + W::oOut;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + W::oBar);  // stage s holds chunk g (g % NS = s)
  uint64_t* empty = full + NS;                                   // every consumer warp is done with stage s

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = prov.ntiles();
  int* const err = prov.err();
  const long long limit = prov.limit();
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NC);
    }
    fence_barrier_init();
  }
  __syncthreads();

  bool ok = true;
  int issued = 0;  // producer: chunks whose copies were issued
  if (warp == 0) {
    // -------- producer
    int g = 0;
    for (int t = int(blockIdx.x); t < ntiles && ok; t += int(gridDim.x)) {
      int mtile, ntile;
      const StepArgs& a = prov.tile(t, mtile, ntile);
      const float* X = a.xg + size_t(ntile) * W::x_floats_per_tile;
      const float* OP = a.ops2 + mtile * MT;  // [3 Np + NFN][MP2], this tile's row slice
      for (int c = 0; c < NCH; ++c, ++g) {
        const int s = g % NS;
        bool got = true;
        if (lane == 0 && g >= NS) got = mbar_wait_bounded(&empty[s], uint32_t(((g / NS) - 1) & 1), err, limit);
        if (!__shfl_sync(0xffffffffu, got, 0)) {
          ok = false;
          break;
        }
        float* A = sA(s);
        float* B = sB(s);
        if (c < NVC) {
          const int j0 = c * KC;
          const int nj = Np - j0 < KC ? Np - j0 : KC;
          if (lane == 0) mbar_arrive_expect_tx(&full[s], uint32_t((3 * MT + NV * NE) * nj * 4));
          __syncwarp();
          for (int i = lane; i < 3 * nj; i += 32) {
            const int d = i / nj, jj = i - d * nj;
            tma_bulk_g2s(A + (d * KC + jj) * MT, OP + size_t(d * Np + j0 + jj) * MP2, uint32_t(MT * 4), &full[s]);
          }
          if (lane < NV)
            tma_bulk_g2s(B + lane * KC * NE, X + size_t(lane * Np + j0) * NE, uint32_t(nj * NE * 4), &full[s]);
        } else {
          const int c0 = (c - NVC) * KC;
          const int nc = NFN - c0 < KC ? NFN - c0 : KC;
          if (lane == 0) mbar_arrive_expect_tx(&full[s], uint32_t(((MT + NXS * NE) * nc + 12 * NE) * 4));
          __syncwarp();
          if (lane < nc) tma_bulk_g2s(A + lane * MT, OP + size_t(3 * Np + c0 + lane) * MP2, uint32_t(MT * 4), &full[s]);
          if (lane < NXS)
            tma_bulk_g2s(B + lane * KC * NE, X + size_t(NV * Np + lane * NFN + c0) * NE, uint32_t(nc * NE * 4),
                         &full[s]);
          if (lane == NXS) tma_bulk_g2s(B + NXS * KC * NE, X + size_t(KXM) * NE, uint32_t(12 * NE * 4), &full[s]);
        }
        issued = g + 1;
        // the tile's AB3 inputs into L2 a few chunks before its epilogue
        if (lane == 0 && c == ab3_prefetch_chunk(NCH) && mtile == 0 && a.mode == 0)
          prefetch_tile_l2<W::Nf, Np, NE>(a, ntile * NE);
      }
    }
  } else {
    // -------- consumers
    const int w = warp - 1;
    const int il = TM * w, e0 = TE * lane;
    int g = 0;
    for (int t = int(blockIdx.x); t < ntiles; t += int(gridDim.x)) {
      int mtile, ntile;
      const StepArgs& a = prov.tile(t, mtile, ntile);
      const int row0 = mtile * MT, kbase = ntile * NE;
      const bool rows_live = row0 + il < Np;  // row groups wholly past Np skip the products
      ProdTile<MODEL, N, TM, TE, true, MT, NE> pt;
      pt.zero();
      for (int c = 0; c < NCH; ++c, ++g) {
        const int s = g % NS;
        const bool got = mbar_wait_bounded(&full[s], uint32_t((g / NS) & 1), err, limit);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        if (rows_live) {
          const float* A = sA(s) + il;
          const float* B = sB(s) + e0;
          if (c < NVC) {
            pt.volume(A, B, Np - c * KC < KC ? Np - c * KC : KC);
            if (c == NVC - 1) pt.boundary(a, kbase + e0);
          } else {
            const int c0 = (c - NVC) * KC;
            pt.lift(A, B, c0, NFN - c0 < KC ? NFN - c0 : KC);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
      }
      // every consumer warp takes the same way out (the epilogue's named
      // barriers need all of them)
      if (!named_bar_and(1, NCT, ok)) {
        ok = false;
        break;
      }
      tile_epilogue<MODEL, N, MT, NE, W::NEP, NCT>(a, pt, sOut, tid - 32, il, e0, row0, kbase,
                                                   [] { named_bar_sync(2, NCT); });
    }
  }

  const bool abort = __syncthreads_or(!ok);
  if (abort && tid == 0) {
    // copies still in flight land before the CTA leaves
    for (int g = (issued > NS ? issued - NS : 0); g < issued; ++g)
      mbar_wait_bounded(&full[g % NS], uint32_t((g / NS) & 1), nullptr);
  }
}

// One solve: row tiles fastest, so that the CTAs that share a column tile of
// X run together and read it from L2.  V selects the design (1 = A, 2 = B).
template <int MODEL, int N, int V>
__global__ void __launch_bounds__(GemmOf<MODEL, N, V>::T::NT, GemmOf<MODEL, N, V>::T::MINB)
    dg_split_gemm_kernel(const StepArgs a) {
  using G = typename GemmOf<MODEL, N, V>::T;
  constexpr int MTILES = G::MTILES_L;
  GemmOf<MODEL, N, V>::body(a, int(blockIdx.x) % MTILES, int(blockIdx.x) / MTILES);
}

// Every solve of a batch: global tile -> (solve, local tile) through the
// batch's tile tables, the solve's arguments from its device-side state.
template <int MODEL, int N, int V>
__global__ void __launch_bounds__(GemmOf<MODEL, N, V>::T::NT, GemmOf<MODEL, N, V>::T::MINB)
    dg_split_gemm_batched_kernel(const BatchArgs b) {
  using G = typename GemmOf<MODEL, N, V>::T;
  constexpr int MTILES = G::MTILES_L;
  const int so = __ldg(b.tile_solve + blockIdx.x);
  const int lt = int(blockIdx.x) - __ldg(b.tile_start + so);
  StepArgs a;
  solve_args(b, b.solves[so], a);
  GemmOf<MODEL, N, V>::body(a, lt % MTILES, lt / MTILES);
}

// Design W: one persistent CTA per resident slot walks the tiles of a solve
// (or of every solve of a batch).
template <int MODEL, int N, int NC, int NS, int MINB, int TM>
__global__ void __launch_bounds__(GemmW<MODEL, N, NC, NS, MINB, TM>::NT, MINB)
    dg_split_gemm_w_kernel(const StepArgs a) {
  using W = GemmW<MODEL, N, NC, NS, MINB, TM>;
  WTilesOne<W::MTILES_L, W::NE> prov{a};
  gemm_w_body<MODEL, N, NC, NS, MINB, TM>(prov);
}
template <int MODEL, int N, int NC, int NS, int MINB, int TM>
__global__ void __launch_bounds__(GemmW<MODEL, N, NC, NS, MINB, TM>::NT, MINB)
    dg_split_gemm_w_batched_kernel(const BatchArgs b) {
  using W = GemmW<MODEL, N, NC, NS, MINB, TM>;
  WTilesBatch<W::MTILES_L> prov{b};
  gemm_w_body<MODEL, N, NC, NS, MINB, TM>(prov);
}

}  // namespace dgk
