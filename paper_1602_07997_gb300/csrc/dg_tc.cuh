// Split step, tensor-core back half: operator products on the 5th-generation
// tensor cores (tcgen05) in split-BF16 arithmetic, FP32 accumulation in TMEM.
//
// The front half (the fused kernel with SPLIT = NE) leaves the GEMM inputs of
// every element in X[tile][row][NE] (FP32, row = input index: the volume
// inputs, then the Fscale-weighted penalty terms; NE elements per tile,
// element fastest).  A tile of this kernel is 128 output rows x NE elements;
// persistent CTAs (one per SM) walk the tiles t = blockIdx.x + j gridDim.x
// with warp-specialised roles:
//   - warp 0 (one lane), producer: per tile the element records, then per
//     chunk of 16 input indices (the K of one MMA) the chunk's operator pieces
//     [D_r D_s D_t] or LIFT, pre-split on the host into NSPLIT BF16 pieces in
//     the no-swizzle K-major core-matrix layout, and the chunk's FP32 input
//     rows: 1-D TMA bulk copies into an NS-stage ring (mbarrier tx counts);
//   - warps 2-3, converters: split every FP32 input x into BF16 pieces
//     x = x_0 + x_1 (+ x_2) (round to nearest, each piece the rounding of the
//     remainder) stored in the same core-matrix layout;
//   - warp 1 (one lane), MMA issuer: tcgen05.mma (M = 128, N = NE, K = 16) for
//     every product and every piece pair (a, b) with a + b < NSPLIT into the
//     tile's TMEM accumulator (two accumulators alternate when they fit in the
//     512 TMEM columns, so that a tile's products run while the previous
//     tile's epilogue drains): NSPLIT = 2 gives the three products of bf16x3,
//     NSPLIT = 3 the six products that leave only terms of relative size 2^-24;
//   - warps 4-7, epilogue: each reads its 32 TMEM lanes (its output rows) and
//     does the geometric combination, the point source and the AB3 update
//     (Eq. updateScheme) as in the fused kernel, rows across lanes: global
//     accesses are coalesced; the AB3 inputs of a group of elements are all in
//     flight before the first store.
// Products (TMEM column blocks of NE):
//   acoustic: G_d = D_d p (0..2), R = sum_d D_d w_d + LIFT P_p (3),
//             L_c = LIFT P_v,c (4..6)
//   elastic:  U_cd = D_d v_c (3c + d), Rv_c = sum_d D_d s_cd + LIFT P_v,c
//             (9 + c), S_x = LIFT P_sig,x (12 + x)
// Every wait is bounded; on expiry a role sets the error word and stops, the
// others stop at their next wait, and the CTA waits (bounded) for its copies
// and products in flight, frees TMEM and returns.
#pragma once

#include <cuda_bf16.h>

#include "dg_kernels.cuh"

namespace dgk {

template <int MODEL, int N, int NSPLIT>
struct TcShape {
  using S = Sz<N>;
  static constexpr int Np = S::Np, NFN = S::NFN;
  static constexpr int Nf = MODEL == 0 ? 4 : 9;
  static constexpr int NV = MODEL == 0 ? 4 : 12;  // volume input vectors
  static constexpr int KX = NV * Np + Nf * NFN;   // X rows per element
  static constexpr int NE = MODEL == 0 ? 32 : 16; // elements per tile (MMA N)
  static constexpr int MT = 128;                  // output rows per tile (MMA M)
  static constexpr int MTILES = (Np + MT - 1) / MT;
  static constexpr int NKD = (Np + 15) / 16;      // K chunks of the volume products
  static constexpr int NKL = (NFN + 15) / 16;     // K chunks of the LIFT products
  static constexpr int NCH = NKD + NKL;
  static constexpr int NACC = MODEL == 0 ? 7 : 18;
  static constexpr int TCOLS = NACC * NE;         // TMEM columns of one accumulator
  static constexpr int NBUF = 2 * TCOLS <= 512 ? 2 : 1;
  static constexpr int TNEED = NBUF * TCOLS;
  static constexpr int TALLOC = TNEED <= 32 ? 32 : TNEED <= 64 ? 64 : TNEED <= 128 ? 128 : TNEED <= 256 ? 256 : 512;
  static constexpr int NB = NV > Nf ? NV : Nf;    // input vectors of one chunk, at most
  static constexpr int PIECE = MT * 16 * 2;       // one BF16 operator piece of one chunk
  static constexpr int A_D = 3 * NSPLIT * PIECE;  // volume chunk: D_r, D_s, D_t pieces
  static constexpr int A_L = NSPLIT * PIECE;      // LIFT chunk
  static constexpr int B32 = NB * 16 * NE * 4;    // FP32 input rows of one chunk
  static constexpr int BV = NE * 16 * 2;          // one BF16 piece of one input vector
  static constexpr int B16 = NSPLIT * NB * BV;
  static constexpr int STAGE = A_D + B32 + B16;
  static constexpr int NS = 3;                    // pipeline stages
  static constexpr int RECB = NE * Rec<MODEL>::size * 4;  // element records of one tile
  static constexpr int NT = 256;                  // 8 warps: producer, MMA, 2 converters, 4 epilogue
  static constexpr size_t OPS_PER_MTILE = size_t(NKD) * A_D + size_t(NKL) * A_L;
  static constexpr size_t smem = size_t(NS) * STAGE + 2 * RECB + 256;
  static_assert(TCOLS <= 512, "TMEM columns");
  static_assert(NE % 16 == 0 && NE <= 256, "MMA N for M = 128");
  static_assert(RECB % 16 == 0, "record copies are whole 16-byte pieces");
};

// ---------------------------------------------------------------- tcgen05 helpers
// Shared-memory matrix descriptor, no swizzle, K-major: core matrices of
// 8 rows x 16 bytes stored as 128 contiguous bytes; lbo = byte distance of
// the two core matrices along K, sbo = byte distance of 8-row groups.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((saddr & 0x3FFFFu) >> 4);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;  // descriptor version of sm_100-class tensor cores
  return d;                // base offset 0, relative lbo, no swizzle
}
// Instruction descriptor of kind::f16: FP32 D, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int Nn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(Nn >> 3) << 17) | (uint32_t(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 32 lanes x 32 bits, 4 or 8 consecutive columns per thread
__device__ __forceinline__ void tc_ld4(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(taddr)
               : "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
}
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int t = 0; t < 8; ++t) v[t] = __uint_as_float(r[t]);
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// pieces of x: x_0 = bf16(x), x_1 = bf16(x - x_0), x_2 = bf16(x - x_0 - x_1);
// the remainders are exact in FP32
template <int NSPLIT>
__device__ __forceinline__ void bf16_pieces(float x, uint16_t* out) {
  float r = x;
#pragma unroll
  for (int h = 0; h < NSPLIT; ++h) {
    const __nv_bfloat16 b = __float2bfloat16_rn(r);
    out[h] = __bfloat16_as_ushort(b);
    r -= __bfloat162float(b);
  }
}

template <int MODEL, int N, int NSPLIT>
__global__ void __launch_bounds__(256, 1) dg_tc_gemm_kernel(const StepArgs a) {
  using TS = TcShape<MODEL, N, NSPLIT>;
  constexpr int Np = TS::Np, NFN = TS::NFN, Nf = TS::Nf, NV = TS::NV, KX = TS::KX, NE = TS::NE;
  constexpr int NKD = TS::NKD, NCH = TS::NCH, NS = TS::NS, NB = TS::NB, NBUF = TS::NBUF, MTILES = TS::MTILES;
  constexpr int REC = Rec<MODEL>::size;
  constexpr uint32_t IDESC = tc_idesc_bf16(128, NE);

  extern __shared__ __align__(1024) uint8_t tsm[];
  float* recs = reinterpret_cast<float*>(tsm + NS * TS::STAGE);  // [2][NE][REC]
  uint64_t* full = reinterpret_cast<uint64_t*>(tsm + NS * TS::STAGE + 2 * TS::RECB);
  uint64_t* conv = full + NS;
  uint64_t* empty = conv + NS;
  uint64_t* tfull = empty + NS;   // accumulator b holds a finished tile
  uint64_t* tempty = tfull + 2;   // accumulator b has been read out
  uint64_t* rfull = tempty + 2;   // records of tile buffer r landed
  uint64_t* rempty = rfull + 2;   // records of tile buffer r no longer read
  uint64_t* done = rempty + 2;    // every product of the CTA has completed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = ((a.K + NE - 1) / NE) * MTILES;
  const int nmine = int(blockIdx.x) < ntiles ? (ntiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 64);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
      mbar_init(&rfull[b], 1);
      mbar_init(&rempty[b], 4);
    }
    mbar_init(done, 1);
    fence_barrier_init();
  }
  if (warp == 1) tc_alloc(tslot, TS::TALLOC);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  // Roles go to whole warps: the idle lanes of the producer and MMA warps wait
  // at __syncwarp, not on an mbarrier, so that the working lane is never held
  // up by its own warp's suspended waits.
  bool ok = true;
  int issued = 0, rissued = 0;  // producer: chunks / tile records whose copies were issued
  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      for (int j = 0; j < nmine && ok; ++j) {
        const int t = int(blockIdx.x) + j * int(gridDim.x);
        const int mtile = t % MTILES, ntile = t / MTILES;
        const int rb = j & 1;
        if (j >= 2 && !mbar_wait_bounded(&rempty[rb], uint32_t(((j >> 1) - 1) & 1), a.err)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&rfull[rb], TS::RECB);
        tma_bulk_g2s(recs + rb * NE * REC, a.rec + size_t(ntile) * NE * REC, TS::RECB, &rfull[rb]);
        rissued = j + 1;
        const float* X = a.xg + size_t(ntile) * KX * NE;
        const uint8_t* OPS = reinterpret_cast<const uint8_t*>(a.opstc) + size_t(mtile) * TS::OPS_PER_MTILE;
        for (int c = 0; c < NCH; ++c, ++g) {
          const int s = g % NS;
          if (g >= NS && !mbar_wait_bounded(&empty[s], uint32_t(((g / NS) - 1) & 1), a.err)) {
            ok = false;
            break;
          }
          uint8_t* st = tsm + s * TS::STAGE;
          float* b32 = reinterpret_cast<float*>(st + TS::A_D);
          const bool vol = c < NKD;
          const int nvec = vol ? NV : Nf;
          const uint32_t abytes = vol ? TS::A_D : TS::A_L;
          const uint32_t rbytes = 16u * NE * 4u;
          mbar_arrive_expect_tx(&full[s], abytes + uint32_t(nvec) * rbytes);
          const uint8_t* asrc = OPS + (vol ? size_t(c) * TS::A_D : size_t(NKD) * TS::A_D + size_t(c - NKD) * TS::A_L);
          tma_bulk_g2s(st, asrc, abytes, &full[s]);
          for (int v = 0; v < nvec; ++v) {
            const int row = vol ? v * Np + c * 16 : NV * Np + v * NFN + (c - NKD) * 16;
            tma_bulk_g2s(b32 + v * 16 * NE, X + size_t(row) * NE, rbytes, &full[s]);
          }
          issued = g + 1;
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      int g = 0;
      for (int j = 0; j < nmine && ok; ++j) {
        const int b = j % NBUF;
        if (j >= NBUF) {
          if (!mbar_wait_bounded(&tempty[b], uint32_t(((j / NBUF) - 1) & 1), a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        const uint32_t tacc = tmem + uint32_t(b * TS::TCOLS);
        for (int c = 0; c < NCH; ++c, ++g) {
          const int s = g % NS;
          if (!mbar_wait_bounded(&conv[s], uint32_t((g / NS) & 1), a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_addr(tsm + s * TS::STAGE);
          const uint32_t sb = sa + TS::A_D + TS::B32;
          auto adesc = [&](int op, int h) { return tc_sdesc(sa + (op * NSPLIT + h) * TS::PIECE, 128, 256); };
          auto bdesc = [&](int v, int h) { return tc_sdesc(sb + (h * NB + v) * TS::BV, 128, 256); };
          // acc: column block; op: operator slot; v: input vector; first:
          // this chunk starts the accumulator
          auto prod = [&](int acc, int op, int v, bool first) {
#pragma unroll
            for (int ha = 0; ha < NSPLIT; ++ha)
#pragma unroll
              for (int hb = 0; hb < NSPLIT - ha; ++hb)
                tc_mma(tacc + uint32_t(acc * NE), adesc(op, ha), bdesc(v, hb), IDESC,
                       (first && ha == 0 && hb == 0) ? 0u : 1u);
          };
          if (c < NKD) {
            const bool c0 = c == 0;
            if constexpr (MODEL == 0) {
              for (int d = 0; d < 3; ++d) prod(d, d, 0, c0);
              for (int d = 0; d < 3; ++d) prod(3, d, 1 + d, c0 && d == 0);
            } else {
              for (int cc = 0; cc < 3; ++cc)
                for (int d = 0; d < 3; ++d) prod(3 * cc + d, d, cc, c0);
              for (int cc = 0; cc < 3; ++cc)
                for (int d = 0; d < 3; ++d) prod(9 + cc, d, 3 + 3 * cc + d, c0 && d == 0);
            }
          } else {
            const bool l0 = c == NKD;
            if constexpr (MODEL == 0) {
              prod(3, 0, 0, false);
              for (int cc = 0; cc < 3; ++cc) prod(4 + cc, 0, 1 + cc, l0);
            } else {
              for (int cc = 0; cc < 3; ++cc) prod(9 + cc, 0, cc, false);
              for (int x = 0; x < 6; ++x) prod(12 + x, 0, 3 + x, l0);
            }
          }
          tc_commit(&empty[s]);
        }
        if (ok) tc_commit(&tfull[b]);
      }
      tc_commit(done);  // arrives once every product issued above has completed
      if (!mbar_wait_bounded(done, 0u, a.err)) ok = false;
    }
    __syncwarp();
  } else if (warp < 4) {
    // -------- converters: FP32 input rows -> BF16 pieces, core-matrix layout
    const int ct = tid - 64;
    int g = 0;
    for (int j = 0; j < nmine && ok; ++j) {
      for (int c = 0; c < NCH; ++c, ++g) {
        const int s = g % NS;
        if (!mbar_wait_bounded(&full[s], uint32_t((g / NS) & 1), a.err)) {
          ok = false;
          break;
        }
        uint8_t* st = tsm + s * TS::STAGE;
        const float* b32 = reinterpret_cast<const float*>(st + TS::A_D);
        uint8_t* b16 = st + TS::A_D + TS::B32;
        const bool vol = c < NKD;
        const int nvec = vol ? NV : Nf;
        const int k0 = vol ? c * 16 : (c - NKD) * 16;
        const int klim = vol ? Np : NFN;
        for (int u = ct; u < nvec * 2 * NE; u += 64) {
          const int e = u % NE, kh = (u / NE) & 1, v = u / (2 * NE);
          uint16_t pc[NSPLIT][8];
#pragma unroll
          for (int tt = 0; tt < 8; ++tt) {
            const int kk = kh * 8 + tt;
            const float x = (k0 + kk < klim) ? b32[(v * 16 + kk) * NE + e] : 0.f;
            uint16_t hp[NSPLIT];
            bf16_pieces<NSPLIT>(x, hp);
#pragma unroll
            for (int h = 0; h < NSPLIT; ++h) pc[h][tt] = hp[h];
          }
#pragma unroll
          for (int h = 0; h < NSPLIT; ++h) {
            uint4 w;
            w.x = uint32_t(pc[h][0]) | (uint32_t(pc[h][1]) << 16);
            w.y = uint32_t(pc[h][2]) | (uint32_t(pc[h][3]) << 16);
            w.z = uint32_t(pc[h][4]) | (uint32_t(pc[h][5]) << 16);
            w.w = uint32_t(pc[h][6]) | (uint32_t(pc[h][7]) << 16);
            *reinterpret_cast<uint4*>(b16 + (h * NB + v) * TS::BV + (e >> 3) * 256 + kh * 128 + (e & 7) * 16) = w;
          }
        }
        fence_proxy_async_smem();
        mbar_arrive(&conv[s]);
      }
    }
  } else {
    // -------- epilogue: warp 4 + q reads TMEM lanes 32 q .. 32 q + 31
    const int quarter = warp - 4;
    constexpr int EC = MODEL == 0 ? 8 : 4;  // elements per group: TMEM loads and AB3 inputs in flight together
    for (int j = 0; j < nmine; ++j) {
      const int t = int(blockIdx.x) + j * int(gridDim.x);
      const int mtile = t % MTILES, ntile = t / MTILES;
      const int b = j % NBUF, rb = j & 1;
      bool got = mbar_wait_bounded(&tfull[b], uint32_t((j / NBUF) & 1), a.err);
      got = got && mbar_wait_bounded(&rfull[rb], uint32_t((j >> 1) & 1), a.err);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const float* srec = recs + rb * NE * REC;
      const int i = mtile * 128 + quarter * 32 + lane;  // output row of this thread
      const bool row_ok = i < Np;
      const uint32_t trow = tmem + uint32_t(b * TS::TCOLS) + (uint32_t(quarter * 32) << 16);
      for (int e0 = 0; e0 < NE; e0 += EC) {
        float v[TS::NACC][EC];
#pragma unroll
        for (int p = 0; p < TS::NACC; ++p) {
          if constexpr (EC == 8)
            tc_ld8(trow + uint32_t(p * NE + e0), v[p]);
          else
            tc_ld4(trow + uint32_t(p * NE + e0), v[p]);
        }
        // AB3 inputs of the whole group before any store (rows across lanes)
        float qa[EC][Nf], r1a[EC][Nf], r2a[EC][Nf];
        if (a.mode == 0) {
#pragma unroll
          for (int tt = 0; tt < EC; ++tt) {
            const int k = ntile * NE + e0 + tt;
            const bool on = row_ok && k < a.K;
            const size_t base = size_t(on ? k : 0) * Nf * Np + (on ? i : 0);
#pragma unroll
            for (int f = 0; f < Nf; ++f) {
              const size_t idx = base + size_t(f) * Np;
              qa[tt][f] = on ? __ldg(a.q + idx) : 0.f;
              r1a[tt][f] = on ? __ldg(a.r1 + idx) : 0.f;
              r2a[tt][f] = on ? a.r2[idx] : 0.f;
            }
          }
        }
        tc_wait_ld();
#pragma unroll
        for (int tt = 0; tt < EC; ++tt) {
          const int el = e0 + tt;
          const int k = ntile * NE + el;
          if (k >= a.K || !row_ok) continue;
          const float* gk = srec + el * REC;
          float gm[9];
#pragma unroll
          for (int x = 0; x < 9; ++x) gm[x] = gk[x];
          float r[Nf];
          if constexpr (MODEL == 0) {
            const float rinv = gk[10];
            r[0] = v[3][tt];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
              r[1 + cc] =
                  v[4 + cc][tt] - rinv * (gm[3 * cc] * v[0][tt] + gm[3 * cc + 1] * v[1][tt] + gm[3 * cc + 2] * v[2][tt]);
          } else {
            const float lam = gk[9], mu = gk[10];
            float gv[3][3];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
#pragma unroll
              for (int x = 0; x < 3; ++x)
                gv[cc][x] =
                    gm[3 * x] * v[3 * cc][tt] + gm[3 * x + 1] * v[3 * cc + 1][tt] + gm[3 * x + 2] * v[3 * cc + 2][tt];
            const float div = gv[0][0] + gv[1][1] + gv[2][2];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) r[cc] = v[9 + cc][tt];
            r[3] = lam * div + 2.f * mu * gv[0][0] + v[12][tt];
            r[4] = lam * div + 2.f * mu * gv[1][1] + v[13][tt];
            r[5] = lam * div + 2.f * mu * gv[2][2] + v[14][tt];
            r[6] = mu * (gv[0][1] + gv[1][0]) + v[15][tt];
            r[7] = mu * (gv[0][2] + gv[2][0]) + v[16][tt];
            r[8] = mu * (gv[1][2] + gv[2][1]) + v[17][tt];
          }
          if (k == a.src_elem && a.srcvec) {
#pragma unroll
            for (int f = 0; f < Nf; ++f) r[f] = fmaf(a.src_amp, __ldg(a.srcvec + f * Np + i), r[f]);
          }
          const size_t base = size_t(k) * Nf * Np + i;
#pragma unroll
          for (int f = 0; f < Nf; ++f) {
            const size_t idx = base + size_t(f) * Np;
            if (a.mode == 0) {
              const float accv = a.a1 * r[f] + a.a2 * r1a[tt][f] + a.a3 * r2a[tt][f];
              a.qn[idx] = fmaf(a.dt, accv, qa[tt][f]);
              a.r2[idx] = r[f];
            } else {
              a.rout[idx] = r[f];
            }
          }
        }
      }
      // accumulator b and record buffer rb are free for tile j + NBUF / j + 2
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&tempty[b]);
        mbar_arrive(&rempty[rb]);
      }
    }
  }

  const bool abort = __syncthreads_or(!ok);
  if (abort && tid == 0) {
    // copies still in flight land before the CTA leaves
    for (int g = (issued > NS ? issued - NS : 0); g < issued; ++g)
      mbar_wait_bounded(&full[g % NS], uint32_t((g / NS) & 1), nullptr);
    for (int j = (rissued > 2 ? rissued - 2 : 0); j < rissued; ++j)
      mbar_wait_bounded(&rfull[j & 1], uint32_t((j >> 1) & 1), nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tc_dealloc(tmem, TS::TALLOC);
  }
}

}  // namespace dgk
