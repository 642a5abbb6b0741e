// Split step, tensor-core back half: operator products on the 5th-generation
// tensor cores (tcgen05) in split-BF16 arithmetic, FP32 accumulation in TMEM.
//
// The front half (the fused kernel with SPLIT = NE, XP = NSPLIT) leaves the
// GEMM inputs of every element already split into NSPLIT BF16 pieces in the
// tcgen05 operand layout (TcX: one contiguous block per column tile of NE
// elements and chunk of 16 input indices).  A tile of this kernel is 128
// output rows x NE elements; persistent CTAs (one per SM) walk the tiles
// t = blockIdx.x + j gridDim.x with warp-specialised roles:
//   - warp 0 (one lane), producer: per tile the element records (and an L2
//     prefetch of the tile's AB3 inputs), then per chunk the operator pieces
//     [D_r D_s D_t] or LIFT (pre-split on the host, same core-matrix layout)
//     and the chunk's input pieces: two 1-D TMA bulk copies into an NS-stage
//     ring (mbarrier transaction counts);
//   - warp 1 (one lane), MMA issuer: tcgen05.mma (M = 128, N = NE, K = 16) for
//     every product and every piece pair (a, b) with a + b < NSPLIT into the
//     tile's TMEM accumulator (two accumulators alternate when they fit in the
//     512 TMEM columns, so that a tile's products run while the previous
//     tile's epilogue drains): NSPLIT = 2 gives the three products of bf16x3,
//     NSPLIT = 3 the six products that leave only terms of relative size 2^-24;
//   - warps 2-9, epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31 (its
//     output rows; two warps per lane quarter, each half of the tile's
//     element columns, so that twice as many AB3 loads are in flight) and
//     does the geometric combination, the point source and
//     the AB3 update (Eq. updateScheme) as in the fused kernel, rows across
//     lanes: global accesses are coalesced; the AB3 inputs of a group of
//     elements are all in flight before the first store.
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

#include <type_traits>

#include "dg_kernels.cuh"

namespace dgk {

template <int MODEL, int N, int NSPLIT>
struct TcShape {
  using TX = TcX<MODEL, N, NSPLIT>;
  static constexpr int Np = TX::Np, NFN = TX::NFN, Nf = TX::Nf, NV = TX::NV, NE = TX::NE;
  static constexpr int MT = 128;                  // output rows per tile (MMA M)
  static constexpr int MTILES = (Np + MT - 1) / MT;
  static constexpr int NKD = TX::NKD, NKL = TX::NKL, NCH = NKD + NKL;
  static constexpr int NACC = MODEL == 0 ? 7 : 18;
  static constexpr int TCOLS = NACC * NE;         // TMEM columns of one accumulator
  static constexpr int NBUF = 2 * TCOLS <= 512 ? 2 : 1;
  static constexpr int TNEED = NBUF * TCOLS;
  static constexpr int TALLOC = TNEED <= 32 ? 32 : TNEED <= 64 ? 64 : TNEED <= 128 ? 128 : TNEED <= 256 ? 256 : 512;
  static constexpr int PIECE = MT * 16 * 2;       // one BF16 operator piece of one chunk
  static constexpr int A_D = 3 * NSPLIT * PIECE;  // volume chunk: D_r, D_s, D_t pieces
  static constexpr int A_L = NSPLIT * PIECE;      // LIFT chunk
  static constexpr int B16 = TX::CD > TX::CL ? TX::CD : TX::CL;
  static constexpr int STAGE = A_D + B16;
  static constexpr int RECB = NE * Rec<MODEL>::size * 4;  // element records of one tile
  static constexpr int NEPI = 8;                  // epilogue warps: two per TMEM lane quarter
  static constexpr int NT = 64 + 32 * NEPI;       // producer, MMA, epilogue warps
  static constexpr size_t OPS_PER_MTILE = size_t(NKD) * A_D + size_t(NKL) * A_L;
  static constexpr size_t FIXED = 2 * RECB + 256;
  static constexpr int NSF = int((225 * 1024 - FIXED) / STAGE);
  static constexpr int NS = NSF > 6 ? 6 : NSF;    // pipeline stages
  static constexpr size_t smem = size_t(NS) * STAGE + FIXED;
  static_assert(NS >= 2, "pipeline stages");
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
// 32 lanes x 32 bits, 2, 4 or 8 consecutive columns per thread
__device__ __forceinline__ void tc_ld4(uint32_t taddr, float* v) {
  uint32_t r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(taddr)
               : "memory");
  v[0] = __uint_as_float(r0); v[1] = __uint_as_float(r1); v[2] = __uint_as_float(r2); v[3] = __uint_as_float(r3);
}
__device__ __forceinline__ void tc_ld2(uint32_t taddr, float* v) {
  uint32_t r0, r1;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(taddr) : "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
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
// Compile-time loop: f(std::integral_constant<int, i>) for i = I .. END - 1.
template <int I, int END>
struct StaticFor {
  template <class F>
  __device__ __forceinline__ static void run(F&& f) {
    if constexpr (I < END) {
      f(std::integral_constant<int, I>{});
      StaticFor<I + 1, END>::run(f);
    }
  }
};

// The MMAs of one product: every piece pair (ha, hb) with ha + hb < NSPLIT,
// operator slot OP against input vector V of the stage (NVS vectors per piece;
// compile-time, so the
// descriptor offsets are immediates added to the stage's base descriptors
// a0 / b0; the 14-bit address field cannot carry below 256 KB); first = 1
// if this product starts its accumulator.
template <int NSPLIT, int NVS, int PIECE, int BV, int OP, int V>
__device__ __forceinline__ void tc_prod(uint32_t tcol, uint64_t a0, uint64_t b0, uint32_t idesc, uint32_t first) {
#pragma unroll
  for (int ha = 0; ha < NSPLIT; ++ha)
#pragma unroll
    for (int hb = 0; hb < NSPLIT - ha; ++hb)
      tc_mma(tcol, a0 + uint64_t(((OP * NSPLIT + ha) * PIECE) >> 4), b0 + uint64_t(((hb * NVS + V) * BV) >> 4), idesc,
             (ha == 0 && hb == 0) ? (first ^ 1u) : 1u);
}

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int MODEL, int N, int NSPLIT>
__global__ void __launch_bounds__(TcShape<MODEL, N, NSPLIT>::NT, 1) dg_tc_gemm_kernel(const StepArgs a) {
  using TS = TcShape<MODEL, N, NSPLIT>;
  using TX = typename TS::TX;
  constexpr int Np = TS::Np, Nf = TS::Nf, NV = TS::NV, NE = TS::NE;
  constexpr int NKD = TS::NKD, NCH = TS::NCH, NS = TS::NS, NBUF = TS::NBUF, MTILES = TS::MTILES;
  constexpr int REC = Rec<MODEL>::size;
  constexpr uint32_t IDESC = tc_idesc_bf16(128, NE);

  extern __shared__ __align__(1024) uint8_t tsm[];
  float* recs = reinterpret_cast<float*>(tsm + NS * TS::STAGE);  // [2][NE][REC]
  uint64_t* full = reinterpret_cast<uint64_t*>(tsm + NS * TS::STAGE + 2 * TS::RECB);
  uint64_t* empty = full + NS;
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
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], TS::NEPI);
      mbar_init(&rfull[b], 1);
      mbar_init(&rempty[b], TS::NEPI);
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
      // -------- producer
      int g = 0;
      for (int j = 0; j < nmine && ok; ++j) {
        const int t = int(blockIdx.x) + j * int(gridDim.x);
        const int mtile = t % MTILES, ntile = t / MTILES;
        const int rb = j & 1;
        if (j >= 2 && !mbar_wait_bounded(&rempty[rb], uint32_t(((j >> 1) - 1) & 1), a.err, a.wait_limit)) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&rfull[rb], TS::RECB);
        tma_bulk_g2s(recs + rb * NE * REC, a.rec + size_t(ntile) * NE * REC, TS::RECB, &rfull[rb]);
        rissued = j + 1;
        const uint8_t* OPS = reinterpret_cast<const uint8_t*>(a.opstc) + size_t(mtile) * TS::OPS_PER_MTILE;
        const uint8_t* XT = reinterpret_cast<const uint8_t*>(a.xg) + size_t(ntile) * TX::TILE;
        for (int c = 0; c < NCH; ++c, ++g) {
          const int s = g % NS;
          if (g >= NS && !mbar_wait_bounded(&empty[s], uint32_t(((g / NS) - 1) & 1), a.err, a.wait_limit)) {
            ok = false;
            break;
          }
          uint8_t* st = tsm + s * TS::STAGE;
          const bool vol = c < NKD;
          const uint32_t abytes = vol ? TS::A_D : TS::A_L;
          const uint32_t xbytes = vol ? TX::CD : TX::CL;
          mbar_arrive_expect_tx(&full[s], abytes + xbytes);
          tma_bulk_g2s(st, OPS + (vol ? size_t(c) * TS::A_D : size_t(NKD) * TS::A_D + size_t(c - NKD) * TS::A_L),
                       abytes, &full[s]);
          tma_bulk_g2s(st + TS::A_D, XT + TX::chunk_off(c), xbytes, &full[s]);
          issued = g + 1;
          if (a.mode == 0 && mtile == 0 && c == ab3_prefetch_chunk(NCH)) {
            // the epilogue's AB3 inputs of this tile into L2, a few chunks
            // before the epilogue reads them (q, r^{m-1}, r^{m-2} are padded
            // past K: whole tiles stay in bounds)
            const size_t e0 = size_t(ntile) * NE * Nf * Np;
            constexpr uint32_t bytes = uint32_t(NE * Nf * Np * 4);
            prefetch_l2(a.q + e0, bytes);
            prefetch_l2(a.r1 + e0, bytes);
            prefetch_l2(a.r2 + e0, bytes);
          }
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
          if (!mbar_wait_bounded(&tempty[b], uint32_t(((j / NBUF) - 1) & 1), a.err, a.wait_limit)) {
            ok = false;
            break;
          }
          tc_fence_after();
        }
        const uint32_t tacc = tmem + uint32_t(b * TS::TCOLS);
        for (int c = 0; c < NCH; ++c, ++g) {
          const int s = g % NS;
          if (!mbar_wait_bounded(&full[s], uint32_t((g / NS) & 1), a.err, a.wait_limit)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_addr(tsm + s * TS::STAGE);
          const uint64_t a0 = tc_sdesc(sa, 128, 256);           // operator pieces of the stage
          const uint64_t b0 = tc_sdesc(sa + TS::A_D, 128, 256);  // BF16 input pieces of the stage
          constexpr int PC = TS::PIECE, BV = TX::BV;
          if (c < NKD) {
            const uint32_t c0 = c == 0 ? 1u : 0u;
            if constexpr (MODEL == 0) {
              // G_d = D_d p; R = sum_d D_d w_d
              StaticFor<0, 3>::run([&](auto ic) {
                constexpr int d = decltype(ic)::value;
                tc_prod<NSPLIT, NV, PC, BV, d, 0>(tacc + uint32_t(d * NE), a0, b0, IDESC, c0);
              });
              StaticFor<0, 3>::run([&](auto ic) {
                constexpr int d = decltype(ic)::value;
                tc_prod<NSPLIT, NV, PC, BV, d, 1 + d>(tacc + uint32_t(3 * NE), a0, b0, IDESC, d == 0 ? c0 : 0u);
              });
            } else {
              // U_cd = D_d v_c; Rv_c = sum_d D_d s_cd
              StaticFor<0, 9>::run([&](auto ic) {
                constexpr int i = decltype(ic)::value, cc = i / 3, d = i % 3;
                tc_prod<NSPLIT, NV, PC, BV, d, cc>(tacc + uint32_t(i * NE), a0, b0, IDESC, c0);
              });
              StaticFor<0, 9>::run([&](auto ic) {
                constexpr int i = decltype(ic)::value, cc = i / 3, d = i % 3;
                tc_prod<NSPLIT, NV, PC, BV, d, 3 + i>(tacc + uint32_t((9 + cc) * NE), a0, b0, IDESC,
                                                      d == 0 ? c0 : 0u);
              });
            }
          } else {
            const uint32_t l0 = c == NKD ? 1u : 0u;
            if constexpr (MODEL == 0) {
              // R += LIFT P_p; L_c = LIFT P_v,c
              tc_prod<NSPLIT, Nf, PC, BV, 0, 0>(tacc + uint32_t(3 * NE), a0, b0, IDESC, 0u);
              StaticFor<0, 3>::run([&](auto ic) {
                constexpr int cc = decltype(ic)::value;
                tc_prod<NSPLIT, Nf, PC, BV, 0, 1 + cc>(tacc + uint32_t((4 + cc) * NE), a0, b0, IDESC, l0);
              });
            } else {
              // Rv_c += LIFT P_v,c; S_x = LIFT P_sig,x
              StaticFor<0, 3>::run([&](auto ic) {
                constexpr int cc = decltype(ic)::value;
                tc_prod<NSPLIT, Nf, PC, BV, 0, cc>(tacc + uint32_t((9 + cc) * NE), a0, b0, IDESC, 0u);
              });
              StaticFor<0, 6>::run([&](auto ic) {
                constexpr int x = decltype(ic)::value;
                tc_prod<NSPLIT, Nf, PC, BV, 0, 3 + x>(tacc + uint32_t((12 + x) * NE), a0, b0, IDESC, l0);
              });
            }
          }
          tc_commit(&empty[s]);
        }
        if (ok) tc_commit(&tfull[b]);
      }
      tc_commit(done);  // arrives once every product issued above has completed
      // (always the default limit: TMEM is freed only after this wait)
      if (!mbar_wait_bounded(done, 0u, a.err)) ok = false;
    }
    __syncwarp();
  } else {
    // -------- epilogue: warp w reads TMEM lanes 32 (w mod 4) .. 32 (w mod 4) + 31
    const int quarter = warp & 3;
    // the two warps of a lane quarter split the tile's element columns
    constexpr int NEH = NE / (TS::NEPI / 4);
    const int ehalf = (warp - 2) / 4;
    constexpr int EC = MODEL == 0 ? 4 : 2;  // elements per group: TMEM loads and AB3 inputs in flight together
    static_assert(NEH % EC == 0 && TS::NEPI % 4 == 0, "whole element groups per epilogue warp");
    for (int j = 0; j < nmine; ++j) {
      const int t = int(blockIdx.x) + j * int(gridDim.x);
      const int mtile = t % MTILES, ntile = t / MTILES;
      const int b = j % NBUF, rb = j & 1;
      bool got = mbar_wait_bounded(&tfull[b], uint32_t((j / NBUF) & 1), a.err, a.wait_limit);
      got = got && mbar_wait_bounded(&rfull[rb], uint32_t((j >> 1) & 1), a.err, a.wait_limit);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const float* srec = recs + rb * NE * REC;
      const int i = mtile * 128 + quarter * 32 + lane;  // output row of this thread
      const bool row_ok = i < Np;
      const uint32_t trow = tmem + uint32_t(b * TS::TCOLS) + (uint32_t(quarter * 32) << 16);
      for (int e0 = ehalf * NEH; e0 < (ehalf + 1) * NEH; e0 += EC) {
        float v[TS::NACC][EC];
#pragma unroll
        for (int p = 0; p < TS::NACC; ++p) {
          if constexpr (EC == 8)
            tc_ld8(trow + uint32_t(p * NE + e0), v[p]);
          else if constexpr (EC == 4)
            tc_ld4(trow + uint32_t(p * NE + e0), v[p]);
          else
            tc_ld2(trow + uint32_t(p * NE + e0), v[p]);
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
