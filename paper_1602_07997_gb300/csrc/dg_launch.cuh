// Launch helpers shared by the per-model instantiation units.
#pragma once
#include "dg_gemm.cuh"
#include "dg_tc.cuh"

namespace dgk {

// number of variants in a table
template <size_t M>
constexpr int count_of(const KernelCfg (&)[M]) {
  return int(M);
}

// threads per CTA: one output tile per thread, at least two warps, warp multiple
template <int N, int EB, int TN>
constexpr int threads_for() {
  constexpr int t = Sz<N>::RT * (EB / TN);
  constexpr int u = t < 64 ? 64 : t;
  return (u + 31) / 32 * 32;
}

// HALO: neighbours outside the block fetched whole by bulk copies (acoustic).
template <int MODEL, int N, int EB, bool OPS_SMEM, bool R_SMEM, int TN = 1, int NT = threads_for<N, EB, TN>(),
          bool HALO = false>
KernelCfg make_cfg() {
  static_assert(Plan<MODEL, N, EB, OPS_SMEM, R_SMEM, MODEL == 0, false, HALO>::bytes <= 227 * 1024,
                "shared memory budget");
  KernelCfg c;
  c.EB = EB;
  c.TN = TN;
  c.NT = NT;
  c.ops_smem = OPS_SMEM;
  c.r_smem = R_SMEM;
  c.smem = Plan<MODEL, N, EB, OPS_SMEM, R_SMEM, MODEL == 0, false, HALO>::bytes;
  c.fn = dg_step_kernel<MODEL, N, EB, TN, NT, OPS_SMEM, R_SMEM, 0, 0, HALO>;
  c.fn_batched = dg_step_batched_kernel<MODEL, N, EB, TN, NT, OPS_SMEM, R_SMEM, 0, HALO>;
  c.split = 0;
  c.fn_gemm = nullptr;
  c.fn_gemm_batched = nullptr;
  c.smem_gemm = 0;
  c.gemm_threads = c.gemm_ne = c.gemm_mt = c.gemm_mtiles = c.gemm_kx = c.gemm_mp2 = c.gemm_nsplit = 0;
  c.gemm_xtile = 0;
  c.gemm_persistent = false;
  return c;
}

// Split variant: front half with EB elements per block, then the FP32 GEMM
// kernel of design V (1 = one thread per 4 rows x TN elements of every
// product, 2 = geometric combination at the volume/LIFT boundary and larger
// register tiles).
template <int MODEL, int N, int EB, int V = 1, int NT = threads_for<N, EB, 1>()>
KernelCfg make_split_cfg() {
  using SS = SplitShape<MODEL, N>;
  using G = typename GemmOf<MODEL, N, V>::T;
  static_assert(Plan<MODEL, N, EB, false, false, MODEL == 0, true>::bytes <= 227 * 1024, "shared memory budget");
  static_assert(G::smem <= 227 * 1024, "shared memory budget (GEMM)");
  static_assert((Sz<N>::Np + G::MT - 1) / G::MT * G::MT <= SS::OPP, "row tiles inside the operator pitch");

  KernelCfg c;
  c.EB = EB;
  c.TN = 1;
  c.NT = NT;
  c.ops_smem = false;
  c.r_smem = false;
  c.smem = Plan<MODEL, N, EB, false, false, MODEL == 0, true>::bytes;
  c.fn = dg_step_kernel<MODEL, N, EB, 1, NT, false, false, SS::NE>;
  c.fn_batched = dg_step_batched_kernel<MODEL, N, EB, 1, NT, false, false, SS::NE>;
  c.split = 1;
  c.fn_gemm = dg_split_gemm_kernel<MODEL, N, V>;
  c.fn_gemm_batched = dg_split_gemm_batched_kernel<MODEL, N, V>;
  c.smem_gemm = G::smem;
  c.gemm_threads = G::NT;
  c.gemm_ne = SS::NE;
  c.gemm_mt = G::MT;
  c.gemm_mtiles = G::MTILES_L;
  c.gemm_kx = SS::KX;
  c.gemm_mp2 = SS::OPP;
  c.gemm_nsplit = 0;
  c.gemm_xtile = size_t(SS::KX) * SS::NE * 4;
  c.gemm_persistent = false;
  return c;
}

// Split variant with the warp-specialised persistent GEMM (design W): NC
// consumer warps of TM rows each (acoustic 8, elastic 4 or 8), an NS-stage
// ring, MINB resident CTAs.
template <int MODEL, int N, int EB, int NC, int NS, int MINB = 1, int NT = threads_for<N, EB, 1>(),
          int TM = (MODEL == 0 ? 8 : 4)>
KernelCfg make_split_w_cfg() {
  using G = GemmW<MODEL, N, NC, NS, MINB, TM>;
  static_assert(Plan<MODEL, N, EB, false, false, MODEL == 0, true>::bytes <= 227 * 1024, "shared memory budget");
  static_assert(G::smem * MINB <= 227 * 1024, "shared memory budget (GEMM)");
  KernelCfg c = make_split_cfg<MODEL, N, EB, 3, NT>();
  c.fn_gemm = dg_split_gemm_w_kernel<MODEL, N, NC, NS, MINB, TM>;
  c.fn_gemm_batched = dg_split_gemm_w_batched_kernel<MODEL, N, NC, NS, MINB, TM>;
  c.smem_gemm = G::smem;
  c.gemm_threads = G::NT;
  c.gemm_mt = G::MT;
  c.gemm_mtiles = G::MTILES_L;
  c.gemm_persistent = true;
  return c;
}

// Tensor-core split variant: front half with EB elements per block writing
// the NSPLIT BF16 pieces of its GEMM inputs in the tensor-core chunk layout,
// then the tcgen05 kernel.
template <int MODEL, int N, int EB, int NSPLIT, int NT = threads_for<N, EB, 1>()>
KernelCfg make_tc_cfg() {
  using TS = TcShape<MODEL, N, NSPLIT>;
  static_assert(Plan<MODEL, N, EB, false, false>::bytes <= 227 * 1024, "shared memory budget");
  static_assert(TS::smem <= 227 * 1024, "shared memory budget (tensor-core kernel)");
  KernelCfg c;
  c.EB = EB;
  c.TN = 1;
  c.NT = NT;
  c.ops_smem = false;
  c.r_smem = false;
  c.smem = Plan<MODEL, N, EB, false, false>::bytes;
  c.fn = dg_step_kernel<MODEL, N, EB, 1, NT, false, false, TS::NE, NSPLIT>;
  c.fn_batched = nullptr;
  c.split = 2;
  c.fn_gemm = dg_tc_gemm_kernel<MODEL, N, NSPLIT>;
  c.fn_gemm_batched = nullptr;
  c.smem_gemm = TS::smem;
  c.gemm_threads = TS::NT;
  c.gemm_ne = TS::NE;
  c.gemm_mt = TS::MT;
  c.gemm_mtiles = TS::MTILES;
  c.gemm_kx = 0;
  c.gemm_mp2 = TS::MTILES * TS::MT;
  c.gemm_nsplit = NSPLIT;
  c.gemm_xtile = TS::TX::TILE;
  c.gemm_persistent = true;
  return c;
}

}  // namespace dgk
