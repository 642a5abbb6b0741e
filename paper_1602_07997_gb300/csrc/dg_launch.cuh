// Launch helpers shared by the per-model instantiation units.
#pragma once
#include "dg_kernels.cuh"

namespace dgk {

// threads per CTA: one output tile per thread, at least two warps, warp multiple
template <int N, int EB, int TN>
constexpr int threads_for() {
  constexpr int t = Sz<N>::RT * (EB / TN);
  constexpr int u = t < 64 ? 64 : t;
  return (u + 31) / 32 * 32;
}

template <int MODEL, int N, int EB, bool OPS_SMEM, bool R_SMEM, int TN = 1, int NT = threads_for<N, EB, TN>()>
KernelCfg make_cfg() {
  static_assert(Plan<MODEL, N, EB, OPS_SMEM, R_SMEM>::bytes <= 227 * 1024, "shared memory budget");
  KernelCfg c;
  c.EB = EB;
  c.TN = TN;
  c.NT = NT;
  c.ops_smem = OPS_SMEM;
  c.r_smem = R_SMEM;
  c.smem = Plan<MODEL, N, EB, OPS_SMEM, R_SMEM>::bytes;
  c.fn = dg_step_kernel<MODEL, N, EB, TN, NT, OPS_SMEM, R_SMEM>;
  c.fn_batched = dg_step_batched_kernel<MODEL, N, EB, TN, NT, OPS_SMEM, R_SMEM>;
  return c;
}

}  // namespace dgk
