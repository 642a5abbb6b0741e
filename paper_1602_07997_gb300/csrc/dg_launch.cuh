// Launch helpers shared by the per-model instantiation units.
#pragma once
#include "dg_kernels.cuh"

namespace dgk {

template <int MODEL, int N, int EB, int TN, int NT, bool OPS_SMEM, bool R_SMEM>
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
  return c;
}

}  // namespace dgk
