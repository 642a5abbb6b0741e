// Acoustic (4-field) instantiations of the fused step kernel, N = 1..8.
// EB elements per block are chosen so that a CTA needs <= ~113 KB of shared
// memory (two CTAs per SM overlap each other's gather and product phases);
// the operator blob stays in shared memory up to N = 5 and is read through
// L1 above; the AB3 history of a block is bulk-copied into shared memory.
#include "dg_launch.cuh"

namespace dgk {

const KernelCfg* kernel_cfg_acoustic(int N) {
  //                                    N   EB TN  NT  ops_smem r_smem
  static const KernelCfg cfg[8] = {
      make_cfg<0, 1, 128, 1, 128, true, true>(), make_cfg<0, 2, 64, 1, 192, true, true>(),
      make_cfg<0, 3, 32, 1, 160, true, true>(),  make_cfg<0, 4, 20, 1, 192, true, true>(),
      make_cfg<0, 5, 8, 1, 128, true, true>(),   make_cfg<0, 6, 12, 1, 256, false, true>(),
      make_cfg<0, 7, 8, 1, 256, false, true>(),  make_cfg<0, 8, 4, 1, 192, false, true>(),
  };
  return (N >= 1 && N <= 8) ? &cfg[N - 1] : nullptr;
}

}  // namespace dgk
