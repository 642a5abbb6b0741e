// Elastic (9-field) instantiations of the fused step kernel, N = 1..8.
// TN = 1 (the 12 accumulator tiles of the volume products take 48
// registers).  Above N = 4 the AB3 history is read from global memory in
// the epilogue instead of being staged, to keep two CTAs per SM.
#include "dg_launch.cuh"

namespace dgk {

const KernelCfg* kernel_cfg_elastic(int N) {
  static const KernelCfg cfg[8] = {
      make_cfg<1, 1, 64, 1, 128, true, true>(),  make_cfg<1, 2, 32, 1, 128, true, true>(),
      make_cfg<1, 3, 16, 1, 128, true, true>(),  make_cfg<1, 4, 8, 1, 128, true, true>(),
      make_cfg<1, 5, 8, 1, 128, false, false>(), make_cfg<1, 6, 4, 1, 128, false, false>(),
      make_cfg<1, 7, 4, 1, 128, false, false>(), make_cfg<1, 8, 4, 1, 192, false, false>(),
  };
  return (N >= 1 && N <= 8) ? &cfg[N - 1] : nullptr;
}

}  // namespace dgk
