// Elastic (9-field) instantiations of the fused step kernel, N = 1..8.
// TN = 1 element per thread tile (the 12 accumulator tiles of the volume
// products already take 48 registers); EB chosen as for the acoustic model.
#include "dg_launch.cuh"

namespace dgk {

const KernelCfg* kernel_cfg_elastic(int N) {
  static const KernelCfg cfg[8] = {
      make_cfg<1, 1, 64, 1, 64, true>(),   make_cfg<1, 2, 32, 1, 96, true>(),
      make_cfg<1, 3, 24, 1, 128, true>(),  make_cfg<1, 4, 12, 1, 128, true>(),
      make_cfg<1, 5, 8, 1, 128, false>(),  make_cfg<1, 6, 8, 1, 192, false>(),
      make_cfg<1, 7, 4, 1, 128, false>(),  make_cfg<1, 8, 4, 1, 192, false>(),
  };
  return (N >= 1 && N <= 8) ? &cfg[N - 1] : nullptr;
}

}  // namespace dgk
