// Acoustic (4-field) instantiations of the fused step kernel, N = 1..8.
// Tile choice per degree: TN = 2 elements per thread tile, EB elements per
// CTA so that (Mpad/4) * (EB/2) output tiles roughly fill NT threads; the
// operator blob is staged in shared memory up to N = 5 and read through L1
// above (it exceeds the shared-memory budget there).
#include "dg_launch.cuh"

namespace dgk {

const KernelCfg* kernel_cfg_acoustic(int N) {
  static const KernelCfg cfg[8] = {
      make_cfg<0, 1, 128, 2, 64, true>(),  make_cfg<0, 2, 64, 2, 96, true>(),
      make_cfg<0, 3, 48, 2, 128, true>(),  make_cfg<0, 4, 28, 2, 128, true>(),
      make_cfg<0, 5, 16, 2, 128, true>(),  make_cfg<0, 6, 12, 2, 128, false>(),
      make_cfg<0, 7, 8, 2, 128, false>(),  make_cfg<0, 8, 8, 2, 192, false>(),
  };
  return (N >= 1 && N <= 8) ? &cfg[N - 1] : nullptr;
}

}  // namespace dgk
