// Acoustic (4-field) instantiations of the fused step kernel, N = 1..8.
// Each degree has a few variants (elements per block EB; threads = one
// 4-node x 1-element tile each); the autotuner times them on the caller's
// mesh and keeps the fastest; variant 0, the default, is the one measured
// fastest on the ~2 M-node sweep meshes.  The operator blob
// is staged in shared memory up to N = 4 and read through L1 above; at N = 1
// the default fetches neighbours outside the block whole (HALO).
#include "dg_launch.cuh"

namespace dgk {

const KernelCfg* kernel_variants_acoustic(int N, int* count) {
  static const KernelCfg v1[] = {make_cfg<0, 1, 32, true, true, 1, 128, true>(),
                                 make_cfg<0, 1, 32, true, true, 1, 128>(), make_cfg<0, 1, 64, true, true>(),
                                 make_cfg<0, 1, 32, true, true>(), make_cfg<0, 1, 128, true, true>(),
                                 make_cfg<0, 1, 16, true, true>(), make_cfg<0, 1, 64, true, true, 1, 256>(),
                                 make_cfg<0, 1, 32, true, true, 1, 256>(), make_cfg<0, 1, 64, true, true, 1, 512>(),
                                 ept_variant(0, 1, 0), ept_variant(0, 1, 1), ept_variant(0, 1, 2)};
  static const KernelCfg v2[] = {make_cfg<0, 2, 24, true, true, 1, 256>(), make_cfg<0, 2, 32, true, true>(),
                                 make_cfg<0, 2, 16, true, true>(), make_cfg<0, 2, 64, true, true>(),
                                 make_cfg<0, 2, 16, true, true, 1, 128>(), make_cfg<0, 2, 8, true, true>(),
                                 make_cfg<0, 2, 16, true, true, 1, 256>(), make_cfg<0, 2, 32, true, true, 1, 512>(),
                                 make_cfg<0, 2, 32, true, true, 1, 256>(), ept_variant(0, 2, 0), ept_variant(0, 2, 1)};
  static const KernelCfg v3[] = {make_cfg<0, 3, 12, true, true, 1, 256>(), make_cfg<0, 3, 4, true, true>(),
                                 make_cfg<0, 3, 16, true, true>(), make_cfg<0, 3, 32, true, true>(),
                                 make_cfg<0, 3, 16, true, true, 1, 128>(), make_cfg<0, 3, 8, true, true>(),
                                 make_cfg<0, 3, 32, true, true, 1, 256>(), make_cfg<0, 3, 32, true, true, 1, 512>(),
                                 make_cfg<0, 3, 16, true, true, 1, 256>(), make_cfg<0, 3, 12, true, true, 1, 192>(),
                                 make_cfg<0, 3, 12, true, false, 1, 256>(), make_cfg<0, 3, 16, true, false, 1, 256>()};
  static const KernelCfg v4[] = {make_cfg<0, 4, 12, true, true, 1, 256>(), make_cfg<0, 4, 4, true, true>(),
                                 make_cfg<0, 4, 8, true, true, 2>(), make_cfg<0, 4, 8, true, true>(),
                                 make_cfg<0, 4, 8, true, true, 1, 128>(), make_cfg<0, 4, 16, true, true, 1, 256>(),
                                 make_cfg<0, 4, 12, true, true>(), make_cfg<0, 4, 8, true, true, 1, 256>(),
                                 make_cfg<0, 4, 12, true, false, 1, 256>(), make_cfg<0, 4, 16, true, false, 1, 256>(),
                                 make_cfg<0, 4, 8, true, false, 1, 256>()};
  static const KernelCfg v5[] = {make_split_cfg<0, 5, 8, 4, 384>(), make_split_cfg<0, 5, 8, 2, 256>(),
                                 make_split_cfg<0, 5, 8, 8, 384>(), make_split_cfg<0, 5, 8, 6, 256>(),
                                 make_split_cfg<0, 5, 8, 7, 384>(),
                                 make_cfg<0, 5, 8, false, true, 2>(), make_cfg<0, 5, 4, true, true>(),
                                 make_cfg<0, 5, 12, false, true, 2>(),
                                 make_split_cfg<0, 5, 8>(), make_cfg<0, 5, 8, false, true>(),
                                 make_split_cfg<0, 5, 4, 2>(), make_split_cfg<0, 5, 8, 2>(),
                                 make_split_cfg<0, 5, 8, 2, 384>(), make_split_cfg<0, 5, 8, 2, 512>(),
                                 make_split_w_cfg<0, 5, 8, 7, 3, 2, 384>()};
  static const KernelCfg v6[] = {make_split_cfg<0, 6, 8, 3, 384>(), make_cfg<0, 6, 4, false, true>(),
                                 make_cfg<0, 6, 8, false, true, 2>(), make_cfg<0, 6, 4, false, true, 2>(),
                                 make_cfg<0, 6, 8, false, true>(), make_split_cfg<0, 6, 4>(),
                                 make_split_cfg<0, 6, 8, 2>(), make_split_cfg<0, 6, 8, 3>(),
                                 make_split_cfg<0, 6, 4, 2>(), make_split_cfg<0, 6, 8>(),
                                 make_split_cfg<0, 6, 8, 1, 512>(), make_split_cfg<0, 6, 8, 1, 384>(),
                                 make_split_cfg<0, 6, 8, 5, 384>(), make_split_cfg<0, 6, 8, 7, 384>(),
                                 make_split_cfg<0, 6, 8, 9, 384>(), make_split_cfg<0, 6, 8, 10, 384>(),
                                 make_split_w_cfg<0, 6, 8, 11, 4, 1, 384>()};
  static const KernelCfg v7[] = {make_split_cfg<0, 7, 8, 5, 512>(), make_cfg<0, 7, 4, false, true, 2>(),
                                 make_cfg<0, 7, 8, false, true, 2>(), make_cfg<0, 7, 4, false, true, 4>(),
                                 make_split_cfg<0, 7, 8>(), make_split_cfg<0, 7, 4>(),
                                 make_split_cfg<0, 7, 8, 2>(), make_cfg<0, 7, 4, false, true>(),
                                 make_split_cfg<0, 7, 4, 3>(), make_split_cfg<0, 7, 8, 3>(),
                                 make_split_cfg<0, 7, 8, 3, 768>(), make_split_cfg<0, 7, 8, 1, 512>(),
                                 make_split_cfg<0, 7, 8, 3, 512>(), make_split_cfg<0, 7, 8, 9, 512>(),
                                 make_split_cfg<0, 7, 8, 7, 512>(), make_split_cfg<0, 7, 8, 10, 512>(),
                                 make_split_w_cfg<0, 7, 8, 15, 4, 1, 512>(), make_split_w_cfg<0, 7, 8, 8, 4, 1, 512>()};
  static const KernelCfg v8[] = {make_split_w_cfg<0, 8, 8, 11, 5, 1, 512>(), make_cfg<0, 8, 4, false, true, 2>(),
                                 make_cfg<0, 8, 4, false, true, 4>(), make_cfg<0, 8, 8, false, true, 2>(),
                                 make_split_cfg<0, 8, 4>(), make_split_cfg<0, 8, 8>(),
                                 make_split_cfg<0, 8, 8, 2>(), make_cfg<0, 8, 4, false, true>(),
                                 make_split_cfg<0, 8, 4, 3>(), make_split_cfg<0, 8, 8, 2, 512>(),
                                 make_split_cfg<0, 8, 8, 5, 768>(), make_split_cfg<0, 8, 8, 7, 512>(),
                                 make_split_cfg<0, 8, 8, 9, 512>(), make_split_cfg<0, 8, 8, 10, 512>(),
                                 make_split_w_cfg<0, 8, 8, 11, 4, 1, 512>(), make_split_cfg<0, 8, 8, 3, 512>()};
  static const KernelCfg* tab[8] = {v1, v2, v3, v4, v5, v6, v7, v8};
  static const int cnt[8] = {count_of(v1), count_of(v2), count_of(v3), count_of(v4),
                             count_of(v5), count_of(v6), count_of(v7), count_of(v8)};
  if (N < 1 || N > 8) return nullptr;
  *count = cnt[N - 1];
  return tab[N - 1];
}

}  // namespace dgk
