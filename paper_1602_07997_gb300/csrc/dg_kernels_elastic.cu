// Elastic (9-field) instantiations of the fused step kernel, N = 1..8, with
// the same variant scheme as the acoustic model.  Above N = 4 the AB3
// history is read from global memory in the update pass instead of being
// staged, to keep the shared-memory footprint down.
#include "dg_launch.cuh"

namespace dgk {

const KernelCfg* kernel_variants_elastic(int N, int* count) {
  static const KernelCfg v1[] = {make_cfg<1, 1, 16, true, true, 1, 128>(), make_cfg<1, 1, 8, true, true>(),
                                 make_cfg<1, 1, 32, true, true>(), make_cfg<1, 1, 16, true, true>(),
                                 make_cfg<1, 1, 32, true, true, 1, 256>(), ept_variant(1, 1, 0), ept_variant(1, 1, 1)};
  static const KernelCfg v2[] = {make_cfg<1, 2, 8, true, true, 1, 128>(), make_cfg<1, 2, 4, true, true>(),
                                 make_cfg<1, 2, 16, true, true>(), make_cfg<1, 2, 8, true, true>(),
                                 make_cfg<1, 2, 16, true, true, 1, 256>()};
  static const KernelCfg v3[] = {make_split_cfg<1, 3, 8, 3, 256>(), make_cfg<1, 3, 4, true, true>(),
                                 make_cfg<1, 3, 16, true, true>(), make_cfg<1, 3, 8, true, true, 1, 128>(),
                                 make_cfg<1, 3, 8, true, true>(), make_cfg<1, 3, 8, true, true, 1, 256>(),
                                 make_split_cfg<1, 3, 8, 2, 256>(), make_split_cfg<1, 3, 8, 7, 256>(),
                                 make_cfg<1, 3, 8, true, false, 1, 256>(), make_cfg<1, 3, 12, true, false, 1, 256>()};
  static const KernelCfg v4[] = {make_split_cfg<1, 4, 8, 3, 256>(), make_cfg<1, 4, 8, false, true>(),
                                 make_cfg<1, 4, 4, false, true>(), make_split_cfg<1, 4, 8>(),
                                 make_split_cfg<1, 4, 8, 2>(), make_cfg<1, 4, 4, true, true, 1, 128>(),
                                 make_cfg<1, 4, 4, true, true, 1, 256>(), make_split_cfg<1, 4, 4, 3, 256>(),
                                 make_cfg<1, 4, 4, true, true>(), make_split_cfg<1, 4, 8, 7, 256>(),
                                 make_cfg<1, 4, 8, true, false, 1, 256>(), make_cfg<1, 4, 4, true, false, 1, 128>()};
  static const KernelCfg v5[] = {make_split_cfg<1, 5, 8, 5, 512>(), make_cfg<1, 5, 4, false, false>(),
                                 make_split_cfg<1, 5, 4>(), make_split_cfg<1, 5, 4, 2>(),
                                 make_cfg<1, 5, 4, false, true>(), make_split_cfg<1, 5, 4, 3, 256>(),
                                 make_split_cfg<1, 5, 4, 3, 384>(), make_split_cfg<1, 5, 4, 3>(),
                                 make_split_cfg<1, 5, 4, 3, 512>(), make_split_cfg<1, 5, 8, 3, 512>(),
                                 make_split_cfg<1, 5, 8, 9, 512>(), make_split_w_cfg<1, 5, 8, 14, 4, 1, 512>()};
  static const KernelCfg v6[] = {make_split_cfg<1, 6, 8, 5, 512>(), make_cfg<1, 6, 4, false, false, 2>(),
                                 make_split_cfg<1, 6, 4>(), make_split_cfg<1, 6, 4, 2>(),
                                 make_cfg<1, 6, 4, false, false>(), make_split_cfg<1, 6, 4, 3, 256>(),
                                 make_split_cfg<1, 6, 4, 3, 384>(), make_split_cfg<1, 6, 4, 3>(),
                                 make_split_cfg<1, 6, 4, 5, 512>(), make_split_cfg<1, 6, 4, 3, 512>(),
                                 make_split_cfg<1, 6, 8, 3, 512>(), make_split_cfg<1, 6, 8, 9, 512>(),
                                 make_split_w_cfg<1, 6, 8, 11, 4, 1, 512>(), make_split_w_cfg<1, 6, 8, 11, 4, 1, 512, 8>()};
  static const KernelCfg v7[] = {make_split_cfg<1, 7, 8, 5, 512>(), make_cfg<1, 7, 4, false, false, 2>(),
                                 make_split_cfg<1, 7, 4>(), make_split_cfg<1, 7, 4, 2>(),
                                 make_cfg<1, 7, 4, false, false>(), make_split_cfg<1, 7, 4, 3, 256>(),
                                 make_split_cfg<1, 7, 4, 3, 384>(), make_split_cfg<1, 7, 4, 3>(),
                                 make_split_cfg<1, 7, 4, 3, 512>(), make_split_cfg<1, 7, 8, 3, 512>(),
                                 make_split_cfg<1, 7, 4, 5, 512>(), make_split_cfg<1, 7, 8, 9, 512>(),
                                 make_split_w_cfg<1, 7, 8, 15, 4, 1, 512>()};
  static const KernelCfg v8[] = {make_split_w_cfg<1, 8, 4, 14, 4, 1, 384>(), make_cfg<1, 8, 4, false, false, 2>(),
                                 make_split_cfg<1, 8, 4>(), make_cfg<1, 8, 4, false, false>(),
                                 make_split_cfg<1, 8, 4, 3>(), make_split_cfg<1, 8, 4, 3, 256>(),
                                 make_split_cfg<1, 8, 4, 3, 384>(), make_split_cfg<1, 8, 4, 2>(),
                                 make_split_cfg<1, 8, 4, 2, 384>(), make_split_cfg<1, 8, 4, 5, 512>(),
                                 make_split_cfg<1, 8, 4, 9, 384>(), make_split_cfg<1, 8, 4, 5, 384>(),
                                 make_split_w_cfg<1, 8, 4, 11, 4, 1, 384, 8>()};
  static const KernelCfg* tab[8] = {v1, v2, v3, v4, v5, v6, v7, v8};
  static const int cnt[8] = {count_of(v1), count_of(v2), count_of(v3), count_of(v4),
                             count_of(v5), count_of(v6), count_of(v7), count_of(v8)};
  if (N < 1 || N > 8) return nullptr;
  *count = cnt[N - 1];
  return tab[N - 1];
}

}  // namespace dgk
