// Tensor-core split-step variants of the elastic model, N = 1..8, for the
// bf16x3 (2 pieces) and bf16x6 (3 pieces) modes.
#include "dg_launch.cuh"

namespace dgk {

const KernelCfg* kernel_variants_tc_acoustic(int N, int nsplit, int* count);

const KernelCfg* kernel_variants_tc_elastic(int N, int nsplit, int* count) {
#define DG_TC_EL(NS)                                                                                              \
  static const KernelCfg e1_##NS[] = {make_tc_cfg<1, 1, 16, NS>(), make_tc_cfg<1, 1, 8, NS>()};                 \
  static const KernelCfg e2_##NS[] = {make_tc_cfg<1, 2, 8, NS>(), make_tc_cfg<1, 2, 4, NS>()};                  \
  static const KernelCfg e3_##NS[] = {make_tc_cfg<1, 3, 8, NS>(), make_tc_cfg<1, 3, 4, NS>()};                  \
  static const KernelCfg e4_##NS[] = {make_tc_cfg<1, 4, 8, NS, 256>(), make_tc_cfg<1, 4, 4, NS>()};             \
  static const KernelCfg e5_##NS[] = {make_tc_cfg<1, 5, 4, NS, 512>(), make_tc_cfg<1, 5, 4, NS>()};     \
  static const KernelCfg e6_##NS[] = {make_tc_cfg<1, 6, 4, NS, 512>(), make_tc_cfg<1, 6, 4, NS>()};     \
  static const KernelCfg e7_##NS[] = {make_tc_cfg<1, 7, 4, NS, 512>(), make_tc_cfg<1, 7, 4, NS>()};     \
  static const KernelCfg e8_##NS[] = {make_tc_cfg<1, 8, 4, NS, 512>(), make_tc_cfg<1, 8, 4, NS>()};     \
  static const KernelCfg* tab_##NS[8] = {e1_##NS, e2_##NS, e3_##NS, e4_##NS, e5_##NS, e6_##NS, e7_##NS, e8_##NS};
  DG_TC_EL(2)
  DG_TC_EL(3)
#undef DG_TC_EL
  static const int cnt[8] = {2, 2, 2, 2, 2, 2, 2, 2};
  if (N < 1 || N > 8 || (nsplit != 2 && nsplit != 3)) return nullptr;
  *count = cnt[N - 1];
  return nsplit == 2 ? tab_2[N - 1] : tab_3[N - 1];
}

const KernelCfg* kernel_variants_tc(int model, int N, int nsplit, int* count) {
  return model == 0 ? kernel_variants_tc_acoustic(N, nsplit, count) : kernel_variants_tc_elastic(N, nsplit, count);
}

}  // namespace dgk
