// Tensor-core split-step variants of the acoustic model, N = 1..8, for the
// bf16x3 (2 pieces) and bf16x6 (3 pieces) modes: front halves with different
// elements per block, the same tcgen05 kernel.
#include "dg_launch.cuh"

namespace dgk {

const KernelCfg* kernel_variants_tc_acoustic(int N, int nsplit, int* count) {
#define DG_TC_AC(NS)                                                                                              \
  static const KernelCfg a1_##NS[] = {make_tc_cfg<0, 1, 16, NS>(), make_tc_cfg<0, 1, 32, NS>()};                \
  static const KernelCfg a2_##NS[] = {make_tc_cfg<0, 2, 16, NS>(), make_tc_cfg<0, 2, 8, NS>()};                 \
  static const KernelCfg a3_##NS[] = {make_tc_cfg<0, 3, 8, NS>(), make_tc_cfg<0, 3, 16, NS>()};                 \
  static const KernelCfg a4_##NS[] = {make_tc_cfg<0, 4, 8, NS, 256>(), make_tc_cfg<0, 4, 8, NS>()};             \
  static const KernelCfg a5_##NS[] = {make_tc_cfg<0, 5, 8, NS, 256>(), make_tc_cfg<0, 5, 8, NS>()};             \
  static const KernelCfg a6_##NS[] = {make_tc_cfg<0, 6, 8, NS, 384>(), make_tc_cfg<0, 6, 8, NS>()};             \
  static const KernelCfg a7_##NS[] = {make_tc_cfg<0, 7, 8, NS, 512>(), make_tc_cfg<0, 7, 8, NS>()};             \
  static const KernelCfg a8_##NS[] = {make_tc_cfg<0, 8, 8, NS, 512>(), make_tc_cfg<0, 8, 8, NS>()};             \
  static const KernelCfg* tab_##NS[8] = {a1_##NS, a2_##NS, a3_##NS, a4_##NS, a5_##NS, a6_##NS, a7_##NS, a8_##NS};
  DG_TC_AC(2)
  DG_TC_AC(3)
#undef DG_TC_AC
  if (N < 1 || N > 8 || (nsplit != 2 && nsplit != 3)) return nullptr;
  *count = 2;
  return nsplit == 2 ? tab_2[N - 1] : tab_3[N - 1];
}

}  // namespace dgk
