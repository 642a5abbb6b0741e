// Helpers of the element-per-thread step kernels (acoustic, low N):
// compile-time face masks and the neighbour words of a block's elements.
#pragma once

#include "dg_facemask.h"
#include "dg_kernels.cuh"

namespace dgk {

// compile-time face masks: FaceNodes<N>::v[f][m] = volume node of face node m of face f
template <int N>
struct FaceNodes {
  struct T {
    int v[4][Sz<N>::Nfp];
  };
  static constexpr T make() {
    T t{};
    for (int f = 0; f < 4; ++f)
      for (int m = 0; m < Sz<N>::Nfp; ++m) t.v[f][m] = face_node(N, f, m);
    return t;
  }
  static constexpr T tab = make();
};

// neighbour word of face f
__device__ __forceinline__ int nbr_word(const int4 nb, int f) {
  return (f == 0) ? nb.x : (f == 1) ? nb.y : (f == 2) ? nb.z : nb.w;
}
// slot of face f among the outside faces of an element (0, 1, ... in face order)
__device__ __forceinline__ int outside_rank(const int4 nb, int f, int k0, int EB) {
  int r = 0;
  for (int g = 0; g < f; ++g) {
    const int w = nbr_word(nb, g);
    if (w >= 0) {
      const int le = (w >> kNbrShift) - k0;
      r += (le < 0 || le >= EB) ? 1 : 0;
    }
  }
  return r;
}

}  // namespace dgk
