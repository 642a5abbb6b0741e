// Compile-time node numbering of the reference tetrahedron (plain C++,
// usable from host and device code).
//
// Nodes are numbered in the order of the equispaced lattice: (i, j, k) with
// i + j + k <= N, i (along r) fastest, then j (s), then k (t); the node's
// barycentric weights are (N - i - j - k, i, j, k) for the vertices
// v1..v4.  Face f is spanned by the vertices kFaceVertsC[f]; its face-local
// node m = (a, b) (b outer, a inner, a + b <= N) has weight a on the face's
// second vertex, b on its third and N - a - b on its first.  These are the
// tables the library builds at run time (face masks); a kernel that unrolls
// its face loops reads them as constants.  dg_setup checks the two agree.
#pragma once

namespace dgk {

constexpr int kFaceVertsC[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

// volume node of lattice point (i, j, k)
constexpr int lattice_node(int N, int i, int j, int k) {
  int n = 0;
  for (int kk = 0; kk < k; ++kk) n += (N - kk + 1) * (N - kk + 2) / 2;
  for (int jj = 0; jj < j; ++jj) n += N - k - jj + 1;
  return n + i;
}

// volume node of face-local node m of face f
constexpr int face_node(int N, int f, int m) {
  int b = 0, a = m;
  while (a > N - b) {
    a -= N - b + 1;
    ++b;
  }
  int w[4] = {0, 0, 0, 0};
  w[kFaceVertsC[f][0]] = N - a - b;
  w[kFaceVertsC[f][1]] = a;
  w[kFaceVertsC[f][2]] = b;
  return lattice_node(N, w[1], w[2], w[3]);
}

}  // namespace dgk
