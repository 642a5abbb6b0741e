// Mesh validation, per-element geometric factors and face connectivity.
//
// Geometric factors (Section 2.2, "g^vol", "g^sur"): for the affine map
// x = x1 + A (1+r, 1+s, 1+t), A = [x2-x1 | x3-x1 | x4-x1] / 2, J = det A,
// g^vol_{ij} = dr_j/dx_i, and per face the outward normal n = g N_f/|g N_f|
// with g^sur = Fscale = sJ/J = |g N_f| (reference area vector 2 N_f).
// Faces are matched by sorted global vertex triples; the face-node
// permutation is the one of the six orientations that maps the neighbour's
// face vertices onto the element's own.
#include <algorithm>
#include <array>
#include <cmath>

#include "dg_internal.h"

namespace dg {

int HostMesh::build(const dg_mesh* m) {
  if (!m || !m->verts || !m->tets || m->ntets <= 0 || m->nverts < 4)
    return fail(DG_EINVAL, "empty or NULL mesh");
  K = m->ntets;
  const int64_t nv = m->nverts;
  A.assign(size_t(K) * 9, 0.0);
  J.assign(K, 0.0);
  g.assign(size_t(K) * 9, 0.0);
  nrm.assign(size_t(K) * 12, 0.0);
  fscale.assign(size_t(K) * 4, 0.0);
  double hmin3 = 1e300, hmax3 = 0;
  for (int64_t k = 0; k < K; ++k) {
    const int64_t* tv = m->tets + 4 * k;
    for (int a = 0; a < 4; ++a)
      if (tv[a] < 0 || tv[a] >= nv) return fail(DG_EINVAL, "tet vertex index out of range");
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b)
        if (tv[a] == tv[b]) return fail(DG_EINVAL, "tet with a repeated vertex");
    const double* x1 = m->verts + 3 * tv[0];
    double* Ak = &A[9 * k];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Ak[3 * i + j] = 0.5 * (m->verts[3 * tv[j + 1] + i] - x1[i]);
    double det = Ak[0] * (Ak[4] * Ak[8] - Ak[5] * Ak[7]) - Ak[1] * (Ak[3] * Ak[8] - Ak[5] * Ak[6]) +
                 Ak[2] * (Ak[3] * Ak[7] - Ak[4] * Ak[6]);
    J[k] = det;
    double scale = 0;
    for (int i = 0; i < 9; ++i) scale = std::max(scale, std::fabs(Ak[i]));
    if (!(det > 1e-12 * scale * scale * scale))
      return fail(DG_EINVAL, "inverted or degenerate tetrahedron " + std::to_string(k));
    hmin3 = std::min(hmin3, det);
    hmax3 = std::max(hmax3, det);
    // inverse: Ainv[j][i] = dr_j/dx_i ; g[i][j] = Ainv[j][i]
    double inv[9];
    inv[0] = (Ak[4] * Ak[8] - Ak[5] * Ak[7]) / det;
    inv[1] = (Ak[2] * Ak[7] - Ak[1] * Ak[8]) / det;
    inv[2] = (Ak[1] * Ak[5] - Ak[2] * Ak[4]) / det;
    inv[3] = (Ak[5] * Ak[6] - Ak[3] * Ak[8]) / det;
    inv[4] = (Ak[0] * Ak[8] - Ak[2] * Ak[6]) / det;
    inv[5] = (Ak[2] * Ak[3] - Ak[0] * Ak[5]) / det;
    inv[6] = (Ak[3] * Ak[7] - Ak[4] * Ak[6]) / det;
    inv[7] = (Ak[1] * Ak[6] - Ak[0] * Ak[7]) / det;
    inv[8] = (Ak[0] * Ak[4] - Ak[1] * Ak[3]) / det;
    double* gk = &g[9 * k];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) gk[3 * i + j] = inv[3 * j + i];
    for (int f = 0; f < 4; ++f) {
      double nv3[3];
      for (int i = 0; i < 3; ++i)
        nv3[i] = gk[3 * i] * kRefNormals[f][0] + gk[3 * i + 1] * kRefNormals[f][1] +
                 gk[3 * i + 2] * kRefNormals[f][2];
      double len = std::sqrt(nv3[0] * nv3[0] + nv3[1] * nv3[1] + nv3[2] * nv3[2]);
      fscale[4 * k + f] = len;
      for (int i = 0; i < 3; ++i) nrm[12 * k + 3 * f + i] = nv3[i] / len;
    }
  }
  // faces: sorted vertex triple -> (k, f).  With fewer than 2^21 vertices
  // the triple packs into one 64-bit key and the sort moves 16-byte records
  // (the served path builds a mesh per request on the host); otherwise the
  // triple itself is the key.
  struct FaceKey {
    std::array<int64_t, 3> v;
    int64_t kf;
  };
  struct PackedKey {
    uint64_t v;
    int64_t kf;
  };
  const bool packed = nv <= (int64_t(1) << 21);
  std::vector<FaceKey> keys;
  std::vector<PackedKey> pkeys;
  if (packed) pkeys.resize(size_t(K) * 4);
  else keys.resize(size_t(K) * 4);
  for (int64_t k = 0; k < K; ++k)
    for (int f = 0; f < 4; ++f) {
      std::array<int64_t, 3> v;
      for (int a = 0; a < 3; ++a) v[a] = m->tets[4 * k + kFaceVerts[f][a]];
      std::sort(v.begin(), v.end());
      if (packed) pkeys[4 * k + f] = {(uint64_t(v[0]) << 42) | (uint64_t(v[1]) << 21) | uint64_t(v[2]), 4 * k + f};
      else keys[4 * k + f] = {v, 4 * k + f};
    }
  if (packed)
    std::sort(pkeys.begin(), pkeys.end(),
              [](const PackedKey& a, const PackedKey& b) { return a.v != b.v ? a.v < b.v : a.kf < b.kf; });
  else
    std::sort(keys.begin(), keys.end(), [](const FaceKey& a, const FaceKey& b) {
      return a.v != b.v ? a.v < b.v : a.kf < b.kf;
    });
  const size_t nkeys = size_t(K) * 4;
  auto same = [&](size_t x, size_t y) { return packed ? pkeys[x].v == pkeys[y].v : keys[x].v == keys[y].v; };
  auto kf_of = [&](size_t x) { return packed ? pkeys[x].kf : keys[x].kf; };
  nbr.assign(size_t(K) * 4, -1);
  code.assign(K, 0u);
  for (int64_t k = 0; k < K; ++k) code[k] = 0x80808080u;  // all faces boundary until matched
  size_t i = 0;
  while (i < nkeys) {
    size_t j = i + 1;
    while (j < nkeys && same(j, i)) ++j;
    if (j - i > 2) return fail(DG_EINVAL, "non-conforming mesh: face shared by more than two tets");
    if (j - i == 2) {
      for (int side = 0; side < 2; ++side) {
        int64_t kf = kf_of(i + side), kf2 = kf_of(i + 1 - side);
        int64_t k = kf / 4, k2 = kf2 / 4;
        int f = int(kf % 4), f2 = int(kf2 % 4);
        if (k == k2) return fail(DG_EINVAL, "tet glued to itself");
        const int64_t* own = m->tets + 4 * k;
        const int64_t* oth = m->tets + 4 * k2;
        int pos[3];
        for (int x = 0; x < 3; ++x) {
          pos[x] = -1;
          for (int y = 0; y < 3; ++y)
            if (own[kFaceVerts[f][y]] == oth[kFaceVerts[f2][x]]) pos[x] = y;
        }
        int c = -1;
        for (int cc = 0; cc < 6; ++cc)
          if (RefElement::kPerms[cc][0] == pos[0] && RefElement::kPerms[cc][1] == pos[1] &&
              RefElement::kPerms[cc][2] == pos[2])
            c = cc;
        if (c < 0) return fail(DG_EINVAL, "face vertex permutation not found");
        nbr[4 * k + f] = int32_t(k2);
        uint32_t b = uint32_t(f2) | (uint32_t(c) << 2);
        code[k] = (code[k] & ~(0xffu << (8 * f))) | (b << (8 * f));
      }
    }
    i = j;
  }
  if (K > (int64_t(1) << 31) - 1) return fail(DG_EINVAL, "too many elements");
  (void)hmin3;
  (void)hmax3;
  return DG_OK;
}

}  // namespace dg
