// Internal declarations of libdg (host side).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/dg.h"

namespace dg {

// thread-local error message, returns the code for convenience
int fail(int code, const std::string& msg);

inline int num_nodes(int N) { return (N + 1) * (N + 2) * (N + 3) / 6; }
inline int num_face_nodes(int N) { return (N + 1) * (N + 2) / 2; }
inline int num_fields(int model) { return model == DG_ACOUSTIC ? 4 : 9; }

// Vertices of each reference face (0-based), shared ordering convention:
// f0 = {v1,v2,v3} (t=-1), f1 = {v1,v2,v4} (s=-1), f2 = {v2,v3,v4}, f3 = {v1,v3,v4} (r=-1).
extern const int kFaceVerts[4][3];
// Outward reference normals scaled so that the reference area vector is 2 * n.
extern const double kRefNormals[4][3];

// Reference element of degree N in double precision.
struct RefElement {
  int N = 0, Np = 0, Nfp = 0;
  std::vector<double> r, s, t;        // [Np] node coordinates
  std::vector<int> lat;               // [Np][4] integer barycentrics (sum N)
  std::vector<double> V;              // [Np][Np] orthonormal Vandermonde V[n][m] = psi_m(x_n)
  std::vector<double> Dr, Ds, Dt;     // [Np][Np]
  std::vector<double> LIFT;           // [Np][4 Nfp], columns face-major, face-local order
  std::vector<int> fmask;             // [4][Nfp] node index of face-local node m
  std::vector<int> perm;              // [6][Nfp] face-local index on the neighbour side
  // permutation code tables: kPerms[c][x] = position y in the own face triple
  // whose global vertex equals the neighbour's x-th face vertex
  static const int kPerms[6][3];
  int build(int N);
  // orthonormal basis (Dubiner) values at one point, [Np]
  void basis(double r, double s, double t, double* out) const;
};

// Per-mesh host geometry, double precision.
struct HostMesh {
  int64_t K = 0;
  std::vector<double> A;       // [K][3][3] dx_i/dr_j
  std::vector<double> J;       // [K]
  std::vector<double> g;       // [K][3][3] dr_j/dx_i stored g[k][i][j]
  std::vector<double> nrm;     // [K][4][3]
  std::vector<double> fscale;  // [K][4]
  std::vector<int32_t> nbr;    // [K][4] neighbour element, -1 on the boundary
  std::vector<uint32_t> code;  // [K] 8 bits per face: f' (2), perm (3), boundary (bit 7)
  int build(const dg_mesh* m);
};

}  // namespace dg
