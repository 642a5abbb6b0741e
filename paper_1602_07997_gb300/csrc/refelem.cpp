// Reference tetrahedron of the nodal DG scheme (Section 2.2): warp-and-blend
// nodes, orthonormal (Dubiner) basis, differentiation and lift matrices.
//
// Route: D_r = V_r V^{-1}, M^{-1} = V V^T (V orthonormal), face mass
// E_f = (V_f V_f^T)^{-1} with the 2-D orthonormal basis on the face's own
// nodes, LIFT = V V^T [E_1 | ... | E_4].  Face nodes and the neighbour
// permutations are derived from the integer lattice barycentrics, so no
// floating-point matching is involved.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>

#include "dg_internal.h"

namespace dg {

const int kFaceVerts[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};
const double kRefNormals[4][3] = {{0, 0, -1}, {0, -1, 0}, {1, 1, 1}, {-1, 0, 0}};
const int RefElement::kPerms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                      {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

namespace {

// In-place inverse of an n x n row-major matrix, Gauss-Jordan with partial pivoting.
bool invert(std::vector<double>& a, int n) {
  std::vector<double> inv(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) inv[size_t(i) * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[size_t(r) * n + c]) > std::fabs(a[size_t(p) * n + c])) p = r;
    if (a[size_t(p) * n + c] == 0.0) return false;
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(a[size_t(p) * n + k], a[size_t(c) * n + k]);
        std::swap(inv[size_t(p) * n + k], inv[size_t(c) * n + k]);
      }
    double d = 1.0 / a[size_t(c) * n + c];
    for (int k = 0; k < n; ++k) {
      a[size_t(c) * n + k] *= d;
      inv[size_t(c) * n + k] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = a[size_t(r) * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[size_t(r) * n + k] -= f * a[size_t(c) * n + k];
        inv[size_t(r) * n + k] -= f * inv[size_t(c) * n + k];
      }
    }
  }
  a.swap(inv);
  return true;
}

// C = A (m x k) * B (k x n), row-major
std::vector<double> matmul(const std::vector<double>& A, const std::vector<double>& B, int m,
                           int k, int n) {
  std::vector<double> C(size_t(m) * n, 0.0);
  for (int i = 0; i < m; ++i)
    for (int l = 0; l < k; ++l) {
      double a = A[size_t(i) * k + l];
      if (a == 0.0) continue;
      for (int j = 0; j < n; ++j) C[size_t(i) * n + j] += a * B[size_t(l) * n + j];
    }
  return C;
}

// Orthonormal Jacobi polynomial P_n^{(a,b)}(x) on [-1,1] (three-term recurrence).
double jacobi(int n, double a, double b, double x) {
  double g0 = std::pow(2.0, a + b + 1) / (a + b + 1) * std::tgamma(a + 1) * std::tgamma(b + 1) /
              std::tgamma(a + b + 1);
  double p0 = 1.0 / std::sqrt(g0);
  if (n == 0) return p0;
  double g1 = (a + 1) * (b + 1) / (a + b + 3) * g0;
  double p1 = ((a + b + 2) * x / 2 + (a - b) / 2) / std::sqrt(g1);
  if (n == 1) return p1;
  double aold = 2 / (2 + a + b) * std::sqrt((a + 1) * (b + 1) / (a + b + 3));
  for (int i = 1; i < n; ++i) {
    double h1 = 2 * i + a + b;
    double anew = 2 / (h1 + 2) *
                  std::sqrt((i + 1) * (i + 1 + a + b) * (i + 1 + a) * (i + 1 + b) /
                            ((h1 + 1) * (h1 + 3)));
    double bnew = -(a * a - b * b) / (h1 * (h1 + 2));
    double p2 = (-aold * p0 + (x - bnew) * p1) / anew;
    p0 = p1;
    p1 = p2;
    aold = anew;
  }
  return p1;
}

double djacobi(int n, double a, double b, double x) {
  if (n == 0) return 0.0;
  return std::sqrt(n * (n + a + b + 1)) * jacobi(n - 1, a + 1, b + 1, x);
}

double ipow(double x, int e) {
  double r = 1.0;
  for (int i = 0; i < e; ++i) r *= x;
  return r;
}

// Collapsed coordinates of a reference point.
void collapse3(double r, double s, double t, double* a, double* b, double* c) {
  *a = (std::fabs(s + t) > 1e-14) ? 2 * (1 + r) / (-s - t) - 1 : -1.0;
  *b = (std::fabs(t - 1) > 1e-14) ? 2 * (1 + s) / (1 - t) - 1 : -1.0;
  *c = t;
}

struct Idx3 {
  int i, j, k;
};
std::vector<Idx3> basis_index(int N) {
  std::vector<Idx3> v;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j)
      for (int k = 0; k <= N - i - j; ++k) v.push_back({i, j, k});
  return v;
}

// value and reference gradient of psi_ijk at (r,s,t)
void psi3(const Idx3& id, double r, double s, double t, double* v, double* dr, double* ds,
          double* dt) {
  double a, b, c;
  collapse3(r, s, t, &a, &b, &c);
  const int i = id.i, j = id.j, k = id.k;
  const double C = 2.0 * std::sqrt(2.0);
  double fa = jacobi(i, 0, 0, a), dfa = djacobi(i, 0, 0, a);
  double gb = jacobi(j, 2 * i + 1, 0, b), dgb = djacobi(j, 2 * i + 1, 0, b);
  double hc = jacobi(k, 2 * i + 2 * j + 2, 0, c), dhc = djacobi(k, 2 * i + 2 * j + 2, 0, c);
  double ob = 1 - b, oc = 1 - c;
  if (v) *v = C * fa * gb * ipow(ob, i) * hc * ipow(oc, i + j);
  if (!dr) return;
  // d/dr = 4/((1-b)(1-c)) d/da
  double Vr = 4 * C * dfa * gb * ipow(ob, std::max(i - 1, 0)) * hc * ipow(oc, std::max(i + j - 1, 0));
  if (i == 0) Vr = 0.0;
  // (2/(1-c)) d/db
  double Tb = 2 * C * fa * (dgb * ipow(ob, i) - (i ? i * gb * ipow(ob, i - 1) : 0.0)) * hc *
              ipow(oc, std::max(i + j - 1, 0));
  if (i + j == 0) Tb = 0.0;
  // d/dc
  double Tc = C * fa * gb * ipow(ob, i) *
              (dhc * ipow(oc, i + j) - (i + j ? (i + j) * hc * ipow(oc, i + j - 1) : 0.0));
  *dr = Vr;
  *ds = 0.5 * (1 + a) * Vr + Tb;
  *dt = 0.5 * (1 + a) * Vr + 0.5 * (1 + b) * Tb + Tc;
}

// 2-D orthonormal basis on {u,v >= -1, u+v <= 0}
double psi2(int i, int j, double u, double v) {
  double a = (std::fabs(v - 1) > 1e-14) ? 2 * (1 + u) / (1 - v) - 1 : -1.0;
  return std::sqrt(2.0) * jacobi(i, 0, 0, a) * jacobi(j, 2 * i + 1, 0, v) * ipow(1 - v, i);
}

// Gauss-Lobatto-Legendre points, ascending (Newton on P_N').
std::vector<double> gll(int N) {
  std::vector<double> x(N + 1);
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double z = -std::cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      // Legendre P_N and its first two derivatives by recurrence
      double p0 = 1.0, p1 = z;
      for (int n = 1; n < N; ++n) {
        double p2 = ((2 * n + 1) * z * p1 - n * p0) / (n + 1);
        p0 = p1;
        p1 = p2;
      }
      double dP = N * (z * p1 - p0) / (z * z - 1);
      double d2P = (2 * z * dP - N * (N + 1) * p1) / (1 - z * z);
      double dz = dP / d2P;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  std::sort(x.begin(), x.end());
  return x;
}

// w(x) = (sum_i (x_gll_i - x_eq_i) l_i^{eq}(x)) / (1 - x^2), written as the
// product over interior equispaced points (the endpoint factors cancel).
double warp_factor(int N, const std::vector<double>& xg, double x) {
  double w = 0.0;
  for (int i = 1; i < N; ++i) {
    double xi = -1.0 + 2.0 * i / N;
    double d = xg[i] - xi;
    double l = 1.0;
    for (int j = 1; j < N; ++j) {
      if (j == i) continue;
      double xj = -1.0 + 2.0 * j / N;
      l *= (x - xj) / (xi - xj);
    }
    w += d * l / (1 - xi * xi);
  }
  return w;
}

}  // namespace

void RefElement::basis(double rr, double ss, double tt, double* out) const {
  auto idx = basis_index(N);
  for (size_t m = 0; m < idx.size(); ++m) psi3(idx[m], rr, ss, tt, &out[m], nullptr, nullptr, nullptr);
}

int RefElement::build(int N_) {
  N = N_;
  if (N < 1 || N > 8) return fail(DG_EINVAL, "polynomial degree N must be in 1..8");
  Np = num_nodes(N);
  Nfp = num_face_nodes(N);
  // equispaced lattice, i (r) fastest, then j (s), then k (t)
  lat.assign(size_t(Np) * 4, 0);
  {
    int n = 0;
    for (int k = 0; k <= N; ++k)
      for (int j = 0; j <= N - k; ++j)
        for (int i = 0; i <= N - k - j; ++i, ++n) {
          lat[4 * n + 0] = N - i - j - k;  // weight of v1
          lat[4 * n + 1] = i;              // v2
          lat[4 * n + 2] = j;              // v3
          lat[4 * n + 3] = k;              // v4
        }
  }
  // warp & blend (blend parameter 0) in an equilateral tetrahedron
  const double s3 = std::sqrt(3.0), s6 = std::sqrt(6.0);
  const double E[4][3] = {{-1, -1 / s3, -1 / s6}, {1, -1 / s3, -1 / s6}, {0, 2 / s3, -1 / s6}, {0, 0, 3 / s6}};
  const double RV[4][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
  std::vector<double> xg = gll(N);
  r.assign(Np, 0);
  s.assign(Np, 0);
  t.assign(Np, 0);
  for (int n = 0; n < Np; ++n) {
    double L[4];
    int nz = 0, nzi[4];
    for (int a = 0; a < 4; ++a) {
      L[a] = double(lat[4 * n + a]) / N;
      if (lat[4 * n + a] != 0) nzi[nz++] = a;
    }
    double X[3] = {0, 0, 0}, D[3] = {0, 0, 0};
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) X[d] += L[a] * E[a][d];
    auto edge_add = [&](int x, int y, double scale, double* acc) {
      double u[3], len = 0;
      for (int d = 0; d < 3; ++d) {
        u[d] = E[y][d] - E[x][d];
        len += u[d] * u[d];
      }
      len = std::sqrt(len);
      for (int d = 0; d < 3; ++d) acc[d] += scale * u[d] / len;
    };
    if (N >= 3) {
      if (nz == 2) {
        int x = nzi[0], y = nzi[1];
        double xi = L[y] - L[x];
        edge_add(x, y, (1 - xi * xi) * warp_factor(N, xg, xi), D);
      } else if (nz > 2) {
        for (int a = 0; a < 4; ++a) {
          int b[3], nb = 0;
          for (int m = 0; m < 4; ++m)
            if (m != a) b[nb++] = m;
          double W[3] = {0, 0, 0};
          const int ed[3][2] = {{b[0], b[1]}, {b[1], b[2]}, {b[2], b[0]}};
          for (auto& e : ed) {
            int x = e[0], y = e[1];
            edge_add(x, y, 4 * L[x] * L[y] * warp_factor(N, xg, L[y] - L[x]), W);
          }
          double den = (L[b[0]] + 0.5 * L[a]) * (L[b[1]] + 0.5 * L[a]) * (L[b[2]] + 0.5 * L[a]);
          double blend = L[b[0]] * L[b[1]] * L[b[2]] / den;
          for (int d = 0; d < 3; ++d) D[d] += blend * W[d];
        }
      }
    }
    for (int d = 0; d < 3; ++d) X[d] += D[d];
    // barycentrics of X in the equilateral tet (solve 4x4), then map to reference
    std::vector<double> M(16);
    for (int a = 0; a < 4; ++a) {
      for (int d = 0; d < 3; ++d) M[d * 4 + a] = E[a][d];
      M[12 + a] = 1.0;
    }
    invert(M, 4);
    double rhs[4] = {X[0], X[1], X[2], 1.0}, mu[4];
    for (int a = 0; a < 4; ++a) {
      mu[a] = 0;
      for (int b = 0; b < 4; ++b) mu[a] += M[a * 4 + b] * rhs[b];
    }
    double P[3] = {0, 0, 0};
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) P[d] += mu[a] * RV[a][d];
    // snap nodes exactly onto faces they belong to (lattice weight zero)
    r[n] = P[0];
    s[n] = P[1];
    t[n] = P[2];
    if (lat[4 * n + 1] == 0) r[n] = -1.0;
    if (lat[4 * n + 2] == 0) s[n] = -1.0;
    if (lat[4 * n + 3] == 0) t[n] = -1.0;
  }
  // Vandermonde and gradient Vandermondes
  auto idx = basis_index(N);
  V.assign(size_t(Np) * Np, 0);
  std::vector<double> Vr(V), Vs(V), Vt(V);
  for (int n = 0; n < Np; ++n)
    for (int m = 0; m < Np; ++m)
      psi3(idx[m], r[n], s[n], t[n], &V[size_t(n) * Np + m], &Vr[size_t(n) * Np + m],
           &Vs[size_t(n) * Np + m], &Vt[size_t(n) * Np + m]);
  std::vector<double> Vinv(V);
  if (!invert(Vinv, Np)) return fail(DG_EINVAL, "singular Vandermonde");
  Dr = matmul(Vr, Vinv, Np, Np, Np);
  Ds = matmul(Vs, Vinv, Np, Np, Np);
  Dt = matmul(Vt, Vinv, Np, Np, Np);

  // face-local numbering: m <-> (i, j): i toward the face's 2nd vertex, j toward its 3rd
  std::map<std::array<int, 4>, int> node_of;
  for (int n = 0; n < Np; ++n)
    node_of[{lat[4 * n], lat[4 * n + 1], lat[4 * n + 2], lat[4 * n + 3]}] = n;
  std::vector<std::pair<int, int>> fij;
  for (int j = 0; j <= N; ++j)
    for (int i = 0; i <= N - j; ++i) fij.push_back({i, j});
  auto flocal = [&](int i, int j) {
    int m = 0;
    for (int jj = 0; jj < j; ++jj) m += N + 1 - jj;
    return m + i;
  };
  fmask.assign(4 * Nfp, 0);
  for (int f = 0; f < 4; ++f)
    for (int m = 0; m < Nfp; ++m) {
      std::array<int, 4> w = {0, 0, 0, 0};
      w[kFaceVerts[f][0]] = N - fij[m].first - fij[m].second;
      w[kFaceVerts[f][1]] = fij[m].first;
      w[kFaceVerts[f][2]] = fij[m].second;
      fmask[f * Nfp + m] = node_of.at(w);
    }
  perm.assign(6 * Nfp, 0);
  for (int c = 0; c < 6; ++c)
    for (int m = 0; m < Nfp; ++m) {
      int w[3] = {N - fij[m].first - fij[m].second, fij[m].first, fij[m].second};
      // neighbour's x-th face vertex is own face vertex kPerms[c][x]
      int i2 = w[kPerms[c][1]], j2 = w[kPerms[c][2]];
      perm[c * Nfp + m] = flocal(i2, j2);
    }

  // face mass matrices with the 2-D orthonormal basis in face coordinates
  std::vector<double> Emat(size_t(Np) * 4 * Nfp, 0.0);
  for (int f = 0; f < 4; ++f) {
    std::vector<double> V2(size_t(Nfp) * Nfp);
    for (int m = 0; m < Nfp; ++m) {
      int n = fmask[f * Nfp + m];
      double u, v;
      if (f == 0) { u = r[n]; v = s[n]; }
      else if (f == 1) { u = r[n]; v = t[n]; }
      else { u = s[n]; v = t[n]; }
      int col = 0;
      for (int i = 0; i <= N; ++i)
        for (int j = 0; j <= N - i; ++j) V2[size_t(m) * Nfp + col++] = psi2(i, j, u, v);
    }
    // E_f = (V2 V2^T)^{-1}
    std::vector<double> G(size_t(Nfp) * Nfp, 0.0);
    for (int a = 0; a < Nfp; ++a)
      for (int b = 0; b < Nfp; ++b) {
        double acc = 0;
        for (int c = 0; c < Nfp; ++c) acc += V2[size_t(a) * Nfp + c] * V2[size_t(b) * Nfp + c];
        G[size_t(a) * Nfp + b] = acc;
      }
    if (!invert(G, Nfp)) return fail(DG_EINVAL, "singular face Vandermonde");
    for (int a = 0; a < Nfp; ++a)
      for (int b = 0; b < Nfp; ++b)
        Emat[size_t(fmask[f * Nfp + a]) * 4 * Nfp + f * Nfp + b] = G[size_t(a) * Nfp + b];
  }
  // LIFT = V (V^T Emat)
  std::vector<double> VT(size_t(Np) * Np);
  for (int a = 0; a < Np; ++a)
    for (int b = 0; b < Np; ++b) VT[size_t(a) * Np + b] = V[size_t(b) * Np + a];
  LIFT = matmul(V, matmul(VT, Emat, Np, Np, 4 * Nfp), Np, Np, 4 * Nfp);
  return DG_OK;
}

}  // namespace dg
