"""Reference tetrahedron of the nodal DG scheme (oracle; test infrastructure).

Section 2.2: fields are represented by their values at Np = (N+1)(N+2)(N+3)/6
nodes per element, placed by the warp-and-blend technique (Warburton 2006),
with the multivariate Lagrange polynomials as basis and test functions.

Conventions (the paper does not fix them; they are the readings used on
both sides of the parity tests):

* reference tetrahedron v1=(-1,-1,-1), v2=(1,-1,-1), v3=(-1,1,-1),
  v4=(-1,-1,1);
* faces f1 = {v1,v2,v3} (t=-1), f2 = {v1,v2,v4} (s=-1),
  f3 = {v2,v3,v4} (r+s+t=-1), f4 = {v1,v3,v4} (r=-1);
* nodes ordered like the equispaced lattice (i,j,k), i+j+k <= N, with
  i (along r) fastest, then j (s), then k (t);
* warp-and-blend with blend parameter alpha = 0 (the optimised alpha
  values of Warburton 2006 are not available here).  The Lagrange
  operators do not depend on the node set except through rounding.

Operators built here by quadrature:
  M[i,j]   = int_T l_i l_j                         (mass)
  Dr[i,j]  = d l_j / dr (x_i), likewise Ds, Dt      (differentiation)
  E_f[i,j] = int_{f} l_i l_j  on the area-2 parametrisation of face f
  LIFT     = M^{-1} [E_1 | E_2 | E_3 | E_4]  restricted to face-node columns.
"""

import math

import numpy as np
from numpy.polynomial import legendre as npleg

REF_VERTS = np.array([[-1.0, -1.0, -1.0],
                      [1.0, -1.0, -1.0],
                      [-1.0, 1.0, -1.0],
                      [-1.0, -1.0, 1.0]])
# vertex indices (0-based) of each face, and the barycentric vanishing on it
FACE_VERTS = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))
FACE_OPPOSITE = (3, 2, 0, 1)
# outward reference normals, scaled so that the reference area vector is 2 * N_f
REF_NORMALS = np.array([[0.0, 0.0, -1.0],
                        [0.0, -1.0, 0.0],
                        [1.0, 1.0, 1.0],
                        [-1.0, 0.0, 0.0]])


def num_nodes(N):
    return (N + 1) * (N + 2) * (N + 3) // 6


def num_face_nodes(N):
    return (N + 1) * (N + 2) // 2


# ----------------------------------------------------------------------------
# node set
# ----------------------------------------------------------------------------

def lattice(N):
    """Integer lattice (i,j,k) of the equispaced nodes, i fastest."""
    out = []
    for k in range(N + 1):
        for j in range(N + 1 - k):
            for i in range(N + 1 - k - j):
                out.append((i, j, k))
    return np.array(out, dtype=np.int64)


def gll_points(N):
    """Gauss-Lobatto-Legendre points on [-1, 1], ascending."""
    if N == 1:
        return np.array([-1.0, 1.0])
    inner = npleg.legroots(npleg.legder([0.0] * N + [1.0]))
    return np.concatenate([[-1.0], np.sort(inner.real), [1.0]])


def _warp_quotient(N):
    """Coefficients (power basis) of w(x) = d(x) / (1 - x^2), where d is the
    degree-N polynomial through the equispaced points x_e with values
    (GLL point - equispaced point)."""
    xe = np.linspace(-1.0, 1.0, N + 1)
    disp = gll_points(N) - xe
    # interpolating polynomial, highest power first
    V = np.vander(xe, N + 1)
    d = np.linalg.solve(V, disp)
    q, rem = np.polydiv(d, np.array([-1.0, 0.0, 1.0]))
    assert np.max(np.abs(rem)) < 1e-12 if N >= 2 else True
    return q if N >= 2 else np.array([0.0])


def warp_blend_nodes(N, equispaced=False):
    """Reference coordinates [Np, 3] of the warp-and-blend nodes (alpha = 0).

    Construction (Warburton 2006): start from the equispaced lattice in an
    equilateral tetrahedron; a node on an edge moves along the edge by the
    1-D displacement from equispaced to GLL points; every other node moves
    by sum_F B_F W_F over the four faces F, where W_F sums, over the three
    edges (x, y) of F, 4 l_x l_y w(l_y - l_x) along the unit edge vector,
    and B_F = l_b l_c l_d / prod_{m in F} (l_m + l_a / 2) blends it into
    the volume (a = vertex opposite F).  The result is mapped back to the
    reference tetrahedron by the affine map that matches vertices.
    """
    lat = lattice(N)
    Np = lat.shape[0]
    lam_int = np.stack([N - lat.sum(axis=1), lat[:, 0], lat[:, 1], lat[:, 2]], axis=1)
    lam = lam_int / float(N)
    if equispaced or N <= 2:
        return lam @ REF_VERTS
    E = np.array([[-1.0, -1.0 / math.sqrt(3.0), -1.0 / math.sqrt(6.0)],
                  [1.0, -1.0 / math.sqrt(3.0), -1.0 / math.sqrt(6.0)],
                  [0.0, 2.0 / math.sqrt(3.0), -1.0 / math.sqrt(6.0)],
                  [0.0, 0.0, 3.0 / math.sqrt(6.0)]])
    wq = _warp_quotient(N)

    def w(x):
        return np.polyval(wq, x)

    def edge_unit(x, y):
        d = E[y] - E[x]
        return d / np.linalg.norm(d)

    X = lam @ E
    shift = np.zeros_like(X)
    for n in range(Np):
        l = lam[n]
        nz = np.nonzero(lam_int[n])[0]
        if len(nz) <= 2:
            if len(nz) == 2:
                x, y = nz
                xi = l[y] - l[x]
                shift[n] = (1.0 - xi * xi) * w(xi) * edge_unit(x, y)
            continue
        for a in range(4):
            bcd = [m for m in range(4) if m != a]
            Wf = np.zeros(3)
            for (x, y) in ((bcd[0], bcd[1]), (bcd[1], bcd[2]), (bcd[2], bcd[0])):
                Wf += 4.0 * l[x] * l[y] * w(l[y] - l[x]) * edge_unit(x, y)
            num = l[bcd[0]] * l[bcd[1]] * l[bcd[2]]
            den = np.prod([l[m] + 0.5 * l[a] for m in bcd])
            shift[n] += (num / den) * Wf
    Xw = X + shift
    # barycentrics of the warped points in the equilateral tet, then map
    A = np.vstack([E.T, np.ones((1, 4))])
    mu = np.linalg.solve(A, np.vstack([Xw.T, np.ones((1, Np))])).T
    return mu @ REF_VERTS


# ----------------------------------------------------------------------------
# basis: Bernstein polynomials in the barycentric coordinates of the tet
# ----------------------------------------------------------------------------

# d lambda_a / d (r, s, t) for lambda = (-(1+r+s+t)/2, (1+r)/2, (1+s)/2, (1+t)/2)
_DLAM = np.array([[-0.5, -0.5, -0.5],
                  [0.5, 0.0, 0.0],
                  [0.0, 0.5, 0.0],
                  [0.0, 0.0, 0.5]])


def barycentric(rst):
    r, s, t = rst[:, 0], rst[:, 1], rst[:, 2]
    return np.stack([-(1 + r + s + t) / 2.0, (1 + r) / 2.0, (1 + s) / 2.0, (1 + t) / 2.0], axis=1)


def basis_exponents(N):
    """Multi-indices (a1, a2, a3, a4), |a| = N, of the Bernstein basis."""
    return [(N - i - j - k, i, j, k) for k in range(N + 1) for j in range(N + 1 - k)
            for i in range(N + 1 - k - j)]


def basis_eval(N, rst, d=(0, 0, 0)):
    """[npts, Np] values (d = (0,0,0)) or one first derivative (d a unit
    triple) of the Bernstein basis B_a = N!/prod(a_m!) prod lambda_m^a_m."""
    lam = barycentric(rst)
    cols = []
    for a in basis_exponents(N):
        c = math.factorial(N) / np.prod([math.factorial(x) for x in a])
        if sum(d) == 0:
            cols.append(c * np.prod([lam[:, m] ** a[m] for m in range(4)], axis=0))
            continue
        axis = int(np.argmax(d))
        val = np.zeros(lam.shape[0])
        for m in range(4):
            if a[m] == 0 or _DLAM[m, axis] == 0.0:
                continue
            term = a[m] * _DLAM[m, axis] * lam[:, m] ** (a[m] - 1)
            for mm in range(4):
                if mm != m:
                    term = term * lam[:, mm] ** a[mm]
            val = val + term
        cols.append(c * val)
    return np.stack(cols, axis=1)


class Lagrange:
    """Lagrange basis of P_N through the given nodes (via a Vandermonde solve)."""

    def __init__(self, N, nodes):
        self.N = N
        self.nodes = nodes
        self.V = basis_eval(N, nodes)
        self.Vinv = np.linalg.inv(self.V)

    def eval(self, pts, d=(0, 0, 0)):
        """[npts, Np]: l_j or its derivative at pts."""
        return basis_eval(self.N, pts, d) @ self.Vinv


# ----------------------------------------------------------------------------
# quadrature (collapsed Gauss-Legendre / Duffy), exact to degree 2q-3
# ----------------------------------------------------------------------------

def tet_quadrature(q):
    x, w = npleg.leggauss(q)
    a, b, c = np.meshgrid(x, x, x, indexing="ij")
    wa, wb, wc = np.meshgrid(w, w, w, indexing="ij")
    r = (1 + a) * (1 - b) * (1 - c) / 4.0 - 1.0
    s = (1 + b) * (1 - c) / 2.0 - 1.0
    t = c
    W = wa * wb * wc * (1 - b) * (1 - c) ** 2 / 8.0
    return np.stack([r.ravel(), s.ravel(), t.ravel()], axis=1), W.ravel()


def tri_quadrature(q):
    """Points (u, v) on {u, v >= -1, u + v <= 0} (area 2) and weights."""
    x, w = npleg.leggauss(q)
    a, b = np.meshgrid(x, x, indexing="ij")
    wa, wb = np.meshgrid(w, w, indexing="ij")
    u = (1 + a) * (1 - b) / 2.0 - 1.0
    v = b
    W = wa * wb * (1 - b) / 2.0
    return np.stack([u.ravel(), v.ravel()], axis=1), W.ravel()


def face_points(f, uv):
    """Reference-tet coordinates of face f at triangle coordinates uv."""
    A, B, C = (REF_VERTS[i] for i in FACE_VERTS[f])
    return (A[None, :] + np.outer((1 + uv[:, 0]) / 2.0, B - A)
            + np.outer((1 + uv[:, 1]) / 2.0, C - A))


# ----------------------------------------------------------------------------
# operators
# ----------------------------------------------------------------------------

class RefElement:
    def __init__(self, N, nodes=None):
        self.N = N
        self.Np = num_nodes(N)
        self.Nfp = num_face_nodes(N)
        self.nodes = warp_blend_nodes(N) if nodes is None else nodes
        self.lag = Lagrange(N, self.nodes)
        r, s, t = self.nodes.T
        tol = 1e-10
        conds = (np.abs(t + 1) < tol, np.abs(s + 1) < tol,
                 np.abs(r + s + t + 1) < tol, np.abs(r + 1) < tol)
        self.Fmask = np.stack([np.nonzero(c)[0] for c in conds])  # [4, Nfp]
        assert self.Fmask.shape == (4, self.Nfp)
        # differentiation matrices: D[i, j] = d l_j / d r (x_i)
        self.Dr = self.lag.eval(self.nodes, (1, 0, 0))
        self.Ds = self.lag.eval(self.nodes, (0, 1, 0))
        self.Dt = self.lag.eval(self.nodes, (0, 0, 1))
        # mass matrix by quadrature
        qp, qw = tet_quadrature(N + 3)
        L = self.lag.eval(qp)
        self.M = L.T @ (qw[:, None] * L)
        self.Minv = np.linalg.inv(self.M)
        # face mass matrices and LIFT
        up, uw = tri_quadrature(N + 3)
        self.E = []
        lift_cols = []
        for f in range(4):
            Lf = self.lag.eval(face_points(f, up))
            Ef = Lf.T @ (uw[:, None] * Lf)
            self.E.append(Ef)
            lift_cols.append(self.Minv @ Ef[:, self.Fmask[f]])
        self.LIFT = np.concatenate(lift_cols, axis=1)  # [Np, 4 Nfp]
