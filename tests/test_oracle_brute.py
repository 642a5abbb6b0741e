"""Brute-force pin of the oracle RHS on a perturbed 6-tet cube.

Independently of the oracle's reference element, every element's RHS is
recomputed from the weak form in *physical* coordinates:
  * Lagrange basis rebuilt from a physical-coordinate monomial Vandermonde
    through the element's physical nodes;
  * volume integrals by a degree-(2N+1) collapsed Gauss rule on the physical
    tet, face integrals by a collapsed Gauss rule on each physical triangle;
  * neighbour traces evaluated pointwise from the neighbour's polynomial at
    the face quadrature points (no face-node matching), face normals from
    cross products of the face's edges;
  * the element mass matrix by the same quadrature, solved in float64.
The penalty values at each quadrature point come from the flux functions,
which are pinned separately against the Riemann problem.  Agreement pins the
geometry, normals, Fscale, face matching and the LIFT convention together.
"""

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import workloads as W
from oracle.dg import Solver, acoustic_penalty, elastic_penalty, SIG


def _gauss01(q):
    x, w = npleg.leggauss(q)
    return (x + 1) / 2, w / 2


def _tet_rule(q):
    """Points (xi1, xi2, xi3) in the unit simplex and weights (sum = 1/6)."""
    x, w = _gauss01(q)
    u, v, s = np.meshgrid(x, x, x, indexing="ij")
    wu, wv, ws = np.meshgrid(w, w, w, indexing="ij")
    xi1 = u
    xi2 = v * (1 - u)
    xi3 = s * (1 - u) * (1 - v)
    W_ = wu * wv * ws * (1 - u) ** 2 * (1 - v)
    return np.stack([xi1.ravel(), xi2.ravel(), xi3.ravel()], 1), W_.ravel()


def _tri_rule(q):
    x, w = _gauss01(q)
    u, v = np.meshgrid(x, x, indexing="ij")
    wu, wv = np.meshgrid(w, w, indexing="ij")
    return np.stack([u.ravel(), (v * (1 - u)).ravel()], 1), (wu * wv * (1 - u)).ravel()


class PhysBasis:
    def __init__(self, N, nodes, centre):
        self.exps = [(a, b, c) for a in range(N + 1) for b in range(N + 1 - a)
                     for c in range(N + 1 - a - b)]
        self.c0 = centre
        self.Cinv = np.linalg.inv(self._mono(nodes))

    def _mono(self, x, d=None):
        y = x - self.c0
        cols = []
        for (a, b, c) in self.exps:
            e = [a, b, c]
            if d is None:
                cols.append(y[:, 0] ** a * y[:, 1] ** b * y[:, 2] ** c)
            else:
                if e[d] == 0:
                    cols.append(np.zeros(len(y)))
                    continue
                f = float(e[d])
                e[d] -= 1
                cols.append(f * y[:, 0] ** e[0] * y[:, 1] ** e[1] * y[:, 2] ** e[2])
        return np.stack(cols, 1)

    def ell(self, x, d=None):
        return self._mono(x, d) @ self.Cinv


def _brute_rhs(S, q):
    m = S.mesh
    verts, tets = m.verts, m.tets
    N, K, Nf = S.N, m.K, S.Nf
    bases = [PhysBasis(N, m.x[k], verts[tets[k]].mean(0)) for k in range(K)]
    tp, tw = _tet_rule(N + 3)
    fp, fw = _tri_rule(N + 3)
    faces = {}
    for k in range(K):
        for skip in range(4):
            key = frozenset(int(v) for j, v in enumerate(tets[k]) if j != skip)
            faces.setdefault(key, []).append(k)
    out = np.zeros_like(q)
    for k in range(K):
        B = bases[k]
        X = verts[tets[k]]
        vol6 = abs(np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], 1)))
        xq = X[0] + tp @ np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]])
        wq = tw * vol6
        L = B.ell(xq)
        G = [B.ell(xq, d) for d in range(3)]
        Mk = L.T @ (wq[:, None] * L)
        val = L @ q[k].T                       # [nq, Nf]
        grad = np.stack([Gd @ q[k].T for Gd in G], 1)  # [nq, 3(dir), Nf]
        rhs = np.zeros((Nf, len(wq)))
        if S.model == "acoustic":
            div = grad[:, 0, 1] + grad[:, 1, 2] + grad[:, 2, 3]
            rhs[0] = -S.kappa[k] * div
            for i in range(3):
                rhs[1 + i] = -grad[:, i, 0] / S.rho[k]
        else:
            dv = grad[:, :, 0:3]               # d_j v_i -> [nq, j, i]
            div = dv[:, 0, 0] + dv[:, 1, 1] + dv[:, 2, 2]
            for i in range(3):
                rhs[i] = sum(grad[:, j, SIG[i, j]] for j in range(3)) / S.rho[k]
                for j in range(i, 3):
                    t = S.mu[k] * (dv[:, j, i] + dv[:, i, j])
                    if i == j:
                        t = t + S.lam[k] * div
                    rhs[SIG[i, j]] = t
        b = (L * wq[:, None]).T @ rhs.T        # [Np, Nf]
        for skip in range(4):
            idx = [j for j in range(4) if j != skip]
            A_, B_, C_ = X[idx[0]], X[idx[1]], X[idx[2]]
            nrm = np.cross(B_ - A_, C_ - A_)
            area2 = np.linalg.norm(nrm)
            n = nrm / area2
            if np.dot(n, X[skip] - A_) > 0:
                n = -n
            xf = A_ + fp @ np.stack([B_ - A_, C_ - A_])
            wf = fw * area2
            Lf = B.ell(xf)
            qm = Lf @ q[k].T
            key = frozenset(int(tets[k, j]) for j in idx)
            other = [e for e in faces[key] if e != k]
            nn = np.broadcast_to(n, (len(wf), 3))
            if S.model == "acoustic":
                if other:
                    e = other[0]
                    qp = bases[e].ell(xf) @ q[e].T
                    ZP = S.Z[e]
                else:
                    qp = qm.copy()
                    vn = qm[:, 1:4] @ n
                    qp[:, 1:4] = qm[:, 1:4] - 2 * vn[:, None] * n
                    ZP = S.Z[k]
                dp, dvv = acoustic_penalty(qm[:, 0], qp[:, 0], qm[:, 1:4], qp[:, 1:4], nn,
                                           S.kappa[k], S.rho[k], S.c[k], ZP, S.flux)
                corr = np.concatenate([dp[:, None], dvv], 1)
            else:
                sm = qm[:, SIG.ravel()].reshape(-1, 3, 3)
                if other:
                    e = other[0]
                    qp = bases[e].ell(xf) @ q[e].T
                    sp = qp[:, SIG.ravel()].reshape(-1, 3, 3)
                    vp = qp[:, 0:3]
                    ZpP, ZsP = S.Zp[e], S.Zs[e]
                else:
                    sgn = -1.0 if S.bc == "free" else 1.0
                    vp, sp = -sgn * qm[:, 0:3], sgn * sm
                    ZpP, ZsP = S.Zp[k], S.Zs[k]
                Psig, pv = elastic_penalty(qm[:, 0:3], vp, sm, sp, nn, S.lam[k], S.mu[k],
                                           S.rho[k], ZpP, ZsP, S.flux)
                corr = np.zeros((len(wf), 9))
                corr[:, 0:3] = pv
                for i in range(3):
                    for j in range(i, 3):
                        corr[:, SIG[i, j]] = Psig[:, i, j]
            b += (Lf * wf[:, None]).T @ corr
        out[k] = np.linalg.solve(Mk, b).T
    return out


@pytest.mark.parametrize("model", ["acoustic", "elastic"])
@pytest.mark.parametrize("flux", ["upwind", "centered"])
@pytest.mark.parametrize("N", [1, 2, 3])
def test_rhs_matches_brute_force_weak_form(model, flux, N):
    verts, tets = W.six_tet_cube(0.1, seed=N + 7)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=N) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=N))
    S = Solver(model, N, verts, tets, coeffs, flux=flux)
    q = W.random_state(K, S.Nf, S.ref.Np, seed=N)
    r = S.rhs(q)
    rb = _brute_rhs(S, q)
    assert np.abs(r - rb).max() < 1e-10 * np.abs(rb).max()


def test_rhs_matches_brute_force_rigid_elastic():
    verts, tets = W.six_tet_cube(0.1, seed=3)
    coeffs = W.elastic_two_layer(verts, tets, seed=5)
    S = Solver("elastic", 2, verts, tets, coeffs, bc="rigid")
    q = W.random_state(6, 9, S.ref.Np, seed=1)
    rb = _brute_rhs(S, q)
    assert np.abs(S.rhs(q) - rb).max() < 1e-10 * np.abs(rb).max()
