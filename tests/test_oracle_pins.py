"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (tests/golden), closed forms (exact differentiation, volumes,
areas, divergence theorem, exact solutions), invariants (semi-discrete
energy), the 1-D Riemann problem, and the order of AB3.
"""

import math
import os

import numpy as np
import pytest

import workloads as W
from oracle.refelem import (RefElement, warp_blend_nodes, tri_quadrature, num_nodes,
                            num_face_nodes, FACE_VERTS)
from oracle.dg import Solver, AB3Stepper, acoustic_penalty, elastic_penalty, AB3

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(x) for x in line.split()])
    return np.array(rows)


def _small_mesh(n=2, seed=11):
    return W.kuhn_cube_mesh(n, 0.1, seed=seed)


# ---------------------------------------------------------------- paper values
def test_paper_table_sizes():
    """Np and 3Np for N = 1..8 as printed in the paper's padding table."""
    tab = _read("paper_sizes.txt")
    for N, Np, _, Np3, _ in tab:
        R = RefElement(int(N))
        assert R.Np == Np == num_nodes(N)
        assert 3 * R.Np == Np3
        assert R.Nfp == num_face_nodes(N) == (N + 1) * (N + 2) // 2
        assert R.Dr.shape == (Np, Np) and R.LIFT.shape == (Np, 4 * R.Nfp)


def test_ab3_coefficients_match_paper():
    a = _read("ab3_coefficients.txt")[0] / 12.0
    assert np.allclose(AB3, a, rtol=0, atol=1e-16)


# ---------------------------------------------------------------- node set
@pytest.mark.parametrize("N", range(1, 9))
def test_nodes_on_faces_and_symmetric(N):
    X = warp_blend_nodes(N)
    R = RefElement(N)
    # every face carries exactly Nfp nodes, edges N+1, vertices are nodes
    assert R.Fmask.shape == (4, num_face_nodes(N))
    for v in ([-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]):
        assert np.min(np.linalg.norm(X - np.array(v), axis=1)) < 1e-14
    # the node set is invariant under the vertex permutation v2<->v3 (r<->s)
    Y = X[:, [1, 0, 2]]
    d = np.linalg.norm(X[:, None, :] - Y[None, :, :], axis=2).min(axis=1)
    assert d.max() < 1e-13
    # edge nodes are the GLL points along the edge
    from oracle.refelem import gll_points
    e = np.sort(X[(np.abs(X[:, 1] + 1) < 1e-12) & (np.abs(X[:, 2] + 1) < 1e-12), 0])
    assert np.allclose(e, gll_points(N), atol=1e-13)


# ---------------------------------------------------------------- operators
@pytest.mark.parametrize("N", range(1, 9))
def test_exact_differentiation_physical(N):
    """Physical D_x,y,z on jittered tets differentiate every monomial of degree <= N exactly."""
    verts, tets = _small_mesh(1, seed=N)
    S = Solver("acoustic", N, verts, tets, np.ones((tets.shape[0], 2)))
    m = S.mesh
    x = m.x  # [K, Np, 3]
    err = 0.0
    for a in range(N + 1):
        for b in range(N + 1 - a):
            for c in range(N + 1 - a - b):
                f = x[..., 0] ** a * x[..., 1] ** b * x[..., 2] ** c
                grad = S._phys_grad(f[:, None, :])[:, 0]       # [K, 3, Np]
                ex = [a * x[..., 0] ** max(a - 1, 0) * x[..., 1] ** b * x[..., 2] ** c,
                      b * x[..., 0] ** a * x[..., 1] ** max(b - 1, 0) * x[..., 2] ** c,
                      c * x[..., 0] ** a * x[..., 1] ** b * x[..., 2] ** max(c - 1, 0)]
                for i in range(3):
                    err = max(err, np.max(np.abs(grad[:, i] - ex[i])))
    assert err < 1e-10


@pytest.mark.parametrize("N", range(1, 9))
def test_mass_and_face_mass_measures(N):
    R = RefElement(N)
    assert abs(R.M.sum() - 4.0 / 3.0) < 1e-13          # reference volume
    for f in range(4):
        assert abs(R.E[f].sum() - 2.0) < 1e-13         # area-2 face parametrisation
        # E_f vanishes outside the face nodes
        other = np.setdiff1d(np.arange(R.Np), R.Fmask[f])
        assert np.abs(R.E[f][other]).max() < 1e-12
    # M LIFT_f = E_f restricted to face columns
    Nfp = R.Nfp
    for f in range(4):
        assert np.allclose(R.M @ R.LIFT[:, f * Nfp:(f + 1) * Nfp], R.E[f][:, R.Fmask[f]], atol=1e-12)


def test_mesh_volume_and_boundary_area():
    verts, tets = _small_mesh(3)
    S = Solver("acoustic", 2, verts, tets, np.ones((tets.shape[0], 2)))
    m = S.mesh
    assert abs(np.sum(m.J) * 4.0 / 3.0 - 1.0) < 1e-13      # unit cube volume
    assert abs(np.sum(2.0 * m.sJ[m.boundary]) - 6.0) < 1e-12  # cube surface
    # every face of every tet: area vectors of the 4 faces sum to zero
    av = (2.0 * m.sJ)[:, :, None] * m.n
    assert np.abs(av.sum(axis=1)).max() < 1e-13
    # interior faces: opposite normals, equal areas
    kk, ff = np.nonzero(~m.boundary)
    k2, f2 = m.EToE[kk, ff], m.EToF[kk, ff]
    assert np.allclose(m.n[kk, ff], -m.n[k2, f2], atol=1e-13)
    assert np.allclose(m.sJ[kk, ff], m.sJ[k2, f2], rtol=1e-13)


@pytest.mark.parametrize("N", [1, 3, 5, 8])
def test_divergence_theorem_by_face_quadrature(N):
    """int_T d q/dx_i = sum_f int_f q n_i dA, surface integral by independent
    quadrature on each physical face (pins n, sJ, D and M together)."""
    verts, tets = _small_mesh(1, seed=3)
    S = Solver("acoustic", N, verts, tets, np.ones((tets.shape[0], 2)))
    m, R = S.mesh, S.ref
    rng = np.random.default_rng(N)
    q = rng.uniform(-1, 1, size=(m.K, R.Np))
    grad = S._phys_grad(q[:, None, :])[:, 0]               # [K, 3, Np]
    vol = m.J[:, None] * np.einsum("kin,nm,m->ki", grad, R.M, np.ones(R.Np))
    up, uw = tri_quadrature(N + 3)
    surf = np.zeros((m.K, 3))
    for k in range(m.K):
        for f in range(4):
            A, B, C = (verts[tets[k, i]] for i in FACE_VERTS[f])
            area = 0.5 * np.linalg.norm(np.cross(B - A, C - A))
            # reference-tet coordinates of the face quadrature points
            xs = A[None] + np.outer((1 + up[:, 0]) / 2, B - A) + np.outer((1 + up[:, 1]) / 2, C - A)
            rst = np.linalg.solve(m.A[k], (xs - verts[tets[k, 0]]).T).T - 1.0
            vals = R.lag.eval(rst) @ q[k]
            surf[k] += (area / 2.0) * np.sum(uw * vals) * m.n[k, f]
    assert np.abs(vol - surf).max() < 1e-11 * max(1.0, np.abs(vol).max())


# ---------------------------------------------------------------- RHS
@pytest.mark.parametrize("model", ["acoustic", "elastic"])
def test_free_stream_heterogeneous(model):
    verts, tets = _small_mesh(2)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=1) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=1))
    for N in (1, 4):
        S = Solver(model, N, verts, tets, coeffs)
        q = np.zeros((K, S.Nf, S.ref.Np))
        q[:, 0] = 0.37        # acoustic: constant p; elastic: constant v_x
        assert np.abs(S.rhs(q)).max() < 1e-12


@pytest.mark.parametrize("N", [1, 2, 4])
def test_linear_pressure_homogeneous(N):
    """p = a.x, v = 0, homogeneous medium: r_v = -a/rho, r_p = 0."""
    verts, tets = _small_mesh(2)
    K = tets.shape[0]
    rho, c = 1.7, 1.3
    S = Solver("acoustic", N, verts, tets, np.tile([rho, c], (K, 1)))
    a = np.array([0.3, -1.1, 0.6])
    q = np.zeros((K, 4, S.ref.Np))
    q[:, 0] = S.mesh.x @ a
    r = S.rhs(q)
    assert np.abs(r[:, 0]).max() < 1e-11
    for i in range(3):
        assert np.abs(r[:, 1 + i] + a[i] / rho).max() < 1e-11


@pytest.mark.parametrize("model", ["acoustic", "elastic"])
@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_energy_identity(model, N):
    """Centred flux + mirror walls: dE_h/dt = 0; upwind: dE_h/dt <= 0."""
    verts, tets = _small_mesh(2, seed=N)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=N) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=N))
    Sc = Solver(model, N, verts, tets, coeffs, flux="centered")
    Su = Solver(model, N, verts, tets, coeffs, flux="upwind")
    for seed in range(3):
        q = W.random_state(K, Sc.Nf, Sc.ref.Np, seed=seed)
        scale = Sc.energy(q) * N * N * 10
        assert abs(Sc.energy_rate(q, Sc.rhs(q))) < 1e-12 * scale
        assert Su.energy_rate(q, Su.rhs(q)) < -1e-6 * scale


@pytest.mark.parametrize("model", ["acoustic", "elastic"])
def test_energy_identity_rigid_and_free(model):
    verts, tets = _small_mesh(2)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=3) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=3))
    for bc in (("rigid",) if model == "acoustic" else ("rigid", "free")):
        S = Solver(model, 2, verts, tets, coeffs, flux="centered", bc=bc)
        q = W.random_state(K, S.Nf, S.ref.Np, seed=9)
        assert abs(S.energy_rate(q, S.rhs(q))) < 1e-12 * S.energy(q) * 100


def test_acoustic_penalty_solves_riemann_problem():
    """Star states recovered from the penalty satisfy both characteristic
    relations p* + Z^- v* = p^- + Z^- v^-, p* - Z^+ v* = p^+ - Z^+ v^+."""
    rng = np.random.default_rng(0)
    m = 200
    n = rng.normal(size=(m, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    pM, pP = rng.normal(size=m), rng.normal(size=m)
    vM, vP = rng.normal(size=(m, 3)), rng.normal(size=(m, 3))
    rhoM, cM = rng.uniform(1, 3, m), rng.uniform(1, 3, m)
    rhoP, cP = rng.uniform(1, 3, m), rng.uniform(1, 3, m)
    ZM, ZP = rhoM * cM, rhoP * cP
    dp, dv = acoustic_penalty(pM, pP, vM, vP, n, rhoM * cM * cM, rhoM, cM, ZP)
    # dp = kappa^- (v_n^- - v_n*),  dv = (p^- - p*) n / rho^-
    vnM, vnP = np.sum(vM * n, 1), np.sum(vP * n, 1)
    vs = vnM - dp / (rhoM * cM * cM)
    ps = pM - rhoM * np.sum(dv * n, 1)
    assert np.allclose(np.cross(dv, n), 0, atol=1e-13)
    assert np.allclose(ps + ZM * vs, pM + ZM * vnM, atol=1e-12)
    assert np.allclose(ps - ZP * vs, pP - ZP * vnP, atol=1e-12)
    # centred flux: star state = average
    dp, dv = acoustic_penalty(pM, pP, vM, vP, n, rhoM * cM * cM, rhoM, cM, ZP, "centered")
    assert np.allclose(vnM - dp / (rhoM * cM * cM), 0.5 * (vnM + vnP), atol=1e-13)
    assert np.allclose(pM - rhoM * np.sum(dv * n, 1), 0.5 * (pM + pP), atol=1e-13)


def test_elastic_penalty_solves_riemann_problem():
    """P and S characteristic relations across the interface, both sides."""
    rng = np.random.default_rng(1)
    m = 200
    n = rng.normal(size=(m, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    vM, vP = rng.normal(size=(m, 3)), rng.normal(size=(m, 3))
    a, b = rng.normal(size=(m, 3, 3)), rng.normal(size=(m, 3, 3))
    sM, sP = a + np.swapaxes(a, 1, 2), b + np.swapaxes(b, 1, 2)
    lamM, muM, rhoM = (rng.uniform(1, 3, m) for _ in range(3))
    lamP, muP, rhoP = (rng.uniform(1, 3, m) for _ in range(3))
    ZpM, ZsM = np.sqrt((lamM + 2 * muM) * rhoM), np.sqrt(muM * rhoM)
    ZpP, ZsP = np.sqrt((lamP + 2 * muP) * rhoP), np.sqrt(muP * rhoP)
    Psig, pv = elastic_penalty(vM, vP, sM, sP, n, lamM, muM, rhoM, ZpP, ZsP)
    # recover dv = v* - v^- from P_sigma = C^-: sym(n (x) dv), and sigma* n from p_v
    Pn = np.einsum("mij,mj->mi", Psig, n)
    dvn = np.sum(Pn * n, 1) / (lamM + 2 * muM)
    dvt = (Pn - np.sum(Pn * n, 1)[:, None] * n) / muM[:, None]
    dv = dvn[:, None] * n + dvt
    # P_sigma must be exactly C^-: sym(n (x) dv)
    sym = 0.5 * (n[:, :, None] * dv[:, None, :] + dv[:, :, None] * n[:, None, :])
    C = lamM[:, None, None] * np.sum(n * dv, 1)[:, None, None] * np.eye(3) + 2 * muM[:, None, None] * sym
    assert np.allclose(Psig, C, atol=1e-12)
    vs = vM + dv
    tM = np.einsum("mij,mj->mi", sM, n) + rhoM[:, None] * pv   # sigma* n
    tP = tM
    tnM, tnP0 = np.einsum("mij,mj->mi", sM, n), np.einsum("mij,mj->mi", sP, n)

    def split(x):
        xn = np.sum(x * n, 1)
        return xn, x - xn[:, None] * n

    (sn_s, st_s), (vn_s, vt_s) = split(tM), split(vs)
    (snM, stM), (vnM, vtM) = split(tnM), split(vM)
    (snP, stP), (vnP, vtP) = split(tnP0), split(vP)
    assert np.allclose(sn_s - ZpM * vn_s, snM - ZpM * vnM, atol=1e-11)
    assert np.allclose(sn_s + ZpP * vn_s, snP + ZpP * vnP, atol=1e-11)
    assert np.allclose(st_s - ZsM[:, None] * vt_s, stM - ZsM[:, None] * vtM, atol=1e-11)
    assert np.allclose(st_s + ZsP[:, None] * vt_s, stP + ZsP[:, None] * vtP, atol=1e-11)
    del tP


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_rhs_independent_of_node_set(N):
    """The RHS polynomial does not depend on the nodes (equispaced vs warp & blend)."""
    verts, tets = _small_mesh(2, seed=4)
    K = tets.shape[0]
    coeffs = W.acoustic_coefficients(K, 1, 3, seed=2)
    Ra = RefElement(N)
    Rb = RefElement(N, nodes=warp_blend_nodes(N, equispaced=True))
    Sa = Solver("acoustic", N, verts, tets, coeffs, ref=Ra)
    Sb = Solver("acoustic", N, verts, tets, coeffs, ref=Rb)
    # one random polynomial per element and field, evaluated at each node set
    rng = np.random.default_rng(N)
    coef = rng.uniform(-1, 1, size=(K, 4, Ra.Np))       # in the Lagrange basis of set a

    def at(R_nodes):
        return np.einsum("nm,kfm->kfn", Ra.lag.eval(R_nodes), coef)

    qa, qb = at(Ra.nodes), at(Rb.nodes)
    ra, rb = Sa.rhs(qa), Sb.rhs(qb)
    pts = np.array([[-0.5, -0.4, -0.3], [0.1, -0.8, -0.6], [-0.9, 0.2, -0.5], [-0.2, -0.2, -0.9]])
    va = np.einsum("pn,kfn->kfp", Ra.lag.eval(pts), ra)
    vb = np.einsum("pn,kfn->kfp", Rb.lag.eval(pts), rb)
    assert np.abs(va - vb).max() < 1e-10 * np.abs(va).max()


def test_source_is_point_evaluation():
    """b = M_k^{-1} l(x_s): for any nodal u, b^T (J_k M) u = u(x_s)."""
    verts, tets = _small_mesh(2)
    S = Solver("acoustic", 3, verts, tets, np.ones((tets.shape[0], 2)))
    xs = np.array([0.41, 0.57, 0.33])
    k = S.set_source(xs, amp=[1.0])
    _, b, _, _ = S.srcs[0]
    rng = np.random.default_rng(0)
    # u = a polynomial of degree 3 in physical coordinates
    cfs = rng.normal(size=4)
    x = S.mesh.x[k]
    u = cfs[0] + cfs[1] * x[:, 0] ** 3 + cfs[2] * x[:, 1] * x[:, 2] + cfs[3] * x[:, 0] * x[:, 1] * x[:, 2]
    ex = cfs[0] + cfs[1] * xs[0] ** 3 + cfs[2] * xs[1] * xs[2] + cfs[3] * xs[0] * xs[1] * xs[2]
    assert abs(b @ (S.mesh.J[k] * S.ref.M) @ u - ex) < 1e-12
    # and the tet really contains x_s
    lam = np.linalg.solve(np.vstack([verts[tets[k]].T, np.ones(4)]), np.append(xs, 1.0))
    assert lam.min() > 0


@pytest.mark.parametrize("model,N", [("acoustic", 2), ("elastic", 1)])
def test_sources_superpose(model, N):
    """The scheme is linear in the forcing: from a zero state, sources A and B
    together give the sum of the runs with A alone and with B alone; two
    sources at one point act as one source with the summed amplitudes."""
    verts, tets = _small_mesh(2)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=5) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=5))
    xa, xb = np.array([0.31, 0.42, 0.27]), np.array([0.7, 0.25, 0.6])
    t = np.arange(12)
    amp_a, amp_b = np.sin(0.7 * t + 0.2), np.cos(0.3 * t) * (t < 9)
    dirb = (0.6, 0.0, 0.8)

    def run(srcs):
        S = Solver(model, N, verts, tets, coeffs)
        for xs, amp, d in srcs:
            S.add_source(xs, amp, d)
        st = AB3Stepper(S, np.zeros((K, S.Nf, S.ref.Np)), S.suggest_dt())
        st.step(12)
        return st.q

    qa = run([(xa, amp_a, (0, 0, 1))])
    qb = run([(xb, amp_b, dirb)])
    qab = run([(xa, amp_a, (0, 0, 1)), (xb, amp_b, dirb)])
    assert np.abs(qa).max() > 0 and np.abs(qb).max() > 0
    assert np.abs(qab - (qa + qb)).max() <= 1e-12 * np.abs(qab).max()
    q2 = run([(xa, amp_a, (0, 0, 1)), (xa, 2.5 * amp_a, (0, 0, 1))])
    assert np.abs(q2 - 3.5 * qa).max() <= 1e-12 * np.abs(q2).max()


# ---------------------------------------------------------------- time stepping
def test_ab3_third_order_and_polynomial_exactness():
    """AB3 with exact history: exact for y' = quadratic in t; third order for y' = l y."""
    # y' = f(t) = 1 + t + t^2 with history from the exact f: exact integration
    class Lin:
        def __init__(self):
            self.t = 0.0
    dt = 0.1
    f = lambda t: 1.0 + t + t * t
    y, t = 0.0, 0.0
    hist = [f(-dt), f(-2 * dt)]
    for m in range(10):
        r = f(t)
        y = y + dt * (AB3[0] * r + AB3[1] * hist[0] + AB3[2] * hist[1])
        hist = [r, hist[0]]
        t += dt
    assert abs(y - (t + t * t / 2 + t ** 3 / 3)) < 1e-12
    # y' = -y, order 3
    errs = []
    for nst in (40, 80, 160):
        dt = 1.0 / nst
        y = 1.0
        hist = [-math.exp(dt), -math.exp(2 * dt)]
        for m in range(nst):
            r = -y
            y = y + dt * (AB3[0] * r + AB3[1] * hist[0] + AB3[2] * hist[1])
            hist = [r, hist[0]]
        errs.append(abs(y - math.exp(-1.0)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.8)


@pytest.mark.slow
def test_upwind_energy_monotone_config1():
    """Config 1 (384 tets, N=2), upwind, AB3 at CFL dt: E_h nonincreasing
    from the second step on (the bootstrap forward-Euler step is not
    energy-stable and may raise E_h by O(dt^2))."""
    cfg = W.config1_acoustic_small()
    S = Solver("acoustic", 2, cfg["verts"], cfg["tets"], cfg["coeffs"])
    q0 = np.zeros((S.K, 4, S.ref.Np))
    q0[:, 0] = W.gaussian_pulse(S.mesh.x)
    dt = S.suggest_dt(cfg["cfl"])
    st = AB3Stepper(S, q0, dt)
    E = [S.energy(st.q)]
    for _ in range(300):
        st.step()
        E.append(S.energy(st.q))
    E = np.array(E)
    assert np.all(np.diff(E[1:]) <= 1e-14 * E[0])
    assert E[1] - E[0] < 1e-2 * E[0]
    assert E[-1] < E[0]


@pytest.mark.slow
@pytest.mark.parametrize("model,N", [("acoustic", 1), ("acoustic", 4), ("acoustic", 8),
                                     ("elastic", 1), ("elastic", 5)])
def test_suggested_dt_is_ab3_stable(model, N):
    """At the suggested dt (cfl 0.4) upwind + AB3 never increases E_h after
    the bootstrap steps, from rough random data (all modes excited)."""
    verts, tets = _small_mesh(2, seed=N)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=N) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=N))
    S = Solver(model, N, verts, tets, coeffs)
    q0 = W.random_state(K, S.Nf, S.ref.Np, seed=5)
    st = AB3Stepper(S, q0, S.suggest_dt())
    E = [S.energy(st.q)]
    for _ in range(150):
        st.step()
        E.append(S.energy(st.q))
    E = np.array(E)
    assert np.all(np.diff(E[2:]) <= 1e-13 * E[0]), np.max(np.diff(E[2:]))


@pytest.mark.parametrize("N", [1, 3, 6])
def test_point_values_reproduce_polynomials(N):
    """Point evaluation of the nodal polynomial (receivers) is exact for fields
    that are polynomials of degree <= N, at interior points and at points on
    faces shared by two elements."""
    verts, tets = W.kuhn_cube_mesh(2, 0.1, seed=11)
    K = tets.shape[0]
    S = Solver("acoustic", N, verts, tets, np.ones((K, 2)))
    rng = np.random.default_rng(N)
    # random polynomial of total degree N per field, evaluated at the nodes
    expo = [(a, b, c) for a in range(N + 1) for b in range(N + 1 - a) for c in range(N + 1 - a - b)]
    coef = rng.uniform(-1, 1, size=(S.Nf, len(expo)))

    def poly(x):
        x = np.atleast_2d(x)
        mon = np.stack([x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c for a, b, c in expo], axis=1)
        return mon @ coef.T

    X = S.mesh.x.reshape(-1, 3)
    q = poly(X).reshape(K, S.ref.Np, S.Nf).transpose(0, 2, 1)
    pts = rng.uniform(0.05, 0.95, size=(20, 3))
    # a point on an interior face: the centroid of a face shared by two tets
    k0 = int(np.argmax(S.mesh.EToE[:, 0] != np.arange(K)))
    fv = verts[tets[k0][[0, 1, 2]]]
    pts = np.vstack([pts, fv.mean(axis=0)])
    assert np.abs(S.point_values(q, pts) - poly(pts)).max() < 1e-10


@pytest.mark.parametrize("model", ["acoustic", "elastic"])
def test_rhs_on_element_subset_equals_full_rows(model):
    """The oracle's RHS restricted to sampled elements (used for the largest
    meshes) is exactly the corresponding rows of the full RHS, source included."""
    verts, tets = W.kuhn_cube_mesh(3, 0.1, seed=17)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=18) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=18))
    S = Solver(model, 3, verts, tets, coeffs)
    ks = S.set_source((0.47, 0.52, 0.44), np.array([0.7, -0.3]))
    q = W.random_state(K, S.Nf, S.ref.Np, seed=4)
    full = S.rhs(q, step=0)
    sample = np.array(sorted({0, 5, K - 1, ks} | set(np.random.default_rng(1).integers(0, K, 20).tolist())))
    assert np.array_equal(S.rhs(q, step=0, elems=sample), full[sample])
