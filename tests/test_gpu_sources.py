"""Several point sources per solve (dg_add_source, and served requests with
nsrc sources) against the FP64 oracle with the same sources, on every
strategy and the tensor-core mode; a served multi-source request equals the
same request run alone, bit for bit.

The sources: two at one point (so two terms land in the same element, one of
them in the step kernels and one in the kernel that adds the others) and one
elsewhere, each with its own amplitude history and direction.
"""

import numpy as np
import pytest

import workloads as W
from oracle.dg import Solver as OSolver, AB3Stepper

RHS_TOL = 1e-5
STEP_TOL = 1e-4


def groups(model):
    return ((0,), (1, 2, 3)) if model == "acoustic" else ((0, 1, 2), tuple(range(3, 9)))


def rel_l2(model, a, b):
    out = 0.0
    for g in groups(model):
        num = np.linalg.norm((np.asarray(a, np.float64)[:, g] - b[:, g]).ravel())
        out = max(out, num / np.linalg.norm(b[:, g].ravel()))
    return out


def _mesh(model, n, seed):
    verts, tets = W.kuhn_cube_mesh(n, 0.1, seed=seed)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=seed + 1) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=seed + 1))
    return verts, tets, coeffs


def _sources(nsteps, dt):
    t = np.arange(nsteps) * dt
    return [((0.31, 0.42, 0.27), W.ricker(t, f0=4.0, t0=0.05), (0.0, 0.0, 1.0)),
            ((0.31, 0.42, 0.27), -0.6 * W.ricker(t, f0=6.0, t0=0.04), (1.0, 0.0, 0.0)),
            ((0.70, 0.25, 0.60), 0.8 * W.ricker(t, f0=5.0, t0=0.03), (0.6, 0.0, 0.8))]


@pytest.fixture(scope="module")
def dg():
    import paper_1602_07997_gb300 as P
    P.lib()
    return P


@pytest.mark.gpu
@pytest.mark.parametrize("model,N,precision,strategy", [
    ("acoustic", 3, "fp32", "fused"), ("acoustic", 6, "fp32", "fused"), ("elastic", 2, "fp32", "fused"),
    ("elastic", 6, "fp32", "fused"), ("acoustic", 2, "fp32", "library"), ("elastic", 3, "fp32", "plain"),
    ("acoustic", 5, "bf16x6", "fused")])
def test_several_sources_60_steps(dg, model, N, precision, strategy):
    verts, tets, coeffs = _mesh(model, 3, 500 + N)
    o = OSolver(model, N, verts, tets, coeffs)
    dt = o.suggest_dt()
    srcs = _sources(60, dt)
    g = dg.Solver(verts, tets, coeffs, N, model, dt=dt, precision=precision, strategy=strategy)
    ks = [o.add_source(xs, amp, d) for xs, amp, d in srcs]
    assert ks[0] == ks[1] != ks[2]
    g.set_source(*srcs[0][:2], direction=srcs[0][2])
    for xs, amp, d in srcs[1:]:
        g.add_source(xs, amp, direction=d)
    q0 = np.zeros((o.K, o.Nf, o.ref.Np))
    g.set_state(q0.astype(np.float32))
    g.step(60)
    g.sync()
    st = AB3Stepper(o, q0, dt)
    st.step(60)
    assert np.abs(st.q).max() > 0
    err = rel_l2(model, g.get_state(), st.q)
    print(f"{model} N={N} {precision} {strategy} 3 sources, 60 steps rel-L2 {err:.2e}")
    assert err <= STEP_TOL, err
    g.close()


@pytest.mark.gpu
@pytest.mark.parametrize("model,N", [("acoustic", 2), ("elastic", 4)])
def test_several_sources_rhs(dg, model, N):
    """dg_rhs and dg_rhs_host_noalloc at step m include every source."""
    verts, tets, coeffs = _mesh(model, 3, 520 + N)
    o = OSolver(model, N, verts, tets, coeffs)
    srcs = _sources(20, o.suggest_dt())
    g = dg.Solver(verts, tets, coeffs, N, model, dt=o.suggest_dt())
    for i, (xs, amp, d) in enumerate(srcs):
        o.add_source(xs, 50.0 * amp, d)
        (g.set_source if i == 0 else g.add_source)(xs, 50.0 * amp, direction=d)
    q = W.random_state(o.K, o.Nf, o.ref.Np, seed=N).astype(np.float32)
    g.set_state(q, step=7)
    ro = o.rhs(q.astype(np.float64), step=7)
    assert rel_l2(model, g.rhs(), ro) <= RHS_TOL
    assert rel_l2(model, g.rhs_host_noalloc(), ro) <= RHS_TOL
    # removing the sources removes all of them
    g.set_source(None, None)
    o.srcs = []
    assert rel_l2(model, g.rhs(), o.rhs(q.astype(np.float64), step=7)) <= RHS_TOL
    g.close()


@pytest.mark.gpu
def test_served_several_sources_equal_solo(dg):
    """A request with three sources next to a one-source and a source-free
    request: each equals its solo run bit for bit."""
    N, steps = 3, 30
    runs = []
    for i, ns in enumerate((3, 1, 0)):
        verts, tets, coeffs = _mesh("acoustic", 3, 540 + i)
        dt = dg.suggest_dt(verts, tets, coeffs, N, "acoustic")
        srcs = _sources(steps, dt)[:ns]
        q0 = np.zeros((tets.shape[0], 4, (N + 1) * (N + 2) * (N + 3) // 6), np.float32)
        g = dg.Solver(verts, tets, coeffs, N, "acoustic", dt=dt)
        q0[:, 0] = W.gaussian_pulse(g.node_coords(), width=0.2)
        for j, (xs, amp, d) in enumerate(srcs):
            (g.set_source if j == 0 else g.add_source)(xs, amp, direction=d)
        g.set_state(q0)
        g.step(steps)
        g.sync()
        runs.append((verts, tets, coeffs, dt, q0, srcs, g.get_state()))
        g.close()
    srv = dg.Server()
    tickets = []
    for verts, tets, coeffs, dt, q0, srcs, _ in runs:
        kw = {}
        if srcs:
            kw = dict(source=np.array([s[0] for s in srcs]), amp=np.array([s[1] for s in srcs]),
                      direction=np.array([s[2] for s in srcs]))
        tickets.append(srv.submit(verts, tets, coeffs, N, q0=q0, dt=dt, nsteps=steps, **kw))
    for t, run in zip(tickets, runs):
        q, _ = srv.wait(t)
        assert np.array_equal(q, run[-1])
    srv.close()
