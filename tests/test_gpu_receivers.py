"""Receivers: the library's recorded traces against the oracle's point values
of its own AB3 solution (the nodal polynomial evaluated at each receiver after
every step), same bar as the states: rel-L2 <= 1e-4 over 40 steps."""

import numpy as np
import pytest

import workloads as W
from oracle.dg import Solver as OSolver, AB3Stepper

STEP_TOL = 1e-4


@pytest.fixture(scope="module")
def dg():
    import paper_1602_07997_gb300 as P
    P.lib()
    return P


@pytest.mark.gpu
@pytest.mark.parametrize("model,N", [("acoustic", 3), ("elastic", 2), ("acoustic", 6)])
def test_receiver_traces_match_oracle(dg, model, N):
    verts, tets = W.kuhn_cube_mesh(3, 0.1, seed=300 + N)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=301) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=301))
    o = OSolver(model, N, verts, tets, coeffs)
    dt = o.suggest_dt()
    steps = 40
    amp = W.ricker(np.arange(steps) * dt, f0=4.0, t0=0.05)
    xs = (0.43, 0.51, 0.48)
    o.set_source(xs, amp)
    rec = np.random.default_rng(N).uniform(0.1, 0.9, size=(7, 3))
    q0 = np.zeros((o.K, o.Nf, o.ref.Np))
    q0[:, 0] = W.gaussian_pulse(o.mesh.x, width=0.3)
    g = dg.Solver(verts, tets, coeffs, N, model, dt=dt)
    g.set_source(xs, amp)
    g.set_receivers(rec)
    g.set_state(q0.astype(np.float32))
    g.step(15)
    g.step(steps - 15)  # the trace buffer grows across calls
    tr = g.traces()
    assert tr.shape == (steps, 7, o.Nf)
    st = AB3Stepper(o, q0, dt)
    ref = []
    for _ in range(steps):
        st.step(1)
        ref.append(o.point_values(st.q, rec))
    ref = np.array(ref)
    err = np.linalg.norm(tr - ref) / np.linalg.norm(ref)
    assert err <= STEP_TOL, err
    g.set_receivers(np.zeros((0, 3)))  # removes them
    g.step(1)
    assert g.traces().shape[0] == 0
    with pytest.raises(dg.DGError) as e:
        g.set_receivers([[2.0, 0.5, 0.5]])  # outside the unit cube
    assert e.value.code == -1
    g.close()
