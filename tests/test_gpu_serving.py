"""Served solves: continuous batching through dg_submit / dg_poll.

Each result in a mixed batch must equal the same request run alone through
dg_step (same kernel variant, same per-element arithmetic: bit-for-bit), and
a served result must match the FP64 oracle like any other 100-step run.
"""

import time

import numpy as np
import pytest

import workloads as W
from oracle.dg import Solver as OSolver, AB3Stepper


@pytest.fixture(scope="module")
def P():
    import paper_1602_07997_gb300 as P
    P.lib()
    return P


def _req(i, N, n, steps, with_src=True):
    verts, tets = W.kuhn_cube_mesh(n, 0.1, seed=300 + i)
    K = tets.shape[0]
    coeffs = W.acoustic_coefficients(K, 1, 3, seed=400 + i)
    rng = np.random.default_rng(i)
    src = tuple(rng.uniform(0.2, 0.8, size=3))
    return dict(verts=verts, tets=tets, coeffs=coeffs, N=N, steps=steps, src=src if with_src else None)


def _alone(P, r, dt, amp):
    g = P.Solver(r["verts"], r["tets"], r["coeffs"], r["N"], "acoustic", dt=dt)
    q0 = np.zeros(g.shape, np.float32)
    q0[:, 0] = W.gaussian_pulse(g.node_coords(), width=0.2)
    if r["src"] is not None:
        g.set_source(r["src"], amp)
    g.set_state(q0)
    g.step(r["steps"])
    g.sync()
    out = g.get_state()
    g.close()
    return q0, out


@pytest.mark.gpu
def test_mixed_batch_equals_solo_runs(P):
    reqs = [_req(0, 3, 3, 40), _req(1, 2, 4, 25), _req(2, 3, 2, 70), _req(3, 1, 5, 55),
            _req(4, 2, 3, 10, with_src=False), _req(5, 4, 2, 33)]
    srv = P.Server()
    tickets, expect = [], []
    for r in reqs:
        dt = P.suggest_dt(r["verts"], r["tets"], r["coeffs"], r["N"], "acoustic")
        amp = W.ricker(np.arange(r["steps"]) * dt, f0=4.0, t0=0.05)
        q0, out = _alone(P, r, dt, amp)
        expect.append(out)
        tickets.append(srv.submit(r["verts"], r["tets"], r["coeffs"], r["N"], q0=q0, dt=dt,
                                  nsteps=r["steps"], source=r["src"], amp=amp))
    for t, e in zip(tickets, expect):
        q, lat = srv.wait(t)
        assert lat > 0
        assert np.array_equal(q, e)
    st = srv.stats()
    assert st["launches"] > 0 and st["queued"] == 0 and st["running"] == 0
    srv.close()


@pytest.mark.gpu
def test_served_result_matches_oracle(P):
    cfg = W.config1_acoustic_small()
    o = OSolver("acoustic", 2, cfg["verts"], cfg["tets"], cfg["coeffs"])
    dt = o.suggest_dt(cfg["cfl"])
    q0 = np.zeros((o.K, 4, o.ref.Np))
    q0[:, 0] = W.gaussian_pulse(o.mesh.x)
    srv = P.Server()
    t = srv.submit(cfg["verts"], cfg["tets"], cfg["coeffs"], 2, q0=q0.astype(np.float32), dt=dt, nsteps=100)
    q, _ = srv.wait(t)
    st = AB3Stepper(o, q0, dt)
    st.step(100)
    for g in ((0,), (1, 2, 3)):
        err = np.linalg.norm(q[:, g] - st.q[:, g]) / np.linalg.norm(st.q[:, g])
        assert err < 1e-4
    srv.close()


@pytest.mark.gpu
def test_admission_budget_and_refusal(P):
    small = [_req(10 + i, 2, 3, 20, with_src=False) for i in range(3)]
    # a budget that holds one of these solves at a time: they run one after another
    srv = P.Server(hbm_budget_bytes=4 << 20)
    ts = []
    for r in small:
        dt = P.suggest_dt(r["verts"], r["tets"], r["coeffs"], 2, "acoustic")
        ts.append(srv.submit(r["verts"], r["tets"], r["coeffs"], 2, dt=dt, nsteps=20))
    for t in ts:
        srv.wait(t)
    # a request larger than the whole budget is refused with DG_ENOMEM
    big = _req(20, 4, 6, 5, with_src=False)
    t = srv.submit(big["verts"], big["tets"], big["coeffs"], 4, dt=1e-4, nsteps=5)
    with pytest.raises(P.DGError) as e:
        srv.wait(t)
    assert e.value.code == -2
    srv.close()


@pytest.mark.gpu
def test_cancel_and_unknown_ticket(P):
    srv = P.Server(max_batch=1)
    r = _req(30, 3, 4, 100000, with_src=False)
    dt = P.suggest_dt(r["verts"], r["tets"], r["coeffs"], 3, "acoustic")
    t_long = srv.submit(r["verts"], r["tets"], r["coeffs"], 3, dt=dt, nsteps=100000)
    t_queued = srv.submit(r["verts"], r["tets"], r["coeffs"], 3, dt=dt, nsteps=10)
    srv.cancel(t_queued)           # still queued behind the long one (max_batch = 1)
    time.sleep(0.2)
    srv.cancel(t_long)             # running: retired at the next chunk boundary
    for t in (t_queued, t_long):
        with pytest.raises(P.DGError) as e:
            srv.wait(t)
        assert e.value.code == -7
    with pytest.raises(P.DGError) as e:
        srv.poll(12345)
    assert e.value.code == -8
    srv.close()


@pytest.mark.gpu
def test_requests_join_a_running_batch(P):
    """A short request submitted while a long one runs finishes first."""
    srv = P.Server()
    r = _req(40, 3, 4, 30000, with_src=False)
    dt = P.suggest_dt(r["verts"], r["tets"], r["coeffs"], 3, "acoustic")
    t_long = srv.submit(r["verts"], r["tets"], r["coeffs"], 3, dt=dt, nsteps=30000)
    time.sleep(0.05)
    s = _req(41, 3, 2, 10, with_src=False)
    dts = P.suggest_dt(s["verts"], s["tets"], s["coeffs"], 3, "acoustic")
    t_short = srv.submit(s["verts"], s["tets"], s["coeffs"], 3, dt=dts, nsteps=10)
    _, lat_short = srv.wait(t_short)
    assert srv.poll(t_long) is None    # the long solve is still running
    srv.wait(t_long)
    srv.close()


@pytest.mark.gpu
@pytest.mark.parametrize("N,which", [(5, 0), (5, -1), (8, 0), (8, -1)])
def test_batched_split_step_equals_solo_runs(P, N, which):
    """A server whose (model, N) variant is the split step (batched front half +
    batched operator GEMM) gives every request the bits of its solo run.  The
    first and the last split variant of a degree: at N = 5 one CTA per GEMM
    tile and the warp-specialised persistent GEMM walking the tiles of every
    solve, at N = 8 the other way round."""
    probe = _req(50, N, 2, 1, with_src=False)
    g = P.Solver(probe["verts"], probe["tets"], probe["coeffs"], N, "acoustic", dt=1e-3)
    split = [i for i in range(g.kernel_info()["variants"]) if (g.set_variant(i) or g.kernel_info()["split"])]
    assert split, "no split variant compiled for this degree"
    g.set_variant(split[which])  # recorded for later handles and servers of the process
    g.close()
    try:
        reqs = [_req(51, N, 3, 30), _req(52, N, 2, 45), _req(53, N, 4, 12, with_src=False)]
        srv = P.Server()
        tickets, expect = [], []
        for r in reqs:
            dt = P.suggest_dt(r["verts"], r["tets"], r["coeffs"], N, "acoustic")
            amp = W.ricker(np.arange(r["steps"]) * dt, f0=4.0, t0=0.05)
            q0, out = _alone(P, r, dt, amp)
            expect.append(out)
            tickets.append(srv.submit(r["verts"], r["tets"], r["coeffs"], N, q0=q0, dt=dt,
                                      nsteps=r["steps"], source=r["src"], amp=amp))
        for t, e in zip(tickets, expect):
            q, _ = srv.wait(t)
            assert np.array_equal(q, e)
        srv.close()
    finally:
        g = P.Solver(probe["verts"], probe["tets"], probe["coeffs"], N, "acoustic", dt=1e-3)
        g.set_variant(0)
        g.close()
