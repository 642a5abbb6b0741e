"""GPU parity: libdg (FP32, CUDA) against the FP64 oracle on the same seeded inputs.

Bar (relative L2 per field group, max over groups; acoustic {p},{v},
elastic {v},{sigma}): <= 1e-5 after one RHS evaluation and <= 1e-4 after 100
AB3 steps.  Meshes span several CTA blocks plus a ragged tail for every N.
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
        den = np.linalg.norm(b[:, g].ravel())
        out = max(out, num / den)
    return out


def _mesh(model, n, seed):
    verts, tets = W.kuhn_cube_mesh(n, 0.1, seed=seed)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=seed + 1) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=seed + 1))
    return verts, tets, coeffs


@pytest.fixture(scope="module")
def dg():
    import paper_1602_07997_gb300 as P
    P.lib()
    return P


@pytest.mark.gpu
@pytest.mark.parametrize("model", ["acoustic", "elastic"])
@pytest.mark.parametrize("N", range(1, 9))
def test_rhs_parity_random_state(dg, model, N):
    n = 5 if N <= 2 else (4 if N <= 5 else 3)
    verts, tets, coeffs = _mesh(model, n, 10 + N)
    o = OSolver(model, N, verts, tets, coeffs)
    g = dg.Solver(verts, tets, coeffs, N, model)
    assert np.abs(g.node_coords() - o.mesh.x).max() < 1e-12
    q = W.random_state(o.K, o.Nf, o.ref.Np, seed=N).astype(np.float32)
    g.set_state(q)
    r = g.rhs()
    ro = o.rhs(q.astype(np.float64))
    err = rel_l2(model, r, ro)
    assert err <= RHS_TOL, err


@pytest.mark.gpu
@pytest.mark.parametrize("model,N,flux,bc", [("acoustic", 3, "centered", None),
                                              ("acoustic", 1, "centered", None),
                                              ("elastic", 3, "centered", None),
                                              ("elastic", 2, "upwind", "rigid"),
                                              ("elastic", 4, "centered", "rigid")])
def test_rhs_parity_flux_and_bc_variants(dg, model, N, flux, bc):
    verts, tets, coeffs = _mesh(model, 3, 40 + N)
    o = OSolver(model, N, verts, tets, coeffs, flux=flux, bc=bc)
    g = dg.Solver(verts, tets, coeffs, N, model, flux=flux, bc=bc)
    q = W.random_state(o.K, o.Nf, o.ref.Np, seed=3).astype(np.float32)
    g.set_state(q)
    assert rel_l2(model, g.rhs(), o.rhs(q.astype(np.float64))) <= RHS_TOL


@pytest.mark.gpu
def test_config1_100_steps(dg):
    """Config 1: 384 tets, N=2, Gaussian pulse, rigid walls, upwind, 100 AB3 steps."""
    cfg = W.config1_acoustic_small()
    o = OSolver("acoustic", 2, cfg["verts"], cfg["tets"], cfg["coeffs"])
    dt = o.suggest_dt(cfg["cfl"])
    q0 = np.zeros((o.K, 4, o.ref.Np))
    q0[:, 0] = W.gaussian_pulse(o.mesh.x)
    g = dg.Solver(cfg["verts"], cfg["tets"], cfg["coeffs"], 2, "acoustic", dt=dt)
    assert abs(dg.suggest_dt(cfg["verts"], cfg["tets"], cfg["coeffs"], 2, "acoustic", cfg["cfl"]) - dt) < 1e-15
    g.set_state(q0.astype(np.float32))
    g.step(100)
    g.sync()
    st = AB3Stepper(o, q0, dt)
    st.step(100)
    err = rel_l2("acoustic", g.get_state(), st.q)
    assert err <= STEP_TOL, err


@pytest.mark.gpu
@pytest.mark.parametrize("model", ["acoustic", "elastic"])
@pytest.mark.parametrize("N", range(1, 9))
def test_100_steps_with_source(dg, model, N):
    """100 AB3 steps from a Gaussian / quiescent state with a Ricker point
    source, every degree of both models in its default kernel variant (fused
    at low N, the split step above)."""
    n = 3 if N <= 4 else 2
    verts, tets, coeffs = _mesh(model, n, 70 + N)
    o = OSolver(model, N, verts, tets, coeffs)
    dt = o.suggest_dt(0.4)
    amp = W.ricker(np.arange(100) * dt, f0=4.0, t0=0.05) * 10.0
    xs = (0.4321, 0.5678, 0.4876)
    ko = o.set_source(xs, amp, direction=(0.3, -0.2, 0.9))
    q0 = np.zeros((o.K, o.Nf, o.ref.Np))
    q0[:, 0] = W.gaussian_pulse(o.mesh.x, width=0.3)
    g = dg.Solver(verts, tets, coeffs, N, model, dt=dt)
    g.set_source(xs, amp, direction=(0.3, -0.2, 0.9))
    g.set_state(q0.astype(np.float32))
    g.step(100)
    g.sync()
    st = AB3Stepper(o, q0, dt)
    st.step(100)
    err = rel_l2(model, g.get_state(), st.q)
    assert err <= STEP_TOL, (err, ko)


@pytest.mark.gpu
def test_rhs_device_buffers_and_history(dg):
    """Device (torch) buffers give the same results as host buffers; a given
    AB3 history is used; get_state returns what set_state put."""
    import torch
    model, N = "acoustic", 3
    verts, tets, coeffs = _mesh(model, 3, 5)
    g = dg.Solver(verts, tets, coeffs, N, model, dt=1e-3)
    rng = np.random.default_rng(0)
    q, r1, r2 = (rng.uniform(-1, 1, size=g.shape).astype(np.float32) for _ in range(3))
    g.set_state(q, r1, r2, step=7)
    qh = g.get_state()
    assert np.array_equal(qh, q) and g.step_index == 7 and g.history == 2
    rh = g.rhs()
    rd = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    g.rhs(rd)
    torch.cuda.synchronize()
    assert np.array_equal(rd.cpu().numpy(), rh)
    # one AB3 step with the supplied history
    g.step(1)
    q1 = g.get_state()
    expect = q + 1e-3 * (23 * rh + -16 * r1 + 5 * r2) / 12.0
    assert np.abs(q1 - expect).max() <= 1e-6 * np.abs(expect).max()
    # device-side set_state
    qd = torch.from_numpy(q).cuda()
    g.set_state(qd)
    assert np.array_equal(g.get_state(), q)


@pytest.mark.gpu
def test_setup_rejects_bad_meshes(dg):
    verts, tets = W.kuhn_cube_mesh(2, 0.1, seed=1)
    K = tets.shape[0]
    coeffs = np.ones((K, 2))
    bad = tets.copy()
    bad[0, [2, 3]] = bad[0, [3, 2]]        # inverted
    with pytest.raises(dg.DGError) as e:
        dg.Solver(verts, bad, coeffs, 2)
    assert e.value.code == -1
    dup = np.concatenate([tets, tets[:1]])  # face shared by 3 tets
    with pytest.raises(dg.DGError):
        dg.Solver(verts, dup, np.ones((K + 1, 2)), 2)
    with pytest.raises(dg.DGError):
        dg.Solver(verts, tets, coeffs, 9)


@pytest.mark.gpu
@pytest.mark.parametrize("model,N", [("acoustic", 3), ("elastic", 2)])
def test_checkpoint_resume_is_bitwise(dg, model, N):
    """50 steps, checkpoint (q, r^{m-1}, r^{m-2}, step) to host, restore into a
    fresh handle, 50 more steps == 100 uninterrupted steps, bit for bit."""
    verts, tets, coeffs = _mesh(model, 3, 90 + N)
    o = OSolver(model, N, verts, tets, coeffs)
    dt = o.suggest_dt(0.4)
    q0 = np.zeros((o.K, o.Nf, o.ref.Np), np.float32)
    q0[:, 0] = W.gaussian_pulse(o.mesh.x, width=0.25)
    a = dg.Solver(verts, tets, coeffs, N, model, dt=dt)
    a.set_state(q0)
    a.step(100)
    ref = a.get_state()
    b = dg.Solver(verts, tets, coeffs, N, model, dt=dt)
    b.set_state(q0)
    b.step(50)
    q = np.empty(b.shape, np.float32)
    r1 = np.empty(b.shape, np.float32)
    r2 = np.empty(b.shape, np.float32)
    b.get_state(q, r1, r2)
    assert b.step_index == 50 and b.history == 2
    c = dg.Solver(verts, tets, coeffs, N, model, dt=dt)
    c.set_state(q, r1, r2, step=50)
    c.step(50)
    assert np.array_equal(c.get_state(), ref)


@pytest.mark.gpu
@pytest.mark.parametrize("model", ["acoustic", "elastic"])
@pytest.mark.parametrize("N", range(1, 9))
def test_every_kernel_variant_rhs_and_steps(dg, model, N):
    """Every compiled variant (block sizes, tiles, split GEMM path) gives the
    oracle's RHS and the same 20-step state as variant 0."""
    n = 4 if N <= 3 else 3
    verts, tets, coeffs = _mesh(model, n, 120 + N)
    o = OSolver(model, N, verts, tets, coeffs)
    dt = o.suggest_dt(0.4)
    q = W.random_state(o.K, o.Nf, o.ref.Np, seed=N).astype(np.float32)
    ro = o.rhs(q.astype(np.float64))
    g = dg.Solver(verts, tets, coeffs, N, model, dt=dt)
    nv = g.kernel_info()["variants"]
    ref_state = None
    for v in range(nv):
        g.set_variant(v)
        g.set_state(q)
        assert rel_l2(model, g.rhs(), ro) <= RHS_TOL, (v, g.kernel_info())
        g.step(20)
        g.sync()
        s = g.get_state()
        if ref_state is None:
            ref_state = s
        else:
            assert rel_l2(model, s, ref_state.astype(np.float64)) <= 1e-5, (v, g.kernel_info())
    g.close()


@pytest.mark.gpu
def test_async_pinned_transfers_on_another_stream(dg):
    """dg_set_state / dg_get_state with page-locked host memory in stream
    order (on_device = 2) on a stream set by dg_set_stream give the same
    state, bit for bit, as the synchronous host path; memory that is not
    page-locked is refused."""
    import torch
    verts, tets, coeffs = _mesh("acoustic", 3, 90)
    ref = dg.Solver(verts, tets, coeffs, 4, "acoustic", dt=1e-3)
    g = dg.Solver(verts, tets, coeffs, 4, "acoustic", dt=1e-3)
    st = torch.cuda.Stream()
    g.set_stream(st.cuda_stream)
    q = W.random_state(ref.K, ref.Nf, ref.Np, seed=5).astype(np.float32)
    pin = torch.from_numpy(q.copy()).pin_memory()
    out = torch.empty(g.shape, dtype=torch.float32).pin_memory()
    for _ in range(3):
        ref.set_state(q)
        ref.step(2)
        q = ref.get_state()
        g.set_state(pin, asynchronous=True)
        g.step(2)
        g.get_state(out, asynchronous=True)
        g.sync()
        pin.copy_(out)
        assert np.array_equal(out.numpy(), q)
    with pytest.raises(dg.DGError) as e:
        g.set_state(np.zeros(g.shape, np.float32), asynchronous=True)
    assert e.value.code == -1
    g.close()
    ref.close()


@pytest.mark.gpu
def test_meshes_stepping_concurrently_on_their_own_streams(dg):
    """Independent meshes of different degrees stepped at the same time, each
    on a stream of its own forked from one stream and joined back (the
    bench's sweep), end in the states they reach stepped one after another,
    bit for bit: the kernels of different handles share no device state."""
    import torch
    cases = [("acoustic", 2, 4, 71), ("acoustic", 5, 3, 72), ("acoustic", 8, 2, 73), ("elastic", 3, 3, 74)]
    solo, conc = [], []
    for model, N, n, seed in cases:
        verts, tets, coeffs = _mesh(model, n, seed)
        q = W.random_state(tets.shape[0], 4 if model == "acoustic" else 9, (N + 1) * (N + 2) * (N + 3) // 6,
                           seed=seed).astype(np.float32)
        for lst in (solo, conc):
            g = dg.Solver(verts, tets, coeffs, N, model, dt=1e-4)
            g.set_state(q)
            lst.append(g)
    for g in solo:
        g.step(7)
        g.sync()
    main = torch.cuda.Stream()
    streams = [torch.cuda.Stream() for _ in conc]
    fork, joins = torch.cuda.Event(), [torch.cuda.Event() for _ in conc]
    fork.record(main)
    for g, st, ev in zip(conc, streams, joins):
        g.set_stream(st.cuda_stream)
        st.wait_event(fork)
        g.step(7)
        ev.record(st)
    for ev in joins:
        main.wait_event(ev)
    main.synchronize()
    for a, b in zip(solo, conc):
        b.sync()
        assert np.array_equal(a.get_state(), b.get_state())
        a.close()
        b.close()


@pytest.mark.gpu
@pytest.mark.parametrize("model,N", [("acoustic", 3), ("acoustic", 6), ("elastic", 2), ("elastic", 5)])
def test_wide_vertex_indices_give_the_same_solver(dg, model, N):
    """A mesh whose vertex array holds more than 2^21 vertices is matched
    face by face on whole index triples instead of 21-bit packed keys; the
    same tets, numbered into such an array, must give the compact mesh's RHS
    and AB3 steps bit for bit (same connectivity, same face rotations)."""
    verts, tets, coeffs = _mesh(model, 3, 81)
    nv = 2 ** 21 + 1
    rng = np.random.default_rng(N)
    slots = np.sort(rng.choice(nv, size=verts.shape[0], replace=False))
    slots[-1] = nv - 1
    big = np.full((nv, 3), 1.0e3)
    big[slots] = verts
    q = W.random_state(tets.shape[0], 4 if model == "acoustic" else 9, (N + 1) * (N + 2) * (N + 3) // 6,
                       seed=N).astype(np.float32)
    out = []
    for vv, tt in ((verts, tets), (big, slots[tets])):
        g = dg.Solver(vv, tt, coeffs, N, model, dt=1e-4)
        g.set_state(q)
        r = g.rhs()
        g.step(5)
        out.append((r, g.get_state()))
        g.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
