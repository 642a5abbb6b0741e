"""Parity at the benchmark's full sizes: the ~2 M-node sweep meshes (K up to
511 104 tets), in the launch configuration bench.py times (the autotuned
variant of each degree), against the FP64 oracle on every output.

Same bars as the small cases: rel-L2 per field group <= 1e-5 after one RHS
(random state, so that every node and face contributes), <= 1e-4 after AB3
steps.
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


@pytest.fixture(scope="module")
def dg():
    import paper_1602_07997_gb300 as P
    P.lib()
    return P


def _full_rhs(dg, model, N, precision="fp32"):
    cfg = W.sweep_mesh(model, N)
    o = OSolver(model, N, cfg["verts"], cfg["tets"], cfg["coeffs"])
    g = dg.Solver(cfg["verts"], cfg["tets"], cfg["coeffs"], N, model, dt=1e-6, precision=precision)
    q = W.random_state(o.K, o.Nf, o.ref.Np, seed=N).astype(np.float32)
    g.set_state(q)
    g.autotune(3)  # the bench's launch configuration
    err = rel_l2(model, g.rhs(), o.rhs(q.astype(np.float64)))
    info = g.kernel_info()
    g.close()
    return err, info, o.K


@pytest.mark.gpu
@pytest.mark.parametrize("N", range(1, 9))
def test_full_size_acoustic_rhs(dg, N):
    err, info, K = _full_rhs(dg, "acoustic", N)
    print(f"acoustic N={N} K={K} variant {info['variant']} split {info['split']} rel-L2 {err:.2e}")
    assert err <= RHS_TOL, err


@pytest.mark.gpu
@pytest.mark.parametrize("N", [2, 5, 8])
def test_full_size_elastic_rhs(dg, N):
    err, info, K = _full_rhs(dg, "elastic", N)
    print(f"elastic N={N} K={K} variant {info['variant']} split {info['split']} rel-L2 {err:.2e}")
    assert err <= RHS_TOL, err


@pytest.mark.gpu
def test_full_size_tensor_core_rhs(dg):
    err, info, K = _full_rhs(dg, "acoustic", 7, precision="bf16x6")
    print(f"bf16x6 acoustic N=7 K={K} rel-L2 {err:.2e}")
    assert info["split"] == 2
    assert err <= RHS_TOL, err


@pytest.mark.gpu
def test_full_size_ab3_steps(dg):
    model, N = "acoustic", 4
    cfg = W.sweep_mesh(model, N)
    o = OSolver(model, N, cfg["verts"], cfg["tets"], cfg["coeffs"])
    dt = o.suggest_dt(0.4)
    q0 = np.zeros((o.K, o.Nf, o.ref.Np))
    q0[:, 0] = W.gaussian_pulse(o.mesh.x)
    g = dg.Solver(cfg["verts"], cfg["tets"], cfg["coeffs"], N, model, dt=dt)
    g.set_state(q0.astype(np.float32))
    g.autotune(3)
    g.step(3)
    g.sync()
    st = AB3Stepper(o, q0, dt)
    st.step(3)
    err = rel_l2(model, g.get_state(), st.q)
    g.close()
    assert err <= STEP_TOL, err


@pytest.mark.gpu
def test_large_elastic_rhs_sampled(dg):
    """The large elastic configuration (N = 7, 131 712 tets, 15.8 M nodes, 2.3 GB
    of state) in the autotuned launch configuration, against the oracle's RHS
    on 400 sampled elements (the same formulas on those elements' rows)."""
    from workloads.configs import config5_elastic_large
    cfg = config5_elastic_large()
    model, N = "elastic", cfg["N"]
    o = OSolver(model, N, cfg["verts"], cfg["tets"], cfg["coeffs"])
    g = dg.Solver(cfg["verts"], cfg["tets"], cfg["coeffs"], N, model, dt=1e-6)
    q = W.random_state(o.K, o.Nf, o.ref.Np, seed=5).astype(np.float32)
    g.set_state(q)
    g.autotune(2)
    r = g.rhs()
    g.close()
    sample = np.sort(np.random.default_rng(5).choice(o.K, size=400, replace=False))
    ro = o.rhs(q, elems=sample)
    err = rel_l2(model, r[sample], ro)
    print(f"large elastic N=7 K={o.K} sampled rel-L2 {err:.2e}")
    assert err <= RHS_TOL, err
