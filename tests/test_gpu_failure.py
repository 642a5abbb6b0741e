"""Failure detection on the GPU, made on the host side of the data.

* A NaN planted in the state (dg_set_state) is found by the finite-state
  check that runs after every k-th step and reported by dg_sync as
  DG_ENONFINITE; the report clears the flag and the handle steps on.
* Bounded device waits: a wait limit of -1 makes the first wait of every CTA
  give up at once (the test hook of dg_set_wait_limit), on every kernel form
  (fused with staged or streamed history, whole-neighbour halos, the FP32
  split step and the tcgen05 split step).  dg_sync reports DG_ETIMEOUT, and
  afterwards the same handle, with the default limit, matches the FP64
  oracle again: the expiry path drained its copies and left the context
  usable.  A short positive limit makes waits expire at varying points of
  the pipeline; whatever it reports, the handle then recovers the same way.
No GPU is faulted, trapped or hung: every expiry is a bounded wait that
returns an error status.
"""

import numpy as np
import pytest

import workloads as W

STEP_TOL = 1e-5


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _setup(model, N, n=3, precision="fp32"):
    import paper_1602_07997_gb300 as P
    from oracle.dg import Solver as OSolver
    verts, tets = W.kuhn_cube_mesh(n, 0.1, seed=11)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=12) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=12))
    o = OSolver(model, N, verts, tets, coeffs)
    dt = o.suggest_dt(0.4)
    g = P.Solver(verts, tets, coeffs, N, model, dt=dt, precision=precision)
    q = W.random_state(K, o.Nf, o.ref.Np, seed=13).astype(np.float32)
    return P, o, g, q, dt


def _steps_match_oracle(o, g, q, dt, n=5):
    from oracle.dg import AB3Stepper
    g.set_state(q)
    g.step(n)
    g.sync()
    st = AB3Stepper(o, q.astype(np.float64), dt)
    st.step(n)
    qg = g.get_state()
    for grp in ([0], [1, 2, 3]) if o.Nf == 4 else (range(3), range(3, 9)):
        grp = list(grp)
        assert _rel(qg[:, grp], st.q[:, grp]) <= STEP_TOL


# fused (acoustic N = 3), split FP32 (acoustic N = 6), tensor cores (acoustic N = 5, bf16x6), elastic split (N = 5)
CASES = [("acoustic", 3, "fp32"), ("acoustic", 6, "fp32"), ("acoustic", 5, "bf16x6"), ("elastic", 5, "fp32")]


@pytest.mark.gpu
@pytest.mark.parametrize("model,N,precision", CASES)
def test_nonfinite_state_is_reported_once(model, N, precision):
    P, o, g, q, dt = _setup(model, N, precision=precision)
    bad = q.copy()
    bad[7, 1, 3] = np.nan
    g.set_state(bad)
    g.set_finite_check(1)
    g.step(1)
    with pytest.raises(P.DGError) as e:
        g.sync()
    assert e.value.code == -4  # DG_ENONFINITE
    g.sync()  # reported once
    _steps_match_oracle(o, g, q, dt)
    g.close()


@pytest.mark.gpu
def test_default_finite_check_interval():
    """With the default interval (100 steps) a NaN is reported by the sync
    after step 100, not before."""
    P, o, g, q, dt = _setup("acoustic", 2)
    bad = q.copy()
    bad[0, 0, 0] = np.inf
    g.set_state(bad)
    g.step(99)
    g.sync()
    g.step(1)
    with pytest.raises(P.DGError) as e:
        g.sync()
    assert e.value.code == -4
    g.set_finite_check(0)
    g.set_state(bad)
    g.step(100)
    g.sync()  # checking turned off
    g.close()


# every kernel form: acoustic N = 1 (whole-neighbour halos), N = 3 (history
# staged in shared memory), N = 6 (FP32 split step), N = 5 bf16x6 (tcgen05);
# elastic N = 2 (fused) and N = 5 (split); N = 8 of both models (the split
# step with the warp-specialised persistent GEMM, their defaults) and the
# last compiled variant of acoustic N = 8 (the split step with one CTA per
# GEMM tile)
FORMS = [("acoustic", 1, "fp32", 0), ("acoustic", 3, "fp32", 0), ("acoustic", 6, "fp32", 0),
         ("acoustic", 5, "bf16x6", 0), ("elastic", 2, "fp32", 0), ("elastic", 5, "fp32", 0),
         ("acoustic", 8, "fp32", 0), ("elastic", 8, "fp32", 0), ("acoustic", 8, "fp32", -1)]


def _form(model, N, precision, variant):
    P, o, g, q, dt = _setup(model, N, n=4, precision=precision)
    if variant != 0:
        g.set_variant(g.kernel_info()["variants"] + variant if variant < 0 else variant)
    return P, o, g, q, dt


@pytest.mark.gpu
@pytest.mark.parametrize("model,N,precision,variant", FORMS)
def test_forced_wait_expiry_is_reported_and_the_handle_recovers(model, N, precision, variant):
    P, o, g, q, dt = _form(model, N, precision, variant)
    g.set_state(q)
    g.set_wait_limit(-1)
    g.step(2)
    with pytest.raises(P.DGError) as e:
        g.sync()
    assert e.value.code == -5  # DG_ETIMEOUT
    g.set_wait_limit(0)
    _steps_match_oracle(o, g, q, dt)
    g.set_variant(0)  # the choice is process-wide
    g.close()


@pytest.mark.gpu
@pytest.mark.parametrize("model,N,precision,variant", FORMS)
def test_short_wait_limit_then_recovery(model, N, precision, variant):
    P, o, g, q, dt = _form(model, N, precision, variant)
    g.set_state(q)
    for limit in (64, 512):
        g.set_wait_limit(limit)
        g.step(3)
        try:
            g.sync()
        except P.DGError as e:
            assert e.code == -5
    g.set_wait_limit(0)
    _steps_match_oracle(o, g, q, dt)
    g.set_variant(0)
    g.close()


@pytest.mark.gpu
def test_launch_count_follows_the_steps():
    P, o, g, q, dt = _setup("acoustic", 6)   # split step: two kernels per step
    g.set_finite_check(0)
    n0 = g.launch_count()
    g.set_state(q)
    g.step(4)
    g.sync()
    assert g.launch_count() - n0 == 8
    g.set_finite_check(2)
    n0 = g.launch_count()
    g.step(4)
    g.sync()
    assert g.launch_count() - n0 == 8 + 2
    g.close()
