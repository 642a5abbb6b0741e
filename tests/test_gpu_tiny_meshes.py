"""GPU parity on meshes smaller than one block of elements.

One tetrahedron (K = 1: every face on the outer boundary, no neighbour
traces at all) and the perturbed six-tet cube (K = 6) exercise the ragged
tail in its most extreme form: every compiled FP32 variant, fused and split
step, must give the oracle's RHS (rel. L2 <= 1e-5) and, over 10 AB3 steps,
its state (<= 1e-4).
"""

import numpy as np
import pytest

import workloads as W
from oracle.dg import Solver as OSolver, AB3Stepper

RHS_TOL = 1e-5
STEP_TOL = 1e-4


def rel_l2(model, a, b):
    gs = ((0,), (1, 2, 3)) if model == "acoustic" else ((0, 1, 2), tuple(range(3, 9)))
    a = np.asarray(a, np.float64)
    return max(np.linalg.norm((a[:, g] - b[:, g]).ravel()) / np.linalg.norm(b[:, g].ravel()) for g in gs)


def tiny_mesh(kind):
    if kind == "one_tet":
        verts = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
        return verts, np.array([[0, 1, 2, 3]], dtype=np.int64)
    return W.six_tet_cube(0.1, seed=3)


@pytest.fixture(scope="module")
def dg():
    import paper_1602_07997_gb300 as P
    P.lib()
    return P


@pytest.mark.gpu
@pytest.mark.parametrize("kind", ["one_tet", "six_tets"])
@pytest.mark.parametrize("model", ["acoustic", "elastic"])
@pytest.mark.parametrize("N", [1, 3, 5, 8])
def test_every_variant_on_a_mesh_smaller_than_a_block(dg, kind, model, N):
    verts, tets = tiny_mesh(kind)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=7) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=7))
    o = OSolver(model, N, verts, tets, coeffs)
    dt = o.suggest_dt(0.4)
    q = W.random_state(o.K, o.Nf, o.ref.Np, seed=N)
    ro = o.rhs(q)
    st = AB3Stepper(o, q, dt)
    st.step(10)
    g = dg.Solver(verts, tets, coeffs, N, model, dt=dt)
    for v in range(g.kernel_info()["variants"]):
        g.set_variant(v)
        g.set_state(q.astype(np.float32))
        assert rel_l2(model, g.rhs(), ro) <= RHS_TOL, (v, g.kernel_info())
        g.step(10)
        g.sync()
        assert rel_l2(model, g.get_state(), st.q) <= STEP_TOL, (v, g.kernel_info())
    g.close()
