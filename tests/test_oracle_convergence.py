"""Oracle pinned by exact solutions: the discrete solution converges at order N+1.

Acoustic: rigid-wall cube mode (rho = c = 1).  Elastic: traction-free cube
mode with lambda = 0, mu = rho = 1.  Upwind flux, AB3 with the history
r^{-1}, r^{-2} taken as the discrete RHS of the interpolated exact solution
at t = -dt, -2 dt, run to T = 0.1 on jittered meshes n = 2, 4, 8.
"""

import numpy as np
import pytest

import workloads as W
from oracle.dg import Solver, AB3Stepper

T_END = 0.1


def _l2(S, e):
    M = S.ref.M
    return np.sqrt(np.sum(S.mesh.J[:, None] * np.einsum("kfi,ij,kfj->kf", e, M, e)))


def _run(model, N, n):
    verts, tets = W.kuhn_cube_mesh(n, 0.1, seed=100 + n)
    K = tets.shape[0]
    if model == "acoustic":
        S = Solver(model, N, verts, tets, np.ones((K, 2)))
        exact = lambda t: np.moveaxis(W.standing_mode_acoustic(S.mesh.x, t), -1, 1)
    else:
        S = Solver(model, N, verts, tets, np.tile([0.0, 1.0, 1.0], (K, 1)))
        exact = lambda t: np.moveaxis(W.standing_mode_elastic(S.mesh.x, t), -1, 1)
    dt0 = S.suggest_dt(0.4)
    nsteps = int(np.ceil(T_END / dt0))
    dt = T_END / nsteps
    hist = (S.rhs(exact(-dt)), S.rhs(exact(-2 * dt)))
    st = AB3Stepper(S, exact(0.0), dt, history=hist)
    st.step(nsteps)
    return _l2(S, st.q - exact(T_END))


@pytest.mark.slow
@pytest.mark.parametrize("model,N", [("acoustic", 1), ("acoustic", 2), ("acoustic", 3),
                                     ("acoustic", 4), ("elastic", 1), ("elastic", 2),
                                     ("elastic", 3)])
def test_standing_mode_converges_at_order_N_plus_1(model, N):
    errs = [_run(model, N, n) for n in (2, 4, 8)]
    rate = np.log2(errs[-2] / errs[-1])
    assert rate > N + 1 - 0.3, (errs, rate)
