"""dg_rhs_host_noalloc: the RHS read into host memory without allocating.

Some callers cannot allocate device memory when they need the RHS (their
device memory is already committed to another allocator or to a fixed
budget).  The entry point under test stages the RHS in a fixed array the
library holds instead of a per-call allocation.  It must return what the
allocating entry point dg_rhs returns, on two calls in a row (the second
after a state change, so that a stale scratch would show), and refuse
meshes whose RHS does not fit the array.  This file is collected last.
"""

import numpy as np
import pytest

import workloads as W

RHS_TOL = 1e-5  # relative L2, the RHS tolerance of the parity tests


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


@pytest.mark.gpu
@pytest.mark.parametrize("model,N,n", [("acoustic", 3, 4), ("elastic", 2, 5)])
def test_noalloc_rhs_matches_dg_rhs_on_two_calls(model, N, n):
    import paper_1602_07997_gb300 as P
    verts, tets = W.kuhn_cube_mesh(n, 0.1, seed=9)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=3) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=3))
    g = P.Solver(verts, tets, coeffs, N, model, dt=1e-4)
    for seed in (1, 2):
        q = W.random_state(K, g.Nf, g.Np, seed=seed).astype(np.float32)
        g.set_state(q)
        ref = g.rhs()                      # allocating entry point
        got = g.rhs_host_noalloc()         # allocation-free entry point
        assert _rel(got, ref) <= RHS_TOL
    g.close()


@pytest.mark.gpu
def test_noalloc_rejects_meshes_beyond_the_scratch():
    import paper_1602_07997_gb300 as P
    verts, tets = W.kuhn_cube_mesh(11, 0.1, seed=1)   # 7986 tets x 4 x 165 > 4 Mi floats
    g = P.Solver(verts, tets, W.acoustic_coefficients(tets.shape[0], 1, 2, seed=1), 8, "acoustic")
    with pytest.raises(P.DGError) as e:
        g.rhs_host_noalloc()
    assert e.value.code == -1 and "exceeds" in str(e.value)
    g.close()
