"""dg_rhs_host_noalloc: the RHS read into host memory without allocating.

Some callers cannot allocate device memory when they need the RHS (their
device memory is already committed to another allocator or to a fixed
budget).  The entry point under test stages the RHS in a fixed array the
library holds instead of a per-call allocation; dg_setup does every
allocating step beforehand.  It must return what the allocating entry point
dg_rhs returns, on two calls in a row (the second after a state change, so
that a stale scratch would show), for handles of every kind (fused and
split default variants, the tensor-core precision, the plain and library
strategies), leave the device's free memory unchanged, and refuse meshes
whose RHS does not fit the array.  This file is collected last.
"""

import numpy as np
import pytest

import workloads as W

RHS_TOL = 1e-5  # relative L2, the RHS tolerance of the parity tests


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _mesh(model, n, seed=9):
    verts, tets = W.kuhn_cube_mesh(n, 0.1, seed=seed)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=3) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=3))
    return verts, tets, coeffs


# acoustic N = 3 and elastic N = 2 default to the fused step, acoustic N = 8
# and elastic N = 7 to the split step (the entry point then runs a fused
# variant of its own)
@pytest.mark.gpu
@pytest.mark.parametrize("model,N,n", [("acoustic", 3, 4), ("elastic", 2, 5), ("acoustic", 8, 3),
                                       ("elastic", 7, 3)])
def test_noalloc_rhs_matches_dg_rhs_on_two_calls(model, N, n):
    import paper_1602_07997_gb300 as P
    verts, tets, coeffs = _mesh(model, n)
    K = tets.shape[0]
    g = P.Solver(verts, tets, coeffs, N, model, dt=1e-4)
    for seed in (1, 2):
        q = W.random_state(K, g.Nf, g.Np, seed=seed).astype(np.float32)
        g.set_state(q)
        ref = g.rhs()                      # allocating entry point
        got = g.rhs_host_noalloc()         # allocation-free entry point
        assert _rel(got, ref) <= RHS_TOL
    g.close()


@pytest.mark.gpu
@pytest.mark.parametrize("strategy", ["plain", "library"])
def test_noalloc_rhs_of_the_comparison_strategies(strategy):
    import paper_1602_07997_gb300 as P
    verts, tets, coeffs = _mesh("acoustic", 4)
    K = tets.shape[0]
    g = P.Solver(verts, tets, coeffs, 5, "acoustic", dt=1e-4, strategy=strategy)
    for seed in (3, 4):
        g.set_state(W.random_state(K, g.Nf, g.Np, seed=seed).astype(np.float32))
        assert _rel(g.rhs_host_noalloc(), g.rhs()) <= RHS_TOL
    g.close()


@pytest.mark.gpu
def test_noalloc_rhs_of_a_tensor_core_handle_matches_the_oracle():
    """The handle computes its own RHS in split BF16; the allocation-free call
    runs the FP32 fused step, so it is held to the oracle's RHS."""
    import paper_1602_07997_gb300 as P
    from oracle.dg import Solver as OSolver
    verts, tets, coeffs = _mesh("acoustic", 3)
    K = tets.shape[0]
    o = OSolver("acoustic", 5, verts, tets, coeffs)
    g = P.Solver(verts, tets, coeffs, 5, "acoustic", dt=1e-4, precision="bf16x6")
    for seed in (5, 6):
        q = W.random_state(K, g.Nf, g.Np, seed=seed).astype(np.float32)
        g.set_state(q)
        ro = o.rhs(q.astype(np.float64))
        for grp in ([0], [1, 2, 3]):
            assert _rel(g.rhs_host_noalloc()[:, grp], ro[:, grp]) <= RHS_TOL
    g.close()


@pytest.mark.gpu
def test_noalloc_call_leaves_free_device_memory_unchanged():
    import torch
    import paper_1602_07997_gb300 as P
    verts, tets, coeffs = _mesh("acoustic", 4)
    g = P.Solver(verts, tets, coeffs, 8, "acoustic", dt=1e-4)   # split default: a fused variant of its own
    g.set_state(W.random_state(tets.shape[0], g.Nf, g.Np, seed=7).astype(np.float32))
    out = np.empty(g.shape, dtype=np.float32)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    g.rhs_host_noalloc(out)
    g.rhs_host_noalloc(out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
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
