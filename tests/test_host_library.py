"""Host-side tests of libdg (no GPU): exports, reference element, dt helper, validation.

The library's reference element is built by a different route (orthonormal
Dubiner basis, V-based mass/lift, integer-lattice face tables) than the
oracle's (Bernstein basis, quadrature, coordinate matching); agreement to
round-off pins both set-up codes against each other.
"""

import os
import re

import numpy as np
import pytest

import workloads as W
from oracle.refelem import RefElement
from oracle.dg import Solver as OSolver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    import paper_1602_07997_gb300 as P
    from paper_1602_07997_gb300 import build as B
    if not os.path.exists(B.LIB):
        B.build()
    P.lib()
    return P


def test_library_exports_every_declared_symbol(P):
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(dg_[a-z_0-9]+)\s*\(", src))
    assert len(names) >= 20
    L = P.lib()
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert names == set(P.EXPORTS)


@pytest.mark.parametrize("N", range(1, 9))
def test_reference_element_matches_oracle(P, N):
    L = P.reference_element(N)
    R = RefElement(N)
    assert np.abs(L["nodes"] - R.nodes).max() < 1e-13
    for a, b in ((L["Dr"], R.Dr), (L["Ds"], R.Ds), (L["Dt"], R.Dt)):
        assert np.abs(a - b).max() < 1e-12 * max(1.0, np.abs(b).max())
    for f in range(4):
        fm = L["fmask"][f]
        assert sorted(fm) == sorted(R.Fmask[f])
        col = [list(R.Fmask[f]).index(n) for n in fm]
        A = L["LIFT"][:, f * R.Nfp:(f + 1) * R.Nfp]
        B = R.LIFT[:, f * R.Nfp:(f + 1) * R.Nfp][:, col]
        assert np.abs(A - B).max() < 1e-12 * np.abs(B).max()


@pytest.mark.parametrize("model", ["acoustic", "elastic"])
def test_suggest_dt_matches_oracle(P, model):
    verts, tets = W.kuhn_cube_mesh(3, 0.1, seed=4)
    K = tets.shape[0]
    coeffs = (W.acoustic_coefficients(K, 1, 3, seed=1) if model == "acoustic"
              else W.elastic_two_layer(verts, tets, seed=1))
    for N in (1, 4, 8):
        o = OSolver(model, N, verts, tets, coeffs)
        assert abs(P.suggest_dt(verts, tets, coeffs, N, model, 0.4) - o.suggest_dt(0.4)) <= 1e-14 * o.suggest_dt(0.4)


def test_host_validation_rejects_bad_input(P):
    verts, tets = W.kuhn_cube_mesh(2, 0.1, seed=1)
    K = tets.shape[0]
    c = np.ones((K, 2))
    bad = tets.copy()
    bad[3, [1, 2]] = bad[3, [2, 1]]
    for args in ((verts, bad, c, 2, "acoustic"),                          # inverted tet
                 (verts, np.concatenate([tets, tets[:1]]), np.ones((K + 1, 2)), 2, "acoustic"),  # 3 tets on a face
                 (verts, tets, c, 0, "acoustic"),                          # N out of range
                 (verts, tets, -c, 2, "acoustic"),                         # negative coefficient
                 (verts, np.where(tets == 0, 10 ** 6, tets), c, 2, "acoustic")):  # index out of range
        with pytest.raises(P.DGError) as e:
            P.suggest_dt(*args)
        assert e.value.code == -1


def test_strategy_and_precision_combinations_checked_before_device_use(P):
    """Each strategy takes only its precision modes (DG_EINVAL otherwise), and
    the check comes before any device allocation."""
    verts, tets = W.kuhn_cube_mesh(2, 0.1, seed=1)
    c = np.ones((tets.shape[0], 2))
    for strategy, precision in (("plain", "bf16x6"), ("plain", "tf32"), ("fused", "tf32"),
                                ("library", "bf16x3"), ("library", "bf16x6")):
        with pytest.raises(P.DGError) as e:
            P.Solver(verts, tets, c, 2, "acoustic", strategy=strategy, precision=precision)
        assert e.value.code == -1, (strategy, precision)


def test_binding_checks_array_shapes(P):
    """The binding refuses arrays whose size would make the library read past
    them (mesh, coefficients), before any call into the library."""
    verts, tets = W.kuhn_cube_mesh(2, 0.1, seed=1)
    K = tets.shape[0]
    for v, t, c, model in ((verts[:, :2], tets, np.ones((K, 2)), "acoustic"),    # 2-D vertices
                           (verts, tets[:, :3], np.ones((K, 2)), "acoustic"),    # triangles
                           (verts, tets, np.ones((K, 3)), "acoustic"),           # elastic coefficients
                           (verts, tets, np.ones((K, 2)), "elastic"),
                           (verts, tets, np.ones((K - 1, 2)), "acoustic")):
        with pytest.raises(ValueError):
            P.suggest_dt(v, t, c, 2, model, 0.4)


def test_binding_checks_source_points(P):
    """Source positions and directions are three coordinates (checked before
    the handle is touched)."""
    import types
    fake = types.SimpleNamespace(h=None)
    for xs, d in (((0.5, 0.5), (0.0, 0.0, 1.0)), ((0.5, 0.5, 0.5), (1.0, 0.0))):
        with pytest.raises(ValueError):
            P.Solver.set_source(fake, xs, [1.0], d)
        with pytest.raises(ValueError):
            P.Solver.add_source(fake, xs, [1.0], d)


def test_empty_mesh_is_refused(P):
    """K = 0 (or fewer than 4 vertices): DG_EINVAL from the host checks."""
    verts, tets = W.kuhn_cube_mesh(2, 0.1, seed=1)
    with pytest.raises(P.DGError) as e:
        P.suggest_dt(verts, tets[:0], np.ones((0, 2)), 2, "acoustic", 0.4)
    assert e.value.code == -1
    with pytest.raises(P.DGError) as e:
        P.suggest_dt(verts[:3], tets[:0], np.ones((0, 2)), 2, "acoustic", 0.4)
    assert e.value.code == -1


def _spread_vertices(verts, tets, nv, seed):
    """The same mesh with its vertices scattered over an array of nv vertices
    (the unused ones far away), so that the face keys need wide indices."""
    rng = np.random.default_rng(seed)
    slots = np.sort(rng.choice(nv, size=verts.shape[0], replace=False))
    slots[-1] = nv - 1  # the widest index is in use
    big = np.full((nv, 3), 1.0e3)
    big[slots] = verts
    return big, slots[tets]


@pytest.mark.parametrize("nv", [2 ** 21, 2 ** 21 + 1])
def test_face_matching_with_wide_vertex_indices(P, nv):
    """Face matching packs a face's sorted vertex triple into one 64-bit key
    when every index fits 21 bits (nv <= 2^21) and sorts the triples
    themselves otherwise.  On both sides of that boundary the host build must
    accept the conforming mesh (every interior face matched with one of its
    six vertex rotations, else "face vertex permutation not found"), give the
    same dt as the compact mesh, and still refuse a face shared by three tets."""
    verts, tets = W.kuhn_cube_mesh(3, 0.1, seed=2)
    K = tets.shape[0]
    c = W.acoustic_coefficients(K, 1, 3, seed=5)
    big, btets = _spread_vertices(verts, tets, nv, seed=nv)
    for N in (1, 5):
        assert P.suggest_dt(big, btets, c, N, "acoustic", 0.4) == P.suggest_dt(verts, tets, c, N, "acoustic", 0.4)
    with pytest.raises(P.DGError) as e:
        P.suggest_dt(big, np.concatenate([btets, btets[:1]]), np.concatenate([c, c[:1]]), 2, "acoustic", 0.4)
    assert e.value.code == -1 and "more than two" in str(e.value)


def test_tune_cache_file_handling(P, tmp_path):
    """The autotune cache: a save with no choices writes only the header, and
    loading it takes nothing; files that are not such a cache or have a
    malformed line are refused with DG_EINVAL before anything is applied."""
    P.tune_clear()
    path = tmp_path / "tune.txt"
    P.tune_save(str(path))
    assert path.read_text().splitlines() == ["# libdg autotune cache v1"]
    assert P.tune_load(str(path)) == 0
    for bad in ("no header\n", "# libdg autotune cache v1\nGB300 10.3 0 4\n",
                "# libdg autotune cache v1\nGB300 103 0 4 0 1 12 256 0 0\n"):
        path.write_text(bad)
        with pytest.raises(P.DGError) as e:
            P.tune_load(str(path))
        assert e.value.code == -1
    with pytest.raises(P.DGError):
        P.tune_load(str(tmp_path / "missing.txt"))
