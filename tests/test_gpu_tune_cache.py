"""The autotuner's choices persisted across processes (dg_tune_save /
dg_tune_load): a choice saved, forgotten and loaded again is the variant
that later handles start with; lines for another device or naming a
variant this build compiles differently are skipped."""

import numpy as np
import pytest

import workloads as W


@pytest.mark.gpu
def test_tune_cache_round_trip(tmp_path):
    import paper_1602_07997_gb300 as P
    verts, tets = W.kuhn_cube_mesh(4, 0.1, seed=21)
    coeffs = W.acoustic_coefficients(tets.shape[0], 1, 3, seed=22)
    P.tune_clear()
    g = P.Solver(verts, tets, coeffs, 3, "acoustic", dt=1e-4)
    assert g.kernel_info()["variant"] == 0
    nv = g.kernel_info()["variants"]
    g.set_variant(nv - 1)            # a choice, as dg_autotune would make it
    g.close()
    path = tmp_path / "tune.txt"
    P.tune_save(str(path))
    lines = path.read_text().splitlines()
    assert lines[0] == "# libdg autotune cache v1" and len(lines) == 2
    P.tune_clear()
    g = P.Solver(verts, tets, coeffs, 3, "acoustic", dt=1e-4)
    assert g.kernel_info()["variant"] == 0
    g.close()
    assert P.tune_load(str(path)) == 1
    g = P.Solver(verts, tets, coeffs, 3, "acoustic", dt=1e-4)
    assert g.kernel_info()["variant"] == nv - 1
    g.close()
    # another device name, and a variant whose shape no longer matches: skipped
    f = lines[1].split()
    other = " ".join(["Some_Other_GPU"] + f[1:])
    stale = " ".join(f[:7] + [str(int(f[7]) + 1)] + f[8:])
    path.write_text("\n".join([lines[0], other, stale]) + "\n")
    P.tune_clear()
    assert P.tune_load(str(path)) == 0
    P.tune_clear()
