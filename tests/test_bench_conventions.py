"""Counting conventions behind bench.py's roofline figures (host logic, no GPU).

The algorithmic bytes and FLOPs per element follow the operator products of
Section 3.2 (Eq. dgLocalRhs): every volume product is one Np x Np matrix
applied to one nodal field, every lift one Np x 4Nfp matrix applied to one
face-node field.  The tests enumerate those products instead of restating
the closed forms in bench.py.
"""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def sizes(N):
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nfp = (N + 1) * (N + 2) // 2
    return Np, Nfp


def products(model):
    """(volume products, lifted face fields) of the unfactored RHS."""
    if model == "acoustic":
        # grad p (3 derivatives of p) and div v (one derivative per velocity component)
        vol = [("p", d) for d in range(3)] + [("v%d" % c, c) for c in range(3)]
        return vol, 4
    # velocity gradient (3 x 3) and stress divergence (3 components x 3 derivatives)
    vol = [("v%d" % c, d) for c in range(3) for d in range(3)] + \
          [("s%d%d" % (c, d), d) for c in range(3) for d in range(3)]
    return vol, 9


@pytest.mark.parametrize("model", ["acoustic", "elastic"])
@pytest.mark.parametrize("N", range(1, 9))
def test_algorithmic_counts_enumerate_the_products(model, N):
    Np, Nfp = sizes(N)
    Nf = 4 if model == "acoustic" else 9
    vol, lifted = products(model)
    mac = len(vol) * Np * Np + lifted * Np * 4 * Nfp
    K = 37
    byt, flop = bench.algorithmic(model, N, K)
    # five FP32 arrays of Nf Np values (q^m, r^m-1, r^m-2 read; q^m+1, r^m written) + the record
    assert byt == K * (5 * 4 * Nf * Np + 84)
    # one multiply-add = 2 flops; AB3 = 8 flops per field-node
    assert flop == K * (2 * mac + 8 * Nf * Np)
    assert bench.executed_flops(model, N, K, False) == flop


@pytest.mark.parametrize("model", ["acoustic", "elastic"])
@pytest.mark.parametrize("N", range(1, 9))
def test_factored_counts(model, N):
    """Surface streams: acoustic lifts 2 streams and rebuilds 3 velocity
    components from 4 face normals; elastic lifts 3 + 3 streams and folds 6
    stress components per face (n.W 3, lambda scaling 1, diagonal 3 x 2,
    off-diagonal 3 x 2 multiply-adds)."""
    Np, Nfp = sizes(N)
    vol, _ = products(model)
    K = 5
    if model == "acoustic":
        streams, fold = 2, 3 * 4
        Nf = 4
    else:
        streams, fold = 6, 4 * (3 + 1 + 6 + 6)
        Nf = 9
    mac = len(vol) * Np * Np + streams * Np * 4 * Nfp + fold * Np
    ex = bench.executed_flops(model, N, K, True)
    assert ex == K * (2 * mac + 8 * Nf * Np)
    # the elastic fold (64 Np) outweighs the saved lifts (12 Np Nfp) at N = 1,
    # where the fused elastic kernel keeps the nine penalty fields
    if model == "acoustic" or N >= 2:
        assert ex < bench.algorithmic(model, N, K)[1]


class _G:
    def __init__(self, split):
        self.split = split

    def kernel_info(self):
        return {"split": self.split}


@pytest.mark.parametrize("split", [0, 1, 2])
def test_which_paths_lift_surface_streams(split):
    g = _G(split)
    # the library route factors in every mode; the plain route never
    for model in ("acoustic", "elastic"):
        assert bench.is_factored(model, g, "fp32", "library")
        assert not bench.is_factored(model, g, "fp32", "plain")
        # the tensor-core front halves lift every penalty field
        assert not bench.is_factored(model, g, "bf16x6", "fused")
    # fused FP32: every acoustic kernel, only the elastic split step
    assert bench.is_factored("acoustic", g, "fp32", "fused")
    assert bench.is_factored("elastic", g, "fp32", "fused") == (split == 1)


def test_clock_summary_keeps_the_timed_window():
    """Only samples that arrived inside the timed region (plus one interval)
    count; throttle reasons are the ones active there."""
    c = bench.ClockSampler(0)
    idle = "1200, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    load = "2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    capped = "1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active"
    c.lines = [(0.00, idle), (0.05, idle), (1.00, load), (1.05, capped), (1.10, load), (3.00, idle)]
    s = c.summary(1.0, 1.08)
    assert s["samples"] == 3 and s["sm_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"]
    # no sample inside the window: every sample counts
    s = c.summary(2.0, 2.5)
    assert s["samples"] == 6
    assert bench.ClockSampler(0).summary()["samples"] == 0


def test_reference_arm_line(capsys):
    """--impl reference: rank 0 prints one JSON line (oracle timed on the host
    cores, the same metric and unit, e2e with no copies); other ranks print
    nothing."""
    import json
    import types
    args = types.SimpleNamespace(steps=2, warmup=1)
    bench.run_reference(args, 1, 2)
    assert capsys.readouterr().out == ""
    bench.run_reference(args, 0, 1)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 2 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_sweep_meshes_have_the_documented_sizes():
    """The ~2 M-node sweep: 6 n^3 Kuhn tets per degree with n = 44, 32, 26,
    21, 18, 16, 14, 13 (6 n^3 Np closest to 2 M), as the measured tables
    and profiles quote them."""
    import workloads as W
    expect = {1: 44, 2: 32, 3: 26, 4: 21, 5: 18, 6: 16, 7: 14, 8: 13}
    for N, n in expect.items():
        assert W.n_for_target_nodes(N) == n
        Np = (N + 1) * (N + 2) * (N + 3) // 6
        nodes = 6 * n ** 3 * Np
        assert 1.9e6 < nodes < 2.2e6
    verts, tets = W.kuhn_cube_mesh(3, jitter=0.1, seed=1)
    assert tets.shape == (6 * 27, 4) and verts.shape == (64, 3)
