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


def _canned_detail():
    """A detail record shaped like a full bench run (every leg present, the
    served stream's per-request lists included)."""
    per_N = {str(N): {"K": 100000, "nodes": 2000000, "ms": 0.123456789, "kernel": {"variant": 3, "split": 1},
                      "updates_per_s": 1.234567e10, "alg_GBs": 1234.5, "alg_GFLOPs": 23456.7,
                      "exec_GFLOPs": 21234.5, "bound": "alu" if N > 4 else "hbm", "roofline_frac": 0.312345}
             for N in range(1, 9)}
    served = {"requests": 64, "steps": 500, "degrees": [3, 5, 7], "mesh_tets": [123456] * 64,
              "capacity_req_per_s": 7.1234, "arrival_rate_req_per_s": 4.987, "p50_s": 0.4321987,
              "p99_s": 1.5432198, "makespan_s": 9.87654, "batched_all_at_once_makespan_s": 8.61234,
              "batched_updates_per_s": 1e10, "launches": 12345, "plain_p50_s": 0.98765,
              "plain_p99_s": 2.28765, "plain_makespan_s": 12.3456, "plain_all_at_once_makespan_s": 11.4321,
              "plain_updates_per_s": 7e9, "rate_sweep": [{"rate_frac": 0.5}] * 3, "note": "x" * 200}
    roof = {"bound": "alu", "achieved": 29.4123456, "peak": 80.512345, "unit": "TFLOP/s", "frac": 0.3651234,
            "exec_achieved": 25.1, "exec_frac": 0.31, "traffic": 242854144,
            "kernel": "split step, acoustic N=8 (front half + FP32 GEMM, variant 0)" * 2,
            "kernel_short": "split acoustic N=8 (FP32 GEMM) v0",
            "peak_source": "measured: dg_fp32_peak FMA microbenchmark"}
    cpu = {"value": 6.7712345e7, "unit": bench.UNIT, "cores": 16, "kind": "oracle",
           "sample": "FP64 oracle, 48 AB3 step(s) on the full acoustic meshes for N=2,4, RHS of element chunks "
                     "on 16 threads", "seconds": 11.1,
           "single_core": {"value": 8.5e6, "unit": bench.UNIT, "cores": 1, "kind": "oracle", "sample": "y" * 90}}
    return {"metric": bench.METRIC, "value": 5.5967123456e10, "unit": bench.UNIT, "n_gpus": 1, "steps": 20,
            "warmup": 5, "ms_per_step": 1.16123456, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": bench.WORKLOAD, "degrees": list(range(1, 9)),
                       "meshes": {str(N): 100000 for N in range(1, 9)}, "l2": "z" * 80,
                       "parallelism": "single GPU"},
            "gpu_launches": 240, "roofline": roof, "per_N": per_N,
            "sweeps": {"elastic_fp32": {"per_N": per_N}}, "cpu_baseline": cpu,
            "e2e": {"value": 1.2345e9, "unit": bench.UNIT, "h2d_bytes_per_step": 123456789,
                    "d2h_bytes_per_step": 123456789, "steps": 5, "note": "n" * 100},
            "served": served,
            "large_elastic": {"K": 131712, "nodes": 15805440, "N": 7, "ms": 3.51234, "steps": 20,
                              "updates_per_s": 4.0512e10, "alg_GBs": 4123.4, "alg_GFLOPs": 31234.5,
                              "hbm_frac": 0.6012345, "alu_frac": 0.4012345, "kernel": {"variant": 0},
                              "traffic": 2876543210, "state_bytes": 2845000000},
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 21},
            "fp32_peak": {"scalar_tflops": 78.91234, "packed_tflops": 79.1234, "ms": 40.1, "tflops": 79.1234,
                          "sm_mhz": 2025.0, "reasons": []},
            "peaks": {"hbm_gbs": 6791.4}}


def test_headline_line_is_short_and_complete():
    """The final stdout line must survive a reader that keeps only the last
    ~3 KB of output: under 2 KB, with the contract's keys, the roofline with
    its traffic, the CPU baseline, e2e, clocks, the per-degree [ms, frac]
    table and the served latencies."""
    import json
    line = bench.headline(_canned_detail())
    text = json.dumps(line)
    assert len(text) < 2000, len(text)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "dtype", "config", "roofline", "cpu_baseline", "e2e", "clocks", "per_N", "served", "gpu_launches"):
        assert k in line, k
    assert line["dtype"] == "f32" and "sweep" in line["config"]["workload"]
    assert line["roofline"]["traffic"] == 242854144 and line["roofline"]["frac"] > 0
    assert line["cpu_baseline"]["cores"] == 16 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 123456789
    assert len(line["per_N"]) == 8 and all(len(v) == 2 for v in line["per_N"].values())
    for k in ("p50_s", "p99_s", "plain_p50_s", "plain_p99_s"):
        assert line["served"][k] > 0
    assert line["large_elastic"]["hbm_frac"] > 0
    # a run with legs switched off still gives a complete, short line
    d = _canned_detail()
    d.update(cpu_baseline=None, e2e=None, served=None, large_elastic=None, fp32_peak=None)
    line = bench.headline(d)
    assert len(json.dumps(line)) < 2000 and line["e2e"] is None


def test_fp32_peak_source():
    """The ALU denominator is the measured FMA throughput when there is one,
    else the unit-count figure (152 SMs x 128 lanes x 2 x 2070 MHz)."""
    p = bench.peaks({"tflops": 77.7})
    assert p["fp32_tflops"] == 77.7 and p["fp32_source"] == "measured"
    q = bench.peaks(None)
    assert abs(q["fp32_tflops"] - 152 * 128 * 2 * 2.070e-3) < 1e-9 and q["fp32_source"] == "unit count"
    assert abs(p["fp32_unit_count_tflops"] - q["fp32_tflops"]) < 1e-12
