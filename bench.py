"""Benchmark: DG node-field updates/s of the fused RHS + AB3 step on GB300.

Workload: the acoustic degree sweep N = 1..8, one jittered Kuhn cube mesh of
~2 M nodes per degree (rho, c ~ U[1,3], rigid walls, upwind flux, random
initial state), FP32.  One bench step = one AB3 time step on each of the
eight meshes (one or two kernel launches each), the meshes on streams of
their own so that their kernels overlap (joined once after the timed steps;
``--join-every-step``: after each; ``--sequential``: one after another on one
stream).  value = sum over meshes of K*Np*Nf field updates / device
time of the step.  The eight meshes hold ~1.3 GB, so consecutive steps on
one mesh never find its state in L2.  The per-degree table and the roofline
come from a second pass over the same steps that times each degree alone.

Before the timed region every mesh's kernel variant is autotuned.

Extra keys: per_N (time, updates/s, algorithmic GB/s and GFLOP/s, kernel
variant per degree), sweeps (the same per-degree table for the acoustic
bf16x6 tensor-core mode and for the elastic model in FP32 and bf16x6, each
timed over --sweep-steps steps; bf16x6 results are compared with the FP32
path on the same meshes), roofline (dominant kernel), cpu_baseline (FP64 oracle on
the host), e2e (same metric through the C ABI with pinned host buffers,
copies inside the timed region), served (64 acoustic shots, N in {3,5,7},
500 steps, Poisson arrivals at 0.7 x the batched capacity: p50/p99 latency,
against the same requests solved one at a time), clocks (nvidia-smi samples
during the timed region).

Multi-GPU: replicas only (the single-GPU path does not shard); each rank runs
the whole sweep and value = sum of the ranks' updates / max rank time.

``--impl reference`` times the FP64 oracle (the reference arm) instead.
``--model elastic`` times the elastic sweep meshes in the main loop instead of
the acoustic ones (used to profile the elastic kernels on their own).
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DG node-field updates/s and % HBM/FP32 roofline per N; served p50/p99 solve latency"
UNIT = "node-field updates/s"
WORKLOAD = ("acoustic DG sweep N=1..8, jittered Kuhn cube meshes of ~2M nodes per degree, "
            "rho,c~U[1,3], rigid walls, upwind flux, FP32, AB3")
WORKLOAD_ELASTIC = ("elastic DG sweep N=1..8, jittered Kuhn cube meshes of ~2M nodes per degree, "
                    "two isotropic layers (lambda,mu,rho~U[1,2] below z=1/2, U[2,3] above), "
                    "traction-free walls, upwind flux, FP32, AB3")
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def peaks(fp32=None):
    """Roofline denominators: HBM from MEASURED_PEAKS.json (burst copy), FP32
    from the live FMA microbenchmark (dg_fp32_peak, the better of its scalar
    and packed forms) when given, else the unit-count derivation at the
    maximum SM clock, which is also kept as a cross-check."""
    p = {"hbm_gbs": 6758.9, "source": "fallback"}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        p["hbm_gbs"] = float(m["hbm_gbs"])
        p["source"] = "measured"
    except Exception:
        pass
    p["fp32_unit_count_tflops"] = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    if fp32 and fp32.get("tflops"):
        p["fp32_tflops"] = fp32["tflops"]
        p["fp32_source"] = "measured"
    else:
        p["fp32_tflops"] = p["fp32_unit_count_tflops"]
        p["fp32_source"] = "unit count"
    return p


def measure_fp32_peak(P, stream, device):
    """FP32 FMA throughput measured on this GPU (scalar and packed FMA forms,
    best launch of each) with the SM clock sampled while it runs."""
    with ClockSampler(device) as clk:
        t_wait = time.perf_counter()
        while clk.proc and not clk.lines and time.perf_counter() - t_wait < 3.0:
            time.sleep(0.01)
        t0 = time.perf_counter()
        r = P.fp32_peak(stream.cuda_stream, reps=10, target_ms=40.0)
        t1 = time.perf_counter()
    c = clk.summary(t0, t1)
    r["tflops"] = max(r["scalar_tflops"], r["packed_tflops"])
    r["sm_mhz"] = c["sm_mhz"]
    r["reasons"] = c["reasons"]
    return r


def algorithmic(model, N, K):
    """Bytes and FLOPs of one fused step over K elements (unpadded, estimated
    convention): AB3 state 5 arrays x 4 B per field-node (read q^m, r^m-1,
    r^m-2; write q^m+1, r^m) + 84 B of element records; FLOPs = 2 x the
    multiply-adds of the operator products + 8 per field-node for AB3."""
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nfp = (N + 1) * (N + 2) // 2
    Nf = 4 if model == "acoustic" else 9
    byt = K * (20 * Nf * Np + 84)
    if model == "acoustic":
        mac = 6 * Np * Np + 16 * Np * Nfp
    else:
        mac = 18 * Np * Np + 36 * Np * Nfp
    flop = K * (2 * mac + 8 * Nf * Np)
    return byt, flop


def executed_flops(model, N, K, factored):
    """FLOPs the kernels execute (same terms as `algorithmic`).  Factored
    paths lift surface streams instead of every penalty field: acoustic, two
    streams per face node, the velocity lift rebuilt from the face normals
    (12 multiply-adds per node); elastic, six streams (Fscale p_v and
    Fscale dv), the stress lift folded face by face from lambda, mu and the
    normal (16 multiply-adds per face and node: n.W, three diagonal and three
    off-diagonal terms)."""
    byt, flop = algorithmic(model, N, K)
    if not factored:
        return flop
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nfp = (N + 1) * (N + 2) // 2
    if model == "acoustic":
        return K * (2 * (6 * Np * Np + 8 * Np * Nfp + 12 * Np) + 8 * 4 * Np)
    return K * (2 * (18 * Np * Np + 24 * Np * Nfp + 64 * Np) + 8 * 9 * Np)


def is_factored(model, g, precision, strategy):
    """Whether g's step lifts surface streams (see `executed_flops`): the
    library route always; the fused FP32 step for every acoustic kernel and
    for the elastic split step; neither the plain route nor the tensor-core
    modes (their front halves lift every penalty field)."""
    if strategy == "plain":
        return False
    if strategy == "library":
        return True
    if precision != "fp32":
        return False
    return model == "acoustic" or g.kernel_info()["split"] == 1


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    INTERVAL_MS = 50

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []  # (host time of arrival, csv line)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0=None, t1=None):
        """Median SM clock, maximum clock and throttle reasons of the samples
        that arrived in [t0, t1 + one interval] (all samples if none did)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if t0 is not None:
            inside = [x for x in lines if t0 <= x[0] <= t1 + self.INTERVAL_MS / 1e3]
            lines = inside or lines
        for _, ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(t_local, updates, world):
    """Job time = max over ranks, job updates = sum over ranks (replicas)."""
    if world <= 1:
        return t_local, float(updates)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([t_local], dtype=torch.float64, device=dev)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def served_benchmark(P, count=64, steps=500, seed=1004, max_n=32, rates=(0.5, 0.9), max_batch=8):
    """Served stream: acoustic shots with Poisson arrivals at 0.7 x the batched
    capacity (measured first with every request submitted at once), p50/p99 of
    submit -> result latency, against the same requests run one at a time; and
    a sweep of the arrival rate (`rates` x capacity, batched server runs; the
    one-at-a-time latencies there follow from a FIFO queue over the service
    times measured at 0.7, since that executor runs one request at a time)."""
    import workloads as W
    from workloads.configs import request_mesh
    reqs = W.config4_requests(count, seed=seed)
    prepared = []
    for r in reqs:
        r = dict(r, n=min(r["n"], max_n), steps=steps)
        verts, tets, coeffs = request_mesh(r)
        dt = P.suggest_dt(verts, tets, coeffs, r["N"], "acoustic", 0.4)
        amp = W.ricker(np.arange(steps) * dt, f0=4.0)
        prepared.append((r, verts, tets, coeffs, dt, amp))
    work = sum(t.shape[0] * (r["N"] + 1) * (r["N"] + 2) * (r["N"] + 3) // 6 * 4 * steps
               for r, v, t, c, d, a in prepared)

    def run_server(arrivals):
        srv = P.Server(max_batch=max_batch)
        t0 = time.perf_counter()
        pending = {}
        lat = []
        i = 0
        while i < len(prepared) or pending:
            now = time.perf_counter() - t0
            while i < len(prepared) and arrivals[i] <= now:
                r, v, t, c, d, a = prepared[i]
                pending[srv.submit(v, t, c, r["N"], dt=d, nsteps=steps, source=r["source"], amp=a)] = i
                i += 1
            for tk in list(pending):
                res = srv.poll(tk)
                if res is not None:
                    lat.append(res[1])
                    del pending[tk]
            time.sleep(0.0005)
        makespan = time.perf_counter() - t0
        launches = srv.stats()["launches"]
        srv.close()
        return makespan, lat, launches

    # capacity: everything at t = 0
    mk0, _, _ = run_server([0.0] * len(prepared))
    capacity = len(prepared) / mk0
    rate = 0.7 * capacity
    rng = np.random.default_rng(seed)
    arr = np.cumsum(rng.exponential(1.0 / rate, size=len(prepared)))
    mk, lat, launches = run_server(list(arr))
    # plain: the same requests one at a time through dg_step, in arrival order
    t0 = time.perf_counter()
    plain_lat, service = [], []
    for (r, v, t, c, d, a), ta in zip(prepared, arr):
        while time.perf_counter() - t0 < ta:
            time.sleep(0.0005)
        ts = time.perf_counter()
        g = P.Solver(v, t, c, r["N"], "acoustic", dt=d)
        g.set_source(r["source"], a)
        g.step(steps)
        g.get_state()
        g.close()
        service.append(time.perf_counter() - ts)
        plain_lat.append(time.perf_counter() - t0 - ta)
    mk_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    for (r, v, t, c, d, a) in prepared:
        g = P.Solver(v, t, c, r["N"], "acoustic", dt=d)
        g.set_source(r["source"], a)
        g.step(steps)
        g.get_state()
        g.close()
    mk_plain0 = time.perf_counter() - t0
    q = lambda x, p: float(np.percentile(np.asarray(x), p))

    def fifo(arrivals):
        free, out = 0.0, []
        for ta, sv in zip(arrivals, service):
            free = max(ta, free) + sv
            out.append(free - ta)
        return out

    sweep = [{"rate_frac": 0.7, "p50_s": q(lat, 50), "p99_s": q(lat, 99), "makespan_s": mk,
              "plain_p50_s": q(plain_lat, 50), "plain_p99_s": q(plain_lat, 99)}]
    for frac in rates:
        af = np.cumsum(np.random.default_rng(seed + int(1000 * frac)).exponential(1.0 / (frac * capacity),
                                                                                  size=len(prepared)))
        mkf, latf, _ = run_server(list(af))
        pl = fifo(af)
        sweep.append({"rate_frac": frac, "p50_s": q(latf, 50), "p99_s": q(latf, 99), "makespan_s": mkf,
                      "plain_p50_s": q(pl, 50), "plain_p99_s": q(pl, 99)})
    sweep.sort(key=lambda x: x["rate_frac"])
    return {"requests": len(prepared), "steps": steps, "degrees": [3, 5, 7],
            "mesh_tets": [int(p[2].shape[0]) for p in prepared],
            "capacity_req_per_s": capacity, "arrival_rate_req_per_s": rate,
            "p50_s": q(lat, 50), "p99_s": q(lat, 99), "makespan_s": mk,
            "batched_all_at_once_makespan_s": mk0,
            "batched_updates_per_s": work / mk0, "launches": launches,
            "plain_p50_s": q(plain_lat, 50), "plain_p99_s": q(plain_lat, 99), "plain_makespan_s": mk_plain,
            "plain_all_at_once_makespan_s": mk_plain0, "plain_updates_per_s": work / mk_plain0,
            "rate_sweep": sweep, "max_batch": max_batch,
            "note": "latency = submit to result in host memory (includes host set-up of the request); "
                    "rate_sweep plain latencies: FIFO over the measured one-at-a-time service times"}


def build_meshes(model, Ns):
    import workloads as W
    out = []
    for N in Ns:
        cfg = W.sweep_mesh(model, N)
        out.append(cfg)
    return out


def cpu_baseline(model="acoustic", Ns=(2, 4), steps=1, steps_mt=0):
    """FP64 oracle on the full ~2 M-node meshes of the listed degrees (a
    bounded sample of the sweep): `steps` AB3 steps on one thread and, if
    steps_mt > 0, `steps_mt` steps on every host core (the oracle's RHS of
    element chunks in a thread pool -- its einsum loops release the GIL --
    joined for the same AB3 stepper; the oracle itself is unchanged)."""
    code = r"""
import json, sys, time, os
sys.path.insert(0, %r)
import numpy as np
from concurrent.futures import ThreadPoolExecutor
import workloads as W
from oracle.dg import Solver, AB3Stepper

class Chunked:
    def __init__(self, S, T):
        self.S, self.pool = S, ThreadPoolExecutor(T)
        self.chunks = np.array_split(np.arange(S.K), T)
    def rhs(self, q, step=None):
        return np.concatenate(list(self.pool.map(lambda E: self.S.rhs(q, step=step, elems=E), self.chunks)))

T = os.cpu_count() or 1
res, res_mt = [], []
for N in %r:
    cfg = W.sweep_mesh(%r, N)
    S = Solver(%r, N, cfg["verts"], cfg["tets"], cfg["coeffs"])
    q = W.random_state(S.K, S.Nf, S.ref.Np, seed=0)
    if %d > 0:
        st = AB3Stepper(S, q, 1e-6)
        t0 = time.perf_counter()
        st.step(%d)
        res.append((S.K * S.ref.Np * S.Nf * %d, time.perf_counter() - t0))
    if %d > 0:
        st = AB3Stepper(Chunked(S, T), q, 1e-6)
        t0 = time.perf_counter()
        st.step(%d)
        res_mt.append((S.K * S.ref.Np * S.Nf * %d, time.perf_counter() - t0))
print(json.dumps({"one": res, "all": res_mt, "threads": T}))
""" % (ROOT, tuple(Ns), model, model, steps, steps, steps, steps_mt, steps_mt, steps_mt)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": p.stderr[-500:]}
    out = json.loads(p.stdout.strip().splitlines()[-1])
    one = None if not out["one"] else {
           "value": sum(r[0] for r in out["one"]) / sum(r[1] for r in out["one"]), "unit": UNIT, "cores": 1,
           "kind": "oracle",
           "sample": "FP64 oracle, %d AB3 step(s) on the full %s meshes for N=%s, single thread"
                     % (steps, model, ",".join(str(n) for n in Ns)),
           "seconds": round(sum(r[1] for r in out["one"]), 2)}
    if not out["all"]:
        return one
    t = sum(r[1] for r in out["all"])
    return {"value": sum(r[0] for r in out["all"]) / t, "unit": UNIT, "cores": out["threads"], "kind": "oracle",
            "sample": "FP64 oracle, %d AB3 step(s) on the full %s meshes for N=%s, RHS of element chunks on "
                      "%d threads" % (steps_mt, model, ",".join(str(n) for n in Ns), out["threads"]),
            "seconds": round(t, 2), "single_core": one}


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle as it stands on the host cores.  The
    N = 2 sweep mesh and its oracle are built once; every bench step is then
    one AB3 step (the oracle's stepper and RHS) on a fixed subset of the
    mesh's elements, its RHS in element chunks on every core, the subset sized
    so that the W + K steps take about two minutes.  value = median over the K
    timed steps of the subset's node-field updates per second."""
    if rank != 0:
        return
    t_start = time.time()
    budget_s = 120.0
    code = r"""
import json, sys, time, os
sys.path.insert(0, %r)
import numpy as np
from concurrent.futures import ThreadPoolExecutor
import workloads as W
from oracle.dg import Solver, AB3Stepper

T = os.cpu_count() or 1
cfg = W.sweep_mesh("acoustic", 2)
S = Solver("acoustic", 2, cfg["verts"], cfg["tets"], cfg["coeffs"])
q = W.random_state(S.K, S.Nf, S.ref.Np, seed=0)
pool = ThreadPoolExecutor(T)

class Subset:
    # the oracle's RHS rows of elements E; the other elements keep their state
    def __init__(self, E):
        self.E, self.chunks = E, np.array_split(E, T)
    def rhs(self, qs, step=None):
        q[self.E] = qs
        return np.concatenate(list(pool.map(lambda c: S.rhs(q, step=step, elems=c), self.chunks)))

steps, warmup, step_s = %d, %d, %r
probe = Subset(np.arange(min(S.K, 1024 * T)))
probe.rhs(q[probe.E])                                     # first call: one-off start-up costs
t0 = time.perf_counter()
probe.rhs(q[probe.E])
rate = len(probe.E) / (time.perf_counter() - t0)          # elements per second
n = int(min(S.K, max(T, rate * step_s)))
for _ in range(2):                                        # rescale at the step's own size
    sub = Subset(np.arange(n))
    t0 = time.perf_counter()
    sub.rhs(q[sub.E])
    n = int(min(S.K, max(T, n * step_s / (time.perf_counter() - t0))))
E = np.arange(n)
st = AB3Stepper(Subset(E), q[E].copy(), 1e-6)
ts = []
for s in range(warmup + steps):
    t0 = time.perf_counter()
    st.step(1)
    if s >= warmup:
        ts.append(time.perf_counter() - t0)
print(json.dumps({"n": n, "K": S.K, "upd": n * S.ref.Np * S.Nf, "ts": ts, "threads": T}))
""" % (ROOT, args.steps, args.warmup, min(0.5, budget_s / max(1, args.steps + args.warmup)))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + p.stderr[-300:]}), flush=True)
        return
    out = json.loads(p.stdout.strip().splitlines()[-1])
    v = statistics.median(out["upd"] / t for t in out["ts"]) if out["ts"] else None
    sample = ("FP64 oracle, one AB3 step per bench step on %d of the %d elements of the acoustic N=2 sweep "
              "mesh, RHS of element chunks on %d threads" % (out["n"], out["K"], out["threads"]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "ms_per_step": statistics.median(out["ts"]) * 1e3 if out["ts"] else None,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": out["threads"], "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(time.time() - t_start, 1)}
    print(json.dumps(line), flush=True)


def make_solvers(P, cfgs, model, precision, stream, tune, variants=None, strategy="fused"):
    solvers = []
    tune = tune and strategy == "fused"
    for i, cfg in enumerate(cfgs):
        N = cfg["N"]
        dt = P.suggest_dt(cfg["verts"], cfg["tets"], cfg["coeffs"], N, model, 0.4)
        g = P.Solver(cfg["verts"], cfg["tets"], cfg["coeffs"], N, model, dt=dt,
                     stream=stream.cuda_stream, precision=precision, strategy=strategy)
        q = np.random.default_rng(N).uniform(-1, 1, size=g.shape).astype(np.float32)
        g.set_state(q)
        if variants is not None and strategy == "fused":
            g.set_variant(variants[i])
        elif tune:
            g.autotune(5)
        solvers.append(g)
    return solvers


def per_degree(model, g, ms, pk, tensor=False, factored=False):
    """One row of the per-degree table: algorithmic bytes and FLOPs over the
    measured time, and the roofline that bounds the path (tensor-core modes:
    the contraction ceiling is far above the FP32 one, so HBM)."""
    byt, flop = algorithmic(model, g.N, g.K)
    gbs = byt / (ms * 1e-3) / 1e9
    gfl = flop / (ms * 1e-3) / 1e9
    ridge = pk["fp32_tflops"] * 1e3 / pk["hbm_gbs"]
    bound = "hbm" if (tensor or flop / byt < ridge) else "alu"
    frac = gbs / pk["hbm_gbs"] if bound == "hbm" else gfl / (pk["fp32_tflops"] * 1e3)
    efl = executed_flops(model, g.N, g.K, factored) / (ms * 1e-3) / 1e9
    return {"K": g.K, "nodes": g.K * g.Np, "ms": round(ms, 5), "kernel": g.kernel_info(),
            "updates_per_s": g.K * g.Np * g.Nf / (ms * 1e-3),
            "alg_GBs": round(gbs, 1), "alg_GFLOPs": round(gfl, 1), "exec_GFLOPs": round(efl, 1),
            "bound": bound, "roofline_frac": round(frac, 4)}


def time_sweep(solvers, steps, stream):
    """Per-degree mean step time (CUDA events on the solvers' stream)."""
    import torch
    for g in solvers:
        g.step(2)
    torch.cuda.synchronize()
    out = []
    for g in solvers:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.step(steps)
        e1.record(stream)
        e1.synchronize()
        g.sync()
        out.append(e0.elapsed_time(e1) / steps)
    return out


def extra_sweeps(P, args, acoustic_cfgs, stream, pk):
    """Acoustic bf16x6, library route and plain route on the headline meshes;
    elastic FP32, bf16x6, library and plain routes on the elastic sweep meshes
    (lambda, mu, rho ~ U[1,3] with a two-layer jump).  The state after
    --sweep-steps steps of every non-reference sweep is compared with the
    fused FP32 path's (relative L2)."""
    Ns = [cfg["N"] for cfg in acoustic_cfgs]
    res = {}
    for model, cfgs in (("acoustic", acoustic_cfgs), ("elastic", None)):
        if cfgs is None:
            cfgs = build_meshes(model, Ns)
        precs = (("bf16x6", "fused"), ("fp32", "library"), ("fp32", "plain")) if model == "acoustic" else \
            (("fp32", "fused"), ("bf16x6", "fused"), ("fp32", "library"), ("fp32", "plain"))
        ref_states = {}
        if model == "acoustic":
            ref = make_solvers(P, cfgs, model, "fp32", stream, False)
            for g in ref:
                g.step(2 + args.sweep_steps)  # as many steps as time_sweep takes
                g.sync()
                ref_states[g.N] = g.get_state()
                g.close()
        for prec, strat in precs:
            solvers = make_solvers(P, cfgs, model, prec, stream, not args.no_tune, strategy=strat)
            ms = time_sweep(solvers, args.sweep_steps, stream)
            rows = {}
            for g, t in zip(solvers, ms):
                rows[str(g.N)] = per_degree(model, g, t, pk, tensor=prec != "fp32",
                                            factored=is_factored(model, g, prec, strat))
                rows[str(g.N)]["strategy"] = strat
                if strat != "fused":
                    del rows[str(g.N)]["kernel"]
            if prec != "fp32" or model == "elastic" or strat != "fused":
                # states after 2 + sweep_steps steps from the same initial state
                for g in solvers:
                    if prec == "fp32" and strat == "fused":
                        ref_states[g.N] = g.get_state()
                    elif g.N in ref_states:
                        a = g.get_state().astype(np.float64)
                        b = ref_states[g.N].astype(np.float64)
                        rows[str(g.N)]["rel_l2_vs_fp32"] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
            tot = sum(ms)
            upd = sum(g.K * g.Np * g.Nf for g in solvers)
            key = "%s_%s" % (model, prec) if strat == "fused" else "%s_%s_%s" % (model, strat, prec)
            res[key] = {"per_N": rows, "ms_per_sweep_step": round(tot, 4),
                                            "updates_per_s": upd / (tot * 1e-3), "steps": args.sweep_steps}
            for g in solvers:
                g.close()
    return res


def run(args, rank, world, local_rank):
    import torch
    import paper_1602_07997_gb300 as P

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if args.large_only:
        # the large elastic workload alone (e.g. to capture its kernels)
        lg = large_elastic(P, args, torch.cuda.Stream(device=dev), peaks(None))
        if rank == 0:
            print(json.dumps({"large_elastic": lg}), flush=True)
        return
    model = args.model
    Ns = [int(x) for x in args.degrees.split(",")]
    stream = torch.cuda.Stream(device=dev)
    cfgs = build_meshes(model, Ns)
    variants = [int(x) for x in args.variants.split(",")] if args.variants else None
    if variants is not None and len(variants) != len(Ns):
        raise SystemExit("--variants needs one index per degree")
    solvers = make_solvers(P, cfgs, model, args.precision, stream, not args.no_tune, variants, args.strategy)
    torch.cuda.synchronize()
    fp32 = None if args.no_peak else measure_fp32_peak(P, stream, local_rank)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # The meshes of the sweep are independent problems: they run on streams
    # of their own (forked from the timing stream, largest degree first, and
    # joined to it after the timed steps; --join-every-step joins them after
    # every sweep step), so that one degree's kernels fill the SMs that
    # another's leave idle at its tail.  --sequential runs them one after
    # another on one stream instead.  The per-degree times (per_N, the
    # roofline) come from a separate sequential pass over the same number of
    # steps, each degree timed alone.
    order = sorted(range(len(solvers)), key=lambda i: -solvers[i].N)
    conc = not args.sequential and len(solvers) > 1
    sstreams = [torch.cuda.Stream(device=dev) for _ in solvers] if conc else None
    e_fork = torch.cuda.Event()
    e_join = [torch.cuda.Event() for _ in solvers]

    def sweep_steps(n):
        if not conc:
            for _ in range(n):
                for g in solvers:
                    g.step(1)
            return
        for _ in range(n if args.join_every_step else 1):
            e_fork.record(stream)
            for i in order:
                sstreams[i].wait_event(e_fork)
                solvers[i].step(1 if args.join_every_step else n)
                e_join[i].record(sstreams[i])
            for i in order:
                stream.wait_event(e_join[i])

    def on_streams(own):
        for i, g in enumerate(solvers):
            g.set_stream((sstreams[i] if own else stream).cuda_stream)

    if conc:
        on_streams(True)
    # warm-up
    sweep_steps(args.warmup)
    barrier()
    nN = len(solvers)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(nN)] for _ in range(args.steps)]
    e_all0, e_all1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        # untimed steps until the sampler is live (at most 3 s), so that its
        # samples cover the timed region
        t_wait = time.perf_counter()
        while clk.proc and not clk.lines and time.perf_counter() - t_wait < 3.0:
            sweep_steps(1)
            torch.cuda.synchronize()
        barrier()
        lc0 = [g.launch_count() for g in solvers]
        t0 = time.perf_counter()
        e_all0.record(stream)
        sweep_steps(args.steps)
        e_all1.record(stream)
        barrier()
        t1 = time.perf_counter()
        # kernels of the library launched in the timed region, as the handles count them
        launches = sum(g.launch_count() - c for g, c in zip(solvers, lc0))
        # per-degree pass: every degree alone on the timing stream
        if conc:
            on_streams(False)
        for s in range(args.steps):
            for i, g in enumerate(solvers):
                ev[s][i][0].record(stream)
                g.step(1)
                ev[s][i][1].record(stream)
        barrier()
    clocks = clk.summary(t0, t1)
    total_ms = e_all0.elapsed_time(e_all1)
    per_ms = [statistics.mean(ev[s][i][0].elapsed_time(ev[s][i][1]) for s in range(args.steps))
              for i in range(nN)]
    for g in solvers:
        g.sync()
    updates = sum(g.K * g.Np * g.Nf for g in solvers) * args.steps
    t_local = total_ms / 1e3
    t_job, upd_job = aggregate(t_local, updates, world)
    value = upd_job / t_job

    pk = peaks(fp32)
    per_N = {}
    dom = None
    for g, ms in zip(solvers, per_ms):
        row = per_degree(model, g, ms, pk, tensor=args.precision != "fp32",
                         factored=is_factored(model, g, args.precision, args.strategy))
        per_N[str(g.N)] = row
        if dom is None or ms > dom[1]:
            byt, flop = algorithmic(model, g.N, g.K)
            dom = (g, ms, byt, flop, row["bound"])
    g, ms, byt, flop, bound = dom
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        ent = tr.get("%s_N%d_%s_v%d" % (model, g.N, args.precision, g.kernel_info()["variant"]))
        if ent and ent.get("kernel_rev") == kernel_rev():
            traffic = ent["dram_bytes_per_launch"]
    except Exception:
        pass
    if bound == "hbm":
        roof = {"bound": "hbm", "achieved": byt / (ms * 1e-3) / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s"}
    else:
        roof = {"bound": "alu", "achieved": flop / (ms * 1e-3) / 1e12, "peak": pk["fp32_tflops"],
                "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if bound != "hbm":
        # the same step against the FLOPs the kernels execute (surface streams lifted)
        roof["exec_achieved"] = (executed_flops(model, g.N, g.K, is_factored(model, g, args.precision, args.strategy))
                                 / (ms * 1e-3) / 1e12)
        roof["exec_frac"] = roof["exec_achieved"] / roof["peak"]
    roof["traffic"] = traffic
    ki = g.kernel_info()
    roof["kernel"] = ("dg_step_kernel<%s, N=%d, EB=%d, TN=%d> (variant %d)"
                      % (model, g.N, ki["block_elems"], ki["tile_elems"], ki["variant"]) if not ki["split"] else
                      "split step, %s N=%d (front half + %s GEMM, variant %d)"
                      % (model, g.N, "tcgen05" if ki["split"] == 2 else "FP32", ki["variant"]))
    roof["kernel_short"] = ("fused %s N=%d v%d" % (model, g.N, ki["variant"]) if not ki["split"] else
                            "split %s N=%d (%s GEMM) v%d" % (model, g.N, "tcgen05" if ki["split"] == 2 else "FP32",
                                                            ki["variant"]))
    roof["peak_source"] = ("MEASURED_PEAKS.json hbm_gbs (burst copy)" if bound == "hbm" else
                           "measured: dg_fp32_peak FMA microbenchmark" if pk["fp32_source"] == "measured" else
                           "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz")

    # e2e through the C ABI: pinned host buffers, H2D of the state and D2H of the
    # result inside the timed region, every step; each mesh on a stream of its
    # own with asynchronous (stream-ordered) transfers, so that one mesh's
    # copies overlap another's kernels, and every mesh synchronised at the end
    # of the step
    e2e = None
    if not args.no_e2e:
        pinned = [torch.empty(g.shape, dtype=torch.float32).pin_memory() for g in solvers]
        e_streams = [torch.cuda.Stream(device=dev) for _ in solvers]
        for p, g, st in zip(pinned, solvers, e_streams):
            g.set_stream(st.cuda_stream)
            g.get_state(p)
        e_steps = max(1, min(args.steps, 5))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            for i in order:  # largest degree first, as in the timed sweep
                p, g = pinned[i], solvers[i]
                g.set_state(p, asynchronous=True)
                g.step(1)
                g.get_state(p, asynchronous=True)
            for g in solvers:
                g.sync()
        barrier()
        te = time.perf_counter() - t0
        e_upd = sum(g.K * g.Np * g.Nf for g in solvers) * e_steps
        nbytes = sum(g.size * 4 for g in solvers)
        e2e = {"value": e_upd * world / te, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": e_steps,
               "note": "per step: for every mesh, on its own stream, dg_set_state(pinned host q, "
                       "asynchronous) + dg_step(1) + dg_get_state(pinned host, asynchronous); then dg_sync of "
                       "every mesh (host wall clock)"}

    for s in solvers:
        s.close()
    sweeps = None
    if rank == 0 and not args.no_sweeps:
        sweeps = extra_sweeps(P, args, cfgs, stream, pk)

    cpu = None
    if rank == 0 and not args.no_cpu and world == 1:
        cpu = cpu_baseline(model, Ns=(2, 4), steps=6, steps_mt=48)  # about 10 s of oracle work each

    served = None
    if rank == 0 and not args.no_serve:
        served = served_benchmark(P, count=args.serve_requests, steps=args.serve_steps,
                                  max_batch=args.serve_max_batch)

    large = None
    if rank == 0 and not args.no_large:
        large = large_elastic(P, args, stream, pk)

    if rank == 0:
        detail = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                  "warmup": args.warmup, "ms_per_step": t_job * 1e3 / args.steps, "higher_is_better": True,
                  "scaling": "weak", "vs_baseline": None,
                  "dtype": "f32" if args.precision == "fp32" else args.precision + " (f32 accumulate)",
                  "data": "synthetic",
                  "config": {"workload": WORKLOAD if model == "acoustic" else WORKLOAD_ELASTIC, "degrees": Ns,
                             "meshes": {str(g.N): g.K for g in solvers},
                             "l2": "inputs larger than L2: the 8 meshes hold ~1.3 GB, each ~130 MB",
                             "parallelism": "replicas" if world > 1 else "single GPU",
                             "sweep": (("concurrent: one stream per degree, largest degree first, joined "
                                        + ("every step" if args.join_every_step else "after the timed steps"))
                                       if conc else "sequential: one stream")},
                  "sequential_ms_per_step": round(sum(per_ms), 5),
                  "gpu_launches": launches, "roofline": roof, "per_N": per_N, "sweeps": sweeps,
                  "cpu_baseline": cpu, "e2e": e2e, "served": served, "large_elastic": large, "clocks": clocks,
                  "fp32_peak": fp32, "peaks": pk}
        print(json.dumps({"bench_detail": detail}), flush=True)
        print(json.dumps(headline(detail)), flush=True)


def _r(x, d=4):
    """Round to d significant digits (None passes through)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return float("%.*g" % (d, x))


def headline(d):
    """The final stdout line: the contract's keys and a short summary of the
    detail line printed before it (kept well under 2 KB, so that a reader
    that keeps only the end of the output still has all of it)."""
    roof = d["roofline"]
    line = {k: d[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "gpu_launches")}
    line["value"] = _r(line["value"], 6)
    line["ms_per_step"] = _r(line["ms_per_step"], 5)
    c = d["config"]
    line["config"] = {"workload": c["workload"], "degrees": c["degrees"], "l2": "inputs > L2 (~1.3 GB)",
                      "parallelism": c["parallelism"], "sweep": c.get("sweep", "")[:10]}
    line["sequential_ms_per_step"] = d.get("sequential_ms_per_step")
    line["roofline"] = {"bound": roof["bound"], "achieved": _r(roof["achieved"]), "peak": _r(roof["peak"]),
                        "unit": roof["unit"], "frac": _r(roof["frac"], 3), "traffic": roof.get("traffic"),
                        "kernel": roof.get("kernel_short"),
                        "peak_source": (roof.get("peak_source") or "").split(":")[0]}
    cpu = d.get("cpu_baseline")
    if cpu:
        line["cpu_baseline"] = {"value": _r(cpu.get("value")), "unit": cpu.get("unit"), "cores": cpu.get("cores"),
                                "kind": cpu.get("kind"), "sample": cpu.get("sample_short", cpu.get("sample")),
                                "one_core": _r((cpu.get("single_core") or {}).get("value"))}
    else:
        line["cpu_baseline"] = None
    e = d.get("e2e")
    line["e2e"] = None if not e else {"value": _r(e["value"]), "unit": e["unit"],
                                      "h2d_bytes_per_step": e["h2d_bytes_per_step"],
                                      "d2h_bytes_per_step": e["d2h_bytes_per_step"]}
    ck = d.get("clocks") or {}
    line["clocks"] = {"sm_mhz": ck.get("sm_mhz"), "sm_max_mhz": ck.get("sm_max_mhz"), "reasons": ck.get("reasons")}
    # per degree: [ms per step, roofline fraction] (HBM at the degrees whose
    # operational intensity is below the ridge, else FP32)
    line["per_N"] = {n: [_r(r["ms"]), _r(r["roofline_frac"], 3)] for n, r in d["per_N"].items()}
    pk = d.get("fp32_peak")
    if pk:
        line["fp32_peak_tflops"] = {"scalar": _r(pk["scalar_tflops"]), "packed": _r(pk["packed_tflops"]),
                                    "sm_mhz": pk.get("sm_mhz")}
    sv = d.get("served")
    if sv:
        line["served"] = {k: _r(sv[k]) for k in ("p50_s", "p99_s", "plain_p50_s", "plain_p99_s",
                                                 "batched_all_at_once_makespan_s", "plain_all_at_once_makespan_s")}
        line["served"]["max_batch"] = sv.get("max_batch")
    lg = d.get("large_elastic")
    if lg:
        line["large_elastic"] = {"ms": _r(lg["ms"]), "updates_per_s": _r(lg["updates_per_s"]),
                                 "hbm_frac": _r(lg["hbm_frac"], 3), "alu_frac": _r(lg["alu_frac"], 3),
                                 "traffic": lg.get("traffic")}
    return line


def large_elastic(P, args, stream, pk):
    """The large elastic workload: N = 7 on the n = 28 Kuhn mesh (131 712
    tets, 15.8 M nodes, layered lambda, mu, rho with +-30 % per tet), the
    autotuned FP32 step, CUDA events over --large-steps steps after three
    warm-up steps; algorithmic GB/s and GFLOP/s against both peaks."""
    import workloads as W
    cfg = W.config5_elastic_large()
    fixed = [args.large_variant] if args.large_variant >= 0 else None
    g = make_solvers(P, [cfg], "elastic", "fp32", stream, not args.no_tune, fixed)[0]
    ms = time_sweep([g], args.large_steps, stream)[0]
    byt, flop = algorithmic("elastic", g.N, g.K)
    ki = g.kernel_info()
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            ent = json.load(f).get("elastic_N7_fp32_v%d_large" % ki["variant"])
        if ent and ent.get("kernel_rev") == kernel_rev():
            traffic = ent["dram_bytes_per_launch"]
    except Exception:
        pass
    out = {"K": g.K, "nodes": g.K * g.Np, "N": g.N, "ms": ms, "steps": args.large_steps,
           "updates_per_s": g.K * g.Np * g.Nf / (ms * 1e-3),
           "alg_GBs": byt / (ms * 1e-3) / 1e9, "alg_GFLOPs": flop / (ms * 1e-3) / 1e9,
           "hbm_frac": byt / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
           "alu_frac": flop / (ms * 1e-3) / 1e12 / pk["fp32_tflops"],
           "kernel": ki, "traffic": traffic,
           "state_bytes": 5 * 4 * g.K * g.Np * g.Nf}
    g.close()
    return out


KERNEL_SOURCES = ("dg_args.h", "dg_kernels.cuh", "dg_gemm.cuh", "dg_tc.cuh", "dg_launch.cuh", "dg_dispatch.cu",
                  "dg_kernels_acoustic.cu", "dg_kernels_elastic.cu", "dg_kernels_tc_acoustic.cu",
                  "dg_kernels_tc_elastic.cu")


def kernel_rev():
    """Hash of the step kernels' sources without their comments (a traffic
    figure is only valid for the code it was measured on)."""
    import hashlib
    import re
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1602_07997_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f), encoding="utf-8") as fh:
            src = re.sub(r"/\*.*?\*/", "", re.sub(r"//[^\n]*", "", fh.read()), flags=re.S)
        h.update("\n".join(l.rstrip() for l in src.splitlines() if l.strip()).encode())
    return h.hexdigest()[:12]


def ingest_traffic(csv_path, key, note):
    """Record the DRAM bytes per step of one degree's step kernels from an ncu
    CSV (--metrics dram__bytes_read.sum,dram__bytes_write.sum --csv) into
    profiles/traffic.json under `key`, with the current kernel_rev.  A step is
    one launch of the front/fused kernel (dg_step_kernel) plus, for the split
    step, its GEMM launch; bytes per step = captured bytes / front launches."""
    import csv
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1024, "MB": 1024 ** 2, "GB": 1024 ** 3}
    rows = list(csv.reader(open(csv_path, encoding="utf-8", errors="replace")))
    hdr = next(i for i, r in enumerate(rows) if "Metric Name" in r)
    H = rows[hdr]
    iid, ik, im, iu, iv = (H.index(x) for x in ("ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"))
    per = {}
    for r in rows[hdr + 1:]:
        if len(r) <= iv or not r[im].startswith("dram__bytes_"):
            continue
        v = float(r[iv].replace(",", "")) * scale.get(r[iu], 1)
        d = per.setdefault(r[iid], {"kernel": r[ik], "read": 0.0, "write": 0.0})
        d["read" if "read" in r[im] else "write"] += v
    fronts = sum(1 for d in per.values() if "dg_step_kernel" in d["kernel"])
    if not fronts:
        raise SystemExit("no dg_step_kernel launch in " + csv_path)
    rd = sum(d["read"] for d in per.values()) / fronts
    wr = sum(d["write"] for d in per.values()) / fronts
    kernels = sorted({d["kernel"].split("(")[0] for d in per.values()})
    path = os.path.join(ROOT, "profiles", "traffic.json")
    tr = json.load(open(path)) if os.path.exists(path) else {}
    tr[key] = {"kernel": " + ".join(kernels), "kernel_rev": kernel_rev(), "dram_bytes_per_launch": int(rd + wr),
               "dram_read": int(rd), "dram_write": int(wr), "launches": len(per), "steps": fronts, "source": note}
    with open(path, "w") as f:
        json.dump(tr, f, indent=1, sort_keys=True)
    print(json.dumps({key: tr[key]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--degrees", default="1,2,3,4,5,6,7,8")
    ap.add_argument("--model", default="acoustic", choices=["acoustic", "elastic"],
                    help="model of the timed sweep (the headline is the acoustic one)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-steps", type=int, default=500)
    ap.add_argument("--serve-max-batch", type=int, default=8,
                    help="solves the served stream's server steps together at most (8: lower p50 under load "
                         "than 64 at about 2 %% more makespan)")
    ap.add_argument("--no-sweeps", action="store_true")
    ap.add_argument("--strategy", default="fused", choices=["fused", "library", "plain"],
                    help="step strategy of the timed sweep (default: the fused step)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16x3", "bf16x6", "tf32"],
                    help="arithmetic of the timed sweep's operator contractions (default FP32)")
    ap.add_argument("--variants", default="",
                    help="kernel variant index per degree instead of autotuning (e.g. to replay a run's choice)")
    ap.add_argument("--sweep-steps", type=int, default=50)
    ap.add_argument("--sequential", action="store_true",
                    help="time the sweep's degrees one after another on one stream (default: concurrently)")
    ap.add_argument("--join-every-step", action="store_true",
                    help="concurrent sweep: join the degrees' streams after every sweep step")
    ap.add_argument("--no-peak", action="store_true", help="skip the FP32 FMA peak measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the large elastic workload")
    ap.add_argument("--large-steps", type=int, default=20)
    ap.add_argument("--large-only", action="store_true", help="time only the large elastic workload")
    ap.add_argument("--large-variant", type=int, default=-1,
                    help="kernel variant of the large elastic workload instead of autotuning")
    ap.add_argument("--ingest-ncu", default="", help="ncu CSV of DRAM bytes to record in profiles/traffic.json")
    ap.add_argument("--traffic-key", default="", help="key of the --ingest-ncu entry, e.g. acoustic_N8_fp32_v0")
    ap.add_argument("--traffic-note", default="", help="where the --ingest-ncu capture came from")
    args = ap.parse_args()
    if args.ingest_ncu:
        ingest_traffic(args.ingest_ncu, args.traffic_key, args.traffic_note)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    from paper_1602_07997_gb300 import build as B
    if not os.path.exists(B.LIB):
        raise RuntimeError("libdg.so is not built: run __graft_entry__.build() first")
    run(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
