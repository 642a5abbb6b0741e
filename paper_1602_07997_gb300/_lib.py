"""ctypes binding of libdg (argument marshalling only; all compute runs in the library).

The shared library is built in-tree by ``paper_1602_07997_gb300.build``.
Importing this module never falls back to anything: if ``libdg.so`` is
missing the first call raises.
"""

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdg.so")

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA, DG_ENONFINITE, DG_ETIMEOUT, DG_EAGAIN, DG_ECANCELED, DG_ENOENT = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
DG_HOST_ASYNC = 2
ACOUSTIC, ELASTIC = 0, 1
FLUX = {"upwind": 0, "centered": 1, "centred": 1}
BC = {None: 0, "default": 0, "rigid": 1, "free": 2}
PRECISION = {"fp32": 0, "bf16x3": 1, "bf16x6": 2, "tf32": 3}
STRATEGY = {"fused": 0, "library": 1, "plain": 2}

# every symbol that include/dg.h declares
EXPORTS = ("dg_setup", "dg_destroy", "dg_info", "dg_set_state", "dg_get_state", "dg_rhs", "dg_step",
           "dg_set_dt", "dg_sync", "dg_autotune", "dg_kernel_info", "dg_set_variant", "dg_node_coords", "dg_set_source", "dg_add_source", "dg_suggest_dt",
           "dg_reference_element", "dg_last_error", "dg_server_create", "dg_submit", "dg_poll",
           "dg_cancel", "dg_server_stats", "dg_server_destroy", "dg_rhs_host_noalloc", "dg_set_receivers",
           "dg_get_traces", "dg_fp32_peak", "dg_set_finite_check", "dg_set_wait_limit", "dg_launch_count",
           "dg_tune_save", "dg_tune_load", "dg_tune_clear", "dg_set_stream")


class DGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libdg error %d: %s" % (code, msg))
        self.code = code


class Mesh(C.Structure):
    _fields_ = [("nverts", C.c_int64), ("ntets", C.c_int64),
                ("verts", C.POINTER(C.c_double)), ("tets", C.POINTER(C.c_int64))]


class Opts(C.Structure):
    _fields_ = [("flux", C.c_int), ("bc", C.c_int), ("precision", C.c_int),
                ("block_elems", C.c_int), ("dt", C.c_double), ("stream", C.c_void_p), ("strategy", C.c_int)]


class Request(C.Structure):
    _fields_ = [("mesh", C.POINTER(Mesh)), ("coeffs", C.POINTER(C.c_double)), ("N", C.c_int),
                ("model", C.c_int), ("opts", Opts), ("q0", C.POINTER(C.c_float)),
                ("src_xyz", C.POINTER(C.c_double)), ("src_dir", C.POINTER(C.c_double)),
                ("src_amp", C.POINTER(C.c_double)), ("src_namp", C.c_int64), ("nsteps", C.c_int),
                ("nsrc", C.c_int)]


_lib = None


def lib():
    """Load libdg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libdg.so not found at %s: build it with "
                           "`python -m paper_1602_07997_gb300.build`" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    P = C.POINTER
    sig = {
        "dg_setup": (i32, [P(Mesh), P(dbl), i32, i32, P(Opts), P(vp)]),
        "dg_destroy": (None, [vp]),
        "dg_info": (i32, [vp, P(i64), P(i32), P(i32), P(i32)]),
        "dg_set_state": (i32, [vp, vp, vp, vp, i64, i32]),
        "dg_get_state": (i32, [vp, vp, vp, vp, P(i64), P(i32), i32]),
        "dg_rhs": (i32, [vp, vp, i32]),
        "dg_step": (i32, [vp, i32]),
        "dg_set_dt": (i32, [vp, dbl]),
        "dg_sync": (i32, [vp]),
        "dg_autotune": (i32, [vp, i32, P(i32), P(dbl), P(dbl)]),
        "dg_kernel_info": (i32, [vp, P(i32), P(i32), P(i64), P(i32), P(i32), P(i32), P(i32)]),
        "dg_set_variant": (i32, [vp, i32]),
        "dg_node_coords": (i32, [vp, P(dbl)]),
        "dg_set_source": (i32, [vp, P(dbl), P(dbl), P(dbl), i64]),
        "dg_add_source": (i32, [vp, P(dbl), P(dbl), P(dbl), i64]),
        "dg_suggest_dt": (i32, [P(Mesh), P(dbl), i32, i32, dbl, P(dbl)]),
        "dg_reference_element": (i32, [i32, P(dbl), P(dbl), P(dbl), P(dbl), P(dbl), P(i32)]),
        "dg_last_error": (C.c_char_p, []),
        "dg_server_create": (i32, [C.c_size_t, i32, P(vp)]),
        "dg_submit": (i32, [vp, P(Request), P(C.c_uint64)]),
        "dg_poll": (i32, [vp, C.c_uint64, vp, P(dbl)]),
        "dg_cancel": (i32, [vp, C.c_uint64]),
        "dg_server_stats": (i32, [vp, P(i64), P(i64), P(i64), P(i64)]),
        "dg_server_destroy": (None, [vp]),
        "dg_rhs_host_noalloc": (i32, [vp, vp]),
        "dg_set_receivers": (i32, [vp, P(dbl), i32]),
        "dg_get_traces": (i32, [vp, vp, P(i64), i32]),
        "dg_fp32_peak": (i32, [vp, i32, dbl, P(dbl), P(dbl), P(dbl)]),
        "dg_set_finite_check": (i32, [vp, i32]),
        "dg_set_wait_limit": (i32, [vp, i64]),
        "dg_launch_count": (i32, [vp, P(i64)]),
        "dg_tune_save": (i32, [C.c_char_p]),
        "dg_tune_load": (i32, [C.c_char_p, P(i32)]),
        "dg_tune_clear": (i32, []),
        "dg_set_stream": (i32, [vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(rc):
    if rc != DG_OK:
        msg = lib().dg_last_error()
        raise DGError(rc, msg.decode() if msg else "")
    return rc


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_mesh(verts, tets):
    verts = np.ascontiguousarray(verts, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int64)
    if verts.ndim != 2 or verts.shape[1] != 3 or tets.ndim != 2 or tets.shape[1] != 4:
        raise ValueError("verts must be [nverts][3] and tets [ntets][4], got %s and %s"
                         % (verts.shape, tets.shape))
    m = Mesh(verts.shape[0], tets.shape[0], _dptr(verts), tets.ctypes.data_as(C.POINTER(C.c_int64)))
    return m, (verts, tets)  # keep the arrays alive with the struct


def _coeffs(coeffs, K, model):
    """Per-element coefficients as contiguous float64: [K][2] (rho, c) for the
    acoustic model, [K][3] (lambda, mu, rho) for the elastic one."""
    cf = np.ascontiguousarray(coeffs, dtype=np.float64)
    nc = 2 if _model(model) == ACOUSTIC else 3
    if cf.size != K * nc:
        raise ValueError("coeffs must be [%d][%d], got %s" % (K, nc, cf.shape))
    return cf


def _point(x):
    """Three contiguous float64 values (a position or a direction)."""
    p = np.ascontiguousarray(x, dtype=np.float64)
    if p.size != 3:
        raise ValueError("expected 3 coordinates, got %s" % (np.shape(x),))
    return p


def _model(model):
    if isinstance(model, str):
        if model not in ("acoustic", "elastic"):
            raise ValueError("model must be 'acoustic' or 'elastic', got %r" % model)
        return ACOUSTIC if model == "acoustic" else ELASTIC
    return int(model)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _buf(x, dtype, count, write=False):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    if _is_torch(x):
        import torch
        if x.dtype != {np.float32: torch.float32, np.float64: torch.float64}[dtype]:
            raise TypeError("tensor dtype must be %s" % dtype)
        if not x.is_contiguous() or x.numel() != count:
            raise ValueError("tensor must be contiguous with %d elements" % count)
        return C.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        if write:
            raise TypeError("output array must be C-contiguous %s" % np.dtype(dtype))
        a = np.ascontiguousarray(a, dtype=dtype)
    if a.size != count:
        raise ValueError("array must have %d elements, got %d" % (count, a.size))
    return C.c_void_p(a.ctypes.data), 0, a


def suggest_dt(verts, tets, coeffs, N, model, cfl=0.5):
    m, keep = make_mesh(verts, tets)
    cf = _coeffs(coeffs, keep[1].shape[0], model)
    out = C.c_double()
    check(lib().dg_suggest_dt(C.byref(m), _dptr(cf), int(N), _model(model), float(cfl), C.byref(out)))
    return out.value


def reference_element(N):
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    Nfp = (N + 1) * (N + 2) // 2
    nodes = np.zeros((Np, 3))
    Dr, Ds, Dt = (np.zeros((Np, Np)) for _ in range(3))
    LIFT = np.zeros((Np, 4 * Nfp))
    fm = np.zeros((4, Nfp), dtype=np.int32)
    check(lib().dg_reference_element(int(N), _dptr(nodes), _dptr(Dr), _dptr(Ds), _dptr(Dt), _dptr(LIFT),
                                     fm.ctypes.data_as(C.POINTER(C.c_int32))))
    return dict(nodes=nodes, Dr=Dr, Ds=Ds, Dt=Dt, LIFT=LIFT, fmask=fm)


def fp32_peak(stream=None, reps=5, target_ms=20.0):
    """FP32 FMA throughput of the current device (dg_fp32_peak): best TFLOP/s
    of the scalar and of the packed two-lane FMA form, and the longer of the
    two best launch times in ms."""
    s, p, ms = C.c_double(), C.c_double(), C.c_double()
    check(lib().dg_fp32_peak(stream, int(reps), float(target_ms), C.byref(s), C.byref(p), C.byref(ms)))
    return {"scalar_tflops": s.value, "packed_tflops": p.value, "ms": ms.value}


def tune_save(path):
    """Write this process's autotuner choices to `path` (dg_tune_save)."""
    check(lib().dg_tune_save(os.fsencode(path)))


def tune_load(path):
    """Take the choices of a saved cache for the current device; returns how many were taken."""
    n = C.c_int()
    check(lib().dg_tune_load(os.fsencode(path), C.byref(n)))
    return n.value


def tune_clear():
    """Forget every autotuner choice of this process."""
    check(lib().dg_tune_clear())


class Solver:
    """One DG discretisation on the GPU (a dg_handle, see dg_setup).

    verts [nverts][3] and tets [K][4] (0-based, positively oriented) define a
    conforming tetrahedral mesh; coeffs is [K][2] (rho, c) for the acoustic
    model or [K][3] (lambda, mu, rho) for the elastic one; N in 1..8.  flux:
    "upwind" or "centred"; bc: None (rigid wall acoustic, traction-free
    elastic), "rigid" or "free"; dt: the step of `step` (see suggest_dt);
    stream: a cudaStream_t as an integer (e.g. torch.cuda.Stream().cuda_stream);
    precision: "fp32", "bf16x3", "bf16x6" or "tf32" (library strategy);
    strategy: "fused", "library" or "plain".  States are [K][Nf][Np] float32,
    as numpy arrays (host) or CUDA tensors (device)."""

    def __init__(self, verts, tets, coeffs, N, model="acoustic", flux="upwind", bc=None, dt=0.0,
                 stream=None, block_elems=0, precision="fp32", strategy="fused"):
        m, keep = make_mesh(verts, tets)
        cf = _coeffs(coeffs, keep[1].shape[0], model)
        o = Opts(FLUX[flux], BC[bc], PRECISION[precision], int(block_elems), float(dt),
                 C.c_void_p(stream or 0), STRATEGY[strategy])
        h = C.c_void_p()
        check(lib().dg_setup(C.byref(m), _dptr(cf), int(N), _model(model), C.byref(o), C.byref(h)))
        self.h = h
        K, Np, Nfp, Nf = C.c_int64(), C.c_int(), C.c_int(), C.c_int()
        check(lib().dg_info(h, C.byref(K), C.byref(Np), C.byref(Nfp), C.byref(Nf)))
        self.K, self.Np, self.Nfp, self.Nf = K.value, Np.value, Nfp.value, Nf.value
        self.N, self.model = int(N), _model(model)
        self.shape = (self.K, self.Nf, self.Np)

    @property
    def size(self):
        return self.K * self.Nf * self.Np

    def close(self):
        if getattr(self, "h", None):
            lib().dg_destroy(self.h)
            self.h = None

    __del__ = close

    def set_state(self, q, r1=None, r2=None, step=0, asynchronous=False):
        """Replace the state by q; r1 = r^{m-1} and r2 = r^{m-2} give the AB3
        history (both or neither: without them the next steps start with Euler
        and AB2).  step = the time-step index of q (it indexes source amplitudes).
        asynchronous: q (and r1, r2) are pinned host tensors and the copy stays
        in stream order (complete at the next sync); leave them untouched until then."""
        if (r1 is None) != (r2 is None):
            raise ValueError("r1 and r2 are given together or not at all")
        pq, dq, kq = _buf(q, np.float32, self.size)
        if asynchronous:
            if dq:
                raise ValueError("asynchronous transfers take pinned host memory")
            dq = DG_HOST_ASYNC
        p1 = p2 = None
        keep = []
        if r1 is not None:
            p1, d1, k1 = _buf(r1, np.float32, self.size)
            p2, d2, k2 = _buf(r2, np.float32, self.size)
            keep += [k1, k2]
            if not (min(dq, 1) == d1 == d2):
                raise ValueError("q, r1 and r2 must all be host or all device")
        check(lib().dg_set_state(self.h, pq, p1, p2, int(step), dq))

    def get_state(self, q=None, r1=None, r2=None, asynchronous=False):
        """The state q (a new host array, or into q / r1 / r2 if given); sets
        self.step_index and self.history (stored RHS levels, 0..2).
        asynchronous: the outputs are pinned host tensors, filled in stream
        order (complete at the next sync)."""
        ret = q is None
        if q is None:
            q = np.empty(self.shape, dtype=np.float32)
        pq, dq, _ = _buf(q, np.float32, self.size, write=True)
        if asynchronous:
            if dq:
                raise ValueError("asynchronous transfers take pinned host memory")
            dq = DG_HOST_ASYNC
        p1 = _buf(r1, np.float32, self.size, write=True)[0] if r1 is not None else None
        p2 = _buf(r2, np.float32, self.size, write=True)[0] if r2 is not None else None
        step, hist = C.c_int64(), C.c_int()
        check(lib().dg_get_state(self.h, pq, p1, p2, C.byref(step), C.byref(hist), dq))
        self.step_index, self.history = step.value, hist.value
        return q if ret else None

    def rhs(self, out=None):
        """r(q^m) at the current state, source included; the state is unchanged."""
        ret = out is None
        if out is None:
            out = np.empty(self.shape, dtype=np.float32)
        p, d, _ = _buf(out, np.float32, self.size, write=True)
        check(lib().dg_rhs(self.h, p, d))
        return out if ret else None

    def rhs_host_noalloc(self, out=None):
        """RHS into host memory through the library's fixed scratch (no device allocation)."""
        ret = out is None
        if out is None:
            out = np.empty(self.shape, dtype=np.float32)
        p, d, _ = _buf(out, np.float32, self.size, write=True)
        if d:
            raise ValueError("rhs_host_noalloc writes host memory")
        check(lib().dg_rhs_host_noalloc(self.h, p))
        return out if ret else None

    def set_stream(self, stream):
        """Issue later work on `stream` (a cudaStream_t as an int, e.g.
        torch.cuda.Stream().cuda_stream); work already issued finishes first."""
        check(lib().dg_set_stream(self.h, C.c_void_p(int(stream) if stream else 0)))

    def set_dt(self, dt):
        check(lib().dg_set_dt(self.h, float(dt)))

    def step(self, n=1):
        """Advance n AB3 steps, asynchronously on the solver's stream."""
        check(lib().dg_step(self.h, int(n)))

    def sync(self):
        """Wait for the stream; raises DGError with DG_ETIMEOUT if a bounded device
        wait expired, or DG_ENONFINITE if a finite-state check found NaN/Inf."""
        check(lib().dg_sync(self.h))

    def set_finite_check(self, every):
        """Check q for NaN/Inf after every `every`-th step (0 = never; default 100)."""
        check(lib().dg_set_finite_check(self.h, int(every)))

    def set_wait_limit(self, cycles):
        """Cycles before a bounded device wait gives up (0 = default; < 0 = at once, a test hook)."""
        check(lib().dg_set_wait_limit(self.h, int(cycles)))

    def launch_count(self):
        """Kernels of this library launched by the handle so far."""
        n = C.c_int64()
        check(lib().dg_launch_count(self.h, C.byref(n)))
        return n.value

    def autotune(self, reps=5):
        """Time every compiled kernel variant on this mesh and keep the fastest.

        Returns (block_elems, ms_per_step, [ms per variant])."""
        nv = self.kernel_info()["variants"]
        eb, ms = C.c_int(), C.c_double()
        vms = (C.c_double * max(nv, 1))()
        check(lib().dg_autotune(self.h, int(reps), C.byref(eb), C.byref(ms), vms))
        return eb.value, ms.value, list(vms)[:nv]

    def kernel_info(self):
        eb, nt, sm, nv, tn, sp = C.c_int(), C.c_int(), C.c_int64(), C.c_int(), C.c_int(), C.c_int()
        vi = C.c_int()
        check(lib().dg_kernel_info(self.h, C.byref(eb), C.byref(nt), C.byref(sm), C.byref(nv), C.byref(tn),
                                   C.byref(sp), C.byref(vi)))
        return dict(block_elems=eb.value, threads=nt.value, smem_bytes=sm.value, variants=nv.value,
                    tile_elems=tn.value, split=sp.value, variant=vi.value)

    def set_variant(self, index):
        check(lib().dg_set_variant(self.h, int(index)))

    def node_coords(self):
        x = np.empty((self.K, self.Np, 3))
        check(lib().dg_node_coords(self.h, _dptr(x)))
        return x

    def set_source(self, xs, amp, direction=(0.0, 0.0, 1.0)):
        if amp is None:
            check(lib().dg_set_source(self.h, None, None, None, 0))
            return
        xs, d = _point(xs), _point(direction)
        a = np.ascontiguousarray(amp, dtype=np.float64)
        check(lib().dg_set_source(self.h, _dptr(xs), _dptr(d), _dptr(a), a.size))

    def add_source(self, xs, amp, direction=(0.0, 0.0, 1.0)):
        """One more point source (several sources add their terms)."""
        xs, d = _point(xs), _point(direction)
        a = np.ascontiguousarray(amp, dtype=np.float64)
        check(lib().dg_add_source(self.h, _dptr(xs), _dptr(d), _dptr(a), a.size))


    def set_receivers(self, xyz):
        """Receivers at xyz [nrec][3]: the fields there are recorded after every step."""
        x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        self.nrec = x.shape[0]
        check(lib().dg_set_receivers(self.h, _dptr(x) if x.size else None, int(self.nrec)))

    def traces(self):
        """Recorded receiver samples, [nsamples][nrec][Nf] float32."""
        n = C.c_int64()
        check(lib().dg_get_traces(self.h, None, C.byref(n), 0))
        out = np.empty((n.value, getattr(self, "nrec", 0), self.Nf), np.float32)
        if out.size:
            check(lib().dg_get_traces(self.h, out.ctypes.data_as(C.c_void_p), C.byref(n), 0))
        return out


class Server:
    """Continuous-batching solve server (dg_server): submit / poll / cancel."""

    def __init__(self, hbm_budget_bytes=0, max_batch=64):
        s = C.c_void_p()
        check(lib().dg_server_create(C.c_size_t(hbm_budget_bytes), int(max_batch), C.byref(s)))
        self.s = s
        self._meta = {}

    def close(self):
        if getattr(self, "s", None):
            lib().dg_server_destroy(self.s)
            self.s = None

    __del__ = close

    def submit(self, verts, tets, coeffs, N, model="acoustic", q0=None, dt=0.0, nsteps=1, flux="upwind",
               bc=None, source=None, amp=None, direction=(0.0, 0.0, 1.0)):
        m, keep = make_mesh(verts, tets)
        cf = _coeffs(coeffs, keep[1].shape[0], model)
        model = _model(model)
        Nf = 4 if model == ACOUSTIC else 9
        Np = (N + 1) * (N + 2) * (N + 3) // 6
        K = keep[1].shape[0]
        r = Request()
        r.mesh = C.pointer(m)
        r.coeffs = _dptr(cf)
        r.N, r.model, r.nsteps = int(N), model, int(nsteps)
        r.opts = Opts(FLUX[flux], BC[bc], 0, 0, float(dt), None)
        q0a = None
        if q0 is not None:
            q0a = np.ascontiguousarray(q0, dtype=np.float32)
            if q0a.size != K * Nf * Np:
                raise ValueError("q0 must have K Nf Np = %d values, got %d" % (K * Nf * Np, q0a.size))
            r.q0 = q0a.ctypes.data_as(C.POINTER(C.c_float))
        xs = d = a = None
        if source is not None and amp is not None:
            # one source: source [3], amp [namp]; several: source [n][3],
            # amp [n][namp], direction [3] (for all) or [n][3]
            xs = np.ascontiguousarray(np.atleast_2d(source), dtype=np.float64)
            if xs.ndim != 2 or xs.shape[1] != 3:
                raise ValueError("source must be [3] or [n][3], got %s" % (np.shape(source),))
            ns = xs.shape[0]
            a = np.ascontiguousarray(np.atleast_2d(amp), dtype=np.float64)
            if a.shape[0] != ns:
                raise ValueError("amp needs one row per source")
            d = np.ascontiguousarray(np.broadcast_to(np.asarray(direction, dtype=np.float64), (ns, 3)))
            r.src_xyz, r.src_dir, r.src_amp, r.src_namp = _dptr(xs), _dptr(d), _dptr(a), a.shape[1]
            r.nsrc = ns
        t = C.c_uint64()
        check(lib().dg_submit(self.s, C.byref(r), C.byref(t)))
        self._meta[t.value] = (K, Nf, Np)
        return t.value

    def poll(self, ticket):
        """None while running; (q [K][Nf][Np], latency_s) when finished; raises on failure."""
        K, Nf, Np = self._meta.get(ticket, (0, 0, 0))
        out = np.empty((K, Nf, Np), dtype=np.float32)
        lat = C.c_double()
        ptr = C.c_void_p(out.ctypes.data) if out.size else None
        rc = lib().dg_poll(self.s, C.c_uint64(ticket), ptr, C.byref(lat))
        if rc == DG_EAGAIN:
            return None
        self._meta.pop(ticket, None)
        check(rc)
        return out, lat.value

    def wait(self, ticket, timeout=300.0, interval=0.001):
        import time
        t0 = time.time()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.time() - t0 > timeout:
                raise TimeoutError("request %d did not finish in %.0f s" % (ticket, timeout))
            time.sleep(interval)

    def cancel(self, ticket):
        check(lib().dg_cancel(self.s, C.c_uint64(ticket)))

    def stats(self):
        q, r, d, n = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().dg_server_stats(self.s, C.byref(q), C.byref(r), C.byref(d), C.byref(n)))
        return dict(queued=q.value, running=r.value, done=d.value, launches=n.value)
