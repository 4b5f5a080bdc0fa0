"""Python front end of the C ABI (argument marshalling only; PyTorch supplies
device memory and the current CUDA stream).

    op = PeriodicOp("laplace", e1=(16, 0), e2=(0, 1), tol=1e-6, precision="mixed",
                    ns_max=N, nt_max=N)
    pot, grad = op(src, q)            # targets = sources
    vel, _ = stokes_op(src, f, trg)   # Stokes / modified Stokes: velocity

Kernels: "laplace", "modhelm" (beta > 0), "stokes", "mstokes" (the modified
Stokeslet, beta > 0).  Options beyond the kernel: singly=True (periodic
along e1 only), we="auto" | "rotated" | "axis" (the west/east plane-wave
direction), part="total" | "far" | "near".
Tensors: src/trg [2, n] float64 (CUDA), q [nrhs, n] or [nrhs, 2, n] (Stokes
kernels).  Outputs: pot [nrhs, nt] (Stokes kernels: velocity [nrhs, 2, nt]),
grad [nrhs, 2, nt] or None.
Every step of the computation runs in the CUDA library; nothing here
computes.
"""
import ctypes

import numpy as np

from . import _lib

_KER = {"laplace": _lib.PFMM_LAPLACE, "modhelm": _lib.PFMM_MODHELM, "stokes": _lib.PFMM_STOKES,
        "mstokes": _lib.PFMM_MSTOKES}
_VEC = ("stokes", "mstokes")  # force in, velocity out
_PREC = {"fp64": _lib.PFMM_FP64, "mixed": _lib.PFMM_MIXED}
_PATH = {"auto": _lib.PFMM_PATH_AUTO, "direct": _lib.PFMM_PATH_DIRECT, "nufft": _lib.PFMM_PATH_NUFFT}
_PART = {"total": 0, "far": _lib.PFMM_FAR_ONLY, "near": _lib.PFMM_NEAR_ONLY}
_WE = {"auto": 0, "rotated": _lib.PFMM_WE_ROTATED, "axis": _lib.PFMM_WE_AXIS}
_NEAR = {"auto": 0, "direct": _lib.PFMM_NEAR_DIRECT, "fmm": _lib.PFMM_NEAR_FMM}


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _check_tensor(name, t, shape, device):
    """Raise ValueError unless t is a contiguous float64 tensor of `shape` on
    `device`: the library reads raw pointers with these sizes, so a wrong
    dtype or shape must not reach it."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch.Tensor, got {type(t).__name__}")
    if t.dtype != torch.float64:
        raise ValueError(f"{name}: dtype {t.dtype}, expected torch.float64")
    if t.device != device:
        raise ValueError(f"{name}: on {t.device}, expected {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: not contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")


def check_inputs(kernel, nrhs, src, q, trg, out=None, grad=True):
    """Validate the tensors of one PeriodicOp call (see _check_tensor); returns
    (ns, nt).  src [2, ns], q [nrhs, ns] or [nrhs, 2, ns] (Stokes kernels),
    trg [2, nt] or None, out (pot, grad) of the output shapes or None."""
    import torch
    if not isinstance(src, torch.Tensor) or src.dim() != 2:
        raise ValueError("src: expected a [2, ns] tensor")
    dev = src.device
    ns = src.shape[1]
    vec = kernel in _VEC
    _check_tensor("src", src, (2, ns), dev)
    _check_tensor("q", q, (nrhs, 2, ns) if vec else (nrhs, ns), dev)
    if trg is None:
        nt = ns
    else:
        if not isinstance(trg, torch.Tensor) or trg.dim() != 2:
            raise ValueError("trg: expected a [2, nt] tensor")
        nt = trg.shape[1]
        _check_tensor("trg", trg, (2, nt), dev)
    if out is not None:
        pot, g = out
        _check_tensor("out pot", pot, (nrhs, 2, nt) if vec else (nrhs, nt), dev)
        if g is not None:
            if vec:
                raise ValueError("out grad: must be None for the Stokes kernels")
            _check_tensor("out grad", g, (nrhs, 2, nt), dev)
    return ns, nt


class PeriodicOp:
    def __init__(self, kernel, e1, e2, beta=0.0, tol=1e-6, precision="mixed", path="auto", nufft_w=0, n_gl=0,
                 nrhs=1, part="total", ns_max=0, nt_max=0, device=None, singly=False, we="auto", near="auto",
                 near_order=0, near_leaf=0, deterministic=False):
        L = _lib.lib()
        o = _lib.Opts()
        o.e1[0], o.e1[1] = float(e1[0]), float(e1[1])
        o.e2[0], o.e2[1] = float(e2[0]), float(e2[1])
        o.kernel = _KER[kernel]
        o.beta = float(beta)
        o.tol = float(tol)
        o.precision = _PREC[precision]
        o.path = _PATH[path]
        o.nufft_w = int(nufft_w)
        o.n_gl = int(n_gl)
        o.nrhs = int(nrhs)
        o.flags = (_PART[part] | (_lib.PFMM_SINGLY_PERIODIC if singly else 0) | _WE[we] | _NEAR[near] |
                   (_lib.PFMM_DETERMINISTIC if deterministic else 0))
        o.near_order = int(near_order)
        o.near_leaf = int(near_leaf)
        self.kernel = kernel
        self.nrhs = int(nrhs)
        self.ns_max, self.nt_max = int(ns_max), int(nt_max)
        h = ctypes.c_void_p()
        _lib.check(L.pfmm_plan_create(ctypes.byref(o), self.ns_max, self.nt_max, ctypes.byref(h)))
        self._h = h
        sz = ctypes.c_size_t()
        _lib.check(L.pfmm_workspace_size(h, ctypes.byref(sz)))
        self.ws_bytes = sz.value
        _lib.check(L.pfmm_workspace_size_host(h, ctypes.byref(sz)))
        self.ws_host_bytes = sz.value
        self.device = device
        self._ws = None
        self._ws_host = None

    def describe(self):
        d = _lib.PlanDesc()
        _lib.check(_lib.lib().pfmm_plan_describe(self._h, ctypes.byref(d)))
        return {k: (list(getattr(d, k)) if k in ("rot", "we_dir") else getattr(d, k)) for k, _ in d._fields_}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                _lib.lib().pfmm_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    def workspace(self, host=False):
        import torch
        dev = self.device or torch.device("cuda", torch.cuda.current_device())
        if host:
            if self._ws_host is None:
                self._ws_host = torch.empty(max(self.ws_host_bytes, 256), dtype=torch.uint8, device=dev)
            return self._ws_host
        if self._ws is None:
            self._ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        return self._ws

    def __call__(self, src, q, trg=None, grad=True, out=None, stream=None):
        """Device tensors in, device tensors out (float64).  trg None -> targets = sources."""
        import torch
        ns, nt = check_inputs(self.kernel, self.nrhs, src, q, trg, out, grad)
        if not src.is_cuda:
            raise ValueError("src: expected CUDA tensors")
        self_t = trg is None
        if self_t:
            trg = src
        stokes = self.kernel in _VEC
        if out is None:
            pot = torch.empty((self.nrhs, 2, nt) if stokes else (self.nrhs, nt), dtype=torch.float64,
                              device=src.device)
            g = torch.empty((self.nrhs, 2, nt), dtype=torch.float64, device=src.device) if (grad and not stokes) else None
        else:
            pot, g = out
        ws = self.workspace()
        st = stream if stream is not None else torch.cuda.current_stream(src.device).cuda_stream
        _lib.check(_lib.lib().pfmm_execute(self._h, _ptr(ws), ws.numel(), ns, _ptr(src), _ptr(q), nt,
                                           _ptr(trg), _ptr(pot), _ptr(g), ctypes.c_void_p(st)))
        return pot, g

    def execute_host(self, src, q, trg=None, grad=True, stream=None):
        """Host numpy arrays in and out through pfmm_execute_host (staged copies)."""
        import torch
        src = np.ascontiguousarray(src, np.float64)
        q = np.ascontiguousarray(q, np.float64)
        self_t = trg is None
        trg = src if self_t else np.ascontiguousarray(trg, np.float64)
        ns, nt = src.shape[1], trg.shape[1]
        stokes = self.kernel in _VEC
        pot = np.empty((self.nrhs, 2, nt) if stokes else (self.nrhs, nt))
        g = np.empty((self.nrhs, 2, nt)) if (grad and not stokes) else None
        ws = self.workspace(host=True)
        st = stream if stream is not None else torch.cuda.current_stream(ws.device).cuda_stream
        vp = lambda a: ctypes.c_void_p(0 if a is None else a.ctypes.data)
        _lib.check(_lib.lib().pfmm_execute_host(self._h, _ptr(ws), ws.numel(), ns, vp(src), vp(q), nt,
                                                vp(src) if self_t else vp(trg), vp(pot), vp(g),
                                                ctypes.c_void_p(st)))
        return pot, g

    def execute_host_ptrs(self, src, q, trg, pot, grad, stream=None):
        """pfmm_execute_host on raw host pointers (e.g. pinned torch CPU tensors)."""
        import torch
        ws = self.workspace(host=True)
        st = stream if stream is not None else torch.cuda.current_stream(ws.device).cuda_stream
        ns, nt = src.shape[1], trg.shape[1]
        _lib.check(_lib.lib().pfmm_execute_host(self._h, _ptr(ws), ws.numel(), ns, _ptr(src), _ptr(q), nt,
                                                _ptr(trg), _ptr(pot), _ptr(grad), ctypes.c_void_p(st)))

    def profile(self, on=True):
        """Enable per-phase CUDA-event timing inside pfmm_execute."""
        _lib.check(_lib.lib().pfmm_profile_enable(self._h, 1 if on else 0))

    def phase_ms(self, sub=False):
        """Milliseconds of [prep, far field, near field] of the last execute;
        sub=True appends the tree code's [tree, upward, traversal, downward,
        leaves] (zeros when the direct P2P ran)."""
        n = 8 if sub else 3
        ms = (ctypes.c_float * n)()
        _lib.check(_lib.lib().pfmm_profile_read(self._h, ms, n))
        return list(ms)

    def pairs(self, stream=None):
        """Near-image pairs the P2P evaluated in the last profiled execute
        (pfmm_profile_pairs; synchronises)."""
        import torch
        ws = self.workspace()
        st = stream if stream is not None else torch.cuda.current_stream(ws.device).cuda_stream
        v = ctypes.c_double()
        _lib.check(_lib.lib().pfmm_profile_pairs(self._h, _ptr(ws), ctypes.c_void_p(st), ctypes.byref(v)))
        return float(v.value)

    def capture(self, src, q, trg=None, grad=True, out=None):
        """Record one execute in a CUDA graph, after an eager execute on the
        same buffers (which uploads the plan's tables into its workspace; the
        captured execute reuses them).  Replaying the graph re-runs the
        operator on the current contents of src, q, trg into out.  Another plan
        must not use this workspace between replays.  Returns (graph, out)."""
        import torch
        out = self(src, q, trg, grad=grad, out=out)
        torch.cuda.synchronize()
        s = torch.cuda.Stream(src.device)
        s.wait_stream(torch.cuda.current_stream(src.device))
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(graph, stream=s):
                self(src, q, trg, grad=grad, out=out, stream=s.cuda_stream)
        torch.cuda.current_stream(src.device).wait_stream(s)
        return graph, out

    def near_stats(self, stream=None):
        """Tree-code statistics of the last execute (pfmm_near_stats; synchronises):
        boxes, M2L interactions, directly summed leaf pairs, directly summed
        point pairs (while profiling), overflow bits."""
        import torch
        ws = self.workspace()
        st = stream if stream is not None else torch.cuda.current_stream(ws.device).cuda_stream
        out = (ctypes.c_int64 * 5)()
        _lib.check(_lib.lib().pfmm_near_stats(self._h, _ptr(ws), ctypes.c_void_p(st), out))
        return dict(boxes=out[0], m2l=out[1], p2p_leaf_pairs=out[2], p2p_pairs=out[3], overflow=out[4])

    def status(self, stream=None):
        """Synchronise and return the device status of the last execute (raises on error)."""
        import torch
        ws = self.workspace()
        st = stream if stream is not None else torch.cuda.current_stream(ws.device).cuda_stream
        _lib.check(_lib.lib().pfmm_get_status(self._h, _ptr(ws), ctypes.c_void_p(st)))


def _opts(kernel, e1, e2, beta, tol, precision, path, nufft_w, n_gl, nrhs, flags):
    o = _lib.Opts()
    o.e1[0], o.e1[1] = float(e1[0]), float(e1[1])
    o.e2[0], o.e2[1] = float(e2[0]), float(e2[1])
    o.kernel = _KER[kernel]
    o.beta = float(beta)
    o.tol = float(tol)
    o.precision = _PREC[precision]
    o.path = _PATH[path]
    o.nufft_w = int(nufft_w)
    o.n_gl = int(n_gl)
    o.nrhs = int(nrhs)
    o.flags = int(flags)
    return o


class BatchOp:
    """Many independent cells in one call (pfmm_batch_*).

    cells: list of dicts with e1, e2 and optionally beta, tol, path, nufft_w
    (per-cell far-field path and ES width, e.g. from tune_batch); shared kernel,
    precision and nrhs.  src_counts / trg_counts: points per cell (targets
    default to the sources).  Inputs are the concatenated arrays
    src [2, NS], q [nrhs, NS] (Stokes [nrhs, 2, NS]), trg [2, NT]."""

    def __init__(self, kernel, cells, src_counts, trg_counts=None, precision="mixed", nrhs=1, tol=1e-6,
                 path="auto", p2p_chunk=0):
        L = _lib.lib()
        n = len(cells)
        arr = (_lib.Opts * n)()
        for i, c in enumerate(cells):
            arr[i] = _opts(kernel, c["e1"], c["e2"], c.get("beta", 0.0), c.get("tol", tol), precision,
                           c.get("path", path), c.get("nufft_w", 0), 0, nrhs, _WE[c.get("we", "auto")])
        so = np.concatenate([[0], np.cumsum(src_counts)]).astype(np.int64)
        self._so = (ctypes.c_int64 * (n + 1))(*so.tolist())
        self._to = None
        if trg_counts is not None:
            to = np.concatenate([[0], np.cumsum(trg_counts)]).astype(np.int64)
            self._to = (ctypes.c_int64 * (n + 1))(*to.tolist())
        h = ctypes.c_void_p()
        _lib.check(L.pfmm_batch_create(arr, n, self._so, self._to, int(p2p_chunk), ctypes.byref(h)))
        self._h = h
        sz = ctypes.c_size_t()
        _lib.check(L.pfmm_batch_workspace_size(h, ctypes.byref(sz)))
        self.ws_bytes = sz.value
        self.kernel, self.nrhs, self.ncell = kernel, int(nrhs), n
        self.NS = int(so[-1])
        self.NT = int(self.NS if trg_counts is None else np.sum(trg_counts))
        self.self_t = trg_counts is None
        self._ws = None

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                _lib.lib().pfmm_batch_destroy(h)
            except Exception:
                pass
            self._h = None

    def workspace(self, device):
        import torch
        if self._ws is None:
            self._ws = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=device)
        return self._ws

    def alloc_out(self, device, grad=True):
        import torch
        stokes = self.kernel in _VEC
        pot = torch.empty((self.nrhs, 2, self.NT) if stokes else (self.nrhs, self.NT), dtype=torch.float64,
                          device=device)
        g = torch.empty((self.nrhs, 2, self.NT), dtype=torch.float64, device=device) if (grad and not stokes) else None
        return pot, g

    def __call__(self, src, q, trg=None, out=None, grad=True, stream=None):
        import torch
        ns, nt = check_inputs(self.kernel, self.nrhs, src, q, trg, out, grad)
        if not src.is_cuda or ns != self.NS or nt != self.NT or (trg is None) != self.self_t:
            raise ValueError(f"batch inputs: CUDA tensors with {self.NS} sources and "
                             f"{'targets = sources' if self.self_t else f'{self.NT} targets'} expected")
        if out is None:
            out = self.alloc_out(src.device, grad)
        pot, g = out
        ws = self.workspace(src.device)
        st = stream if stream is not None else torch.cuda.current_stream(src.device).cuda_stream
        _lib.check(_lib.lib().pfmm_batch_execute(self._h, _ptr(ws), ws.numel(), _ptr(src), _ptr(q), _ptr(trg),
                                                 _ptr(pot), _ptr(g), ctypes.c_void_p(st)))
        return pot, g

    def status(self, device, stream=None):
        import torch
        ws = self.workspace(device)
        st = stream if stream is not None else torch.cuda.current_stream(device).cuda_stream
        _lib.check(_lib.lib().pfmm_batch_get_status(self._h, _ptr(ws), ctypes.c_void_p(st)))

    def profile(self, on=True, count_pairs=True):
        """Record CUDA events around the per-cell phases and the batched P2P of
        every execute, also inside a captured graph (pfmm_batch_profile_enable);
        count_pairs: also count the near-image pairs evaluated (eager executes)."""
        mode = 0 if not on else (1 if count_pairs else 2)
        _lib.check(_lib.lib().pfmm_batch_profile_enable(self._h, mode))

    def phase_ms(self):
        """(per-cell phases ms, batched P2P ms, kernels launched, near-image
        pairs evaluated) of the last profiled execute; waits for its events."""
        ms = (ctypes.c_float * 2)()
        n = ctypes.c_int()
        pairs = ctypes.c_double()
        _lib.check(_lib.lib().pfmm_batch_profile_read(self._h, ms, 2, ctypes.byref(n), ctypes.byref(pairs)))
        return float(ms[0]), float(ms[1]), int(n.value), float(pairs.value)

    def capture(self, src, q, trg=None, out=None, grad=True):
        """Record one execute in a CUDA graph (after a first execute on the same
        buffers, which uploads the descriptors).  Returns (graph, out)."""
        import torch
        if out is None:
            out = self.alloc_out(src.device, grad)
        self(src, q, trg, out=out)  # uploads descriptors for these buffers
        torch.cuda.synchronize()
        s = torch.cuda.Stream(src.device)
        s.wait_stream(torch.cuda.current_stream(src.device))
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            # the upload is keyed on the buffers; the same buffers -> kernels only
            with torch.cuda.graph(graph, stream=s):
                self(src, q, trg, out=out, stream=s.cuda_stream)
        torch.cuda.current_stream(src.device).wait_stream(s)
        return graph, out


class StokesPressure:
    """Pressure of the periodic Stokeslet sum, p = -(d/dx phi[f_x] + d/dy phi[f_y])
    with phi the periodic Laplace potential (pfmm_stokes_pressure): a Laplace
    PeriodicOp with 2 * nrhs right-hand sides on the same lattice.

        pres = StokesPressure(e1, e2, tol=1e-6, precision="mixed")(src, f, trg)
    """

    def __init__(self, e1, e2, tol=1e-6, precision="mixed", path="auto", nrhs=1, ns_max=0, nt_max=0, singly=False,
                 we="auto"):
        self.nrhs = int(nrhs)
        self.op = PeriodicOp("laplace", e1, e2, tol=tol, precision=precision, path=path, nrhs=2 * self.nrhs,
                             ns_max=ns_max, nt_max=nt_max, singly=singly, we=we)

    def __call__(self, src, f, trg=None, out=None, stream=None):
        import torch
        ns, nt = check_inputs("stokes", self.nrhs, src, f, trg)
        if not src.is_cuda:
            raise ValueError("src: expected CUDA tensors")
        tr = src if trg is None else trg
        if out is None:
            out = torch.empty((self.nrhs, nt), dtype=torch.float64, device=src.device)
        _check_tensor("out", out, (self.nrhs, nt), src.device)
        ws = self.op.workspace()
        st = stream if stream is not None else torch.cuda.current_stream(src.device).cuda_stream
        _lib.check(_lib.lib().pfmm_stokes_pressure(self.op._h, _ptr(ws), ws.numel(), ns, _ptr(src),
                                                   _ptr(f.contiguous()), nt, _ptr(tr), _ptr(out),
                                                   ctypes.c_void_p(st)))
        return out

    def status(self, stream=None):
        self.op.status(stream)


def autotune_batch(make_op, src, q, trg=None, candidates=(1024, 2048, 4096, 8192), reps=2, cache=None, key=None):
    """Pick the P2P source-chunk size of a batch by timing each candidate
    (CUDA events); make_op(p2p_chunk) -> BatchOp.  With a cache path and key,
    results persist across runs as JSON.  Returns (best_chunk, timings_ms)."""
    import json
    import os
    import torch
    if cache and key and os.path.exists(cache):
        try:
            d = json.load(open(cache))
            if key in d:
                return d[key]["p2p_chunk"], d[key]["ms"]
        except Exception:
            pass
    times = {}
    for c in candidates:
        op = make_op(c)
        out = op(src, q, trg)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            op(src, q, trg, out=out)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        times[c] = best
        del op
    chunk = min(times, key=times.get)
    if cache and key:
        d = {}
        if os.path.exists(cache):
            try:
                d = json.load(open(cache))
            except Exception:
                d = {}
        d[key] = {"p2p_chunk": chunk, "ms": times}
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        json.dump(d, open(cache, "w"), indent=1)
    return chunk, times


def _time_graph(op, src, q, trg, reps, grad):
    """Median of `reps` CUDA-graph replays of one batch execute (CUDA events)."""
    import statistics
    import torch
    graph, _ = op.capture(src, q, trg, grad=grad)
    torch.cuda.synchronize()
    graph.replay()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        graph.replay()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    del graph
    return statistics.median(ts)


def tune_batch(kernel, cells, src_counts, src, q, trg=None, trg_counts=None, precision="mixed", nrhs=1, tol=1e-6,
               chunks=(1024, 2048, 4096, 8192, 16384), crossovers=(32, 64, 128, None), reps=3, grad=False, cache=None,
               key=None):
    """Tune a batch's execution choices by timing CUDA-graph replays:

      - the direct / NUFFT crossover: cells with M >= crossover take the NUFFT
        south/north path (None: no NUFFT), M from each cell's plan;
      - the ES spreading width w of the NUFFT cells, among the widths whose
        error bound meets the tolerance (w >= ceil(log10(1/tol)) + 1, up to
        the plan's default ceil(log10(1/tol)) + 2);
      - the P2P source chunk.

    Coordinate search in that order, each step keeping the best so far.
    Every candidate is exact to the tolerance by construction (both paths and
    every admissible width meet it), so the choice is by time alone.  Returns
    (config, timings) with config = {"crossover", "nufft_w", "p2p_chunk"}; with
    a cache path and key the result persists as JSON.  Build the tuned batch
    with tuned_batch(kernel, cells, src_counts, config, ...)."""
    import json
    import math
    import os
    if cache and key and os.path.exists(cache):
        try:
            d = json.load(open(cache))
            if key in d:
                return d[key]["config"], d[key]["ms"]
        except Exception:
            pass
    # ceil(log10(1/tol)) with a guard below (log10 of an exact power of ten
    # may round up past the integer)
    wmin = max(2, math.ceil(math.log10(1.0 / tol) - 1e-9) + 1)
    widths = tuple(range(wmin, min(16, wmin + 1) + 1))
    timings = {}

    def run(cfg):
        name = json.dumps(cfg, sort_keys=True)
        if name not in timings:
            op = tuned_batch(kernel, cells, src_counts, cfg, trg_counts=trg_counts, precision=precision, nrhs=nrhs,
                             tol=tol)
            timings[name] = _time_graph(op, src, q, trg, reps, grad)
            del op
        return timings[name]

    cfg = {"crossover": 64, "nufft_w": 0, "p2p_chunk": 4096}
    for field, cands in (("crossover", crossovers), ("nufft_w", widths), ("p2p_chunk", chunks)):
        best = None
        for c in cands:
            trial = dict(cfg, **{field: c})
            t = run(trial)
            if best is None or t < best[0]:
                best = (t, c)
        cfg[field] = best[1]
    if cache and key:
        d = {}
        if os.path.exists(cache):
            try:
                d = json.load(open(cache))
            except Exception:
                d = {}
        d[key] = {"config": cfg, "ms": timings}
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        json.dump(d, open(cache, "w"), indent=1)
    return cfg, timings


def tuned_batch(kernel, cells, src_counts, config, trg_counts=None, precision="mixed", nrhs=1, tol=1e-6):
    """A BatchOp with tune_batch's choices: per-cell path from the crossover on
    the cell's mode count M, the ES width for its NUFFT cells, the P2P chunk."""
    cx = config.get("crossover")
    w = int(config.get("nufft_w") or 0)
    cc = []
    for c in cells:
        m = PeriodicOp(kernel, c["e1"], c["e2"], beta=c.get("beta", 0.0), tol=c.get("tol", tol), precision=precision,
                       nrhs=nrhs, ns_max=1, nt_max=1).describe()["M"]
        nufft = cx is not None and m >= cx and m <= 2047  # the single-block FFT holds fine grids up to 8192
        cc.append(dict(c, path="nufft" if nufft else "direct", nufft_w=w if nufft else 0))
    return BatchOp(kernel, cc, src_counts, trg_counts, precision=precision, nrhs=nrhs, tol=tol,
                   p2p_chunk=int(config.get("p2p_chunk") or 0))


def _adjoint(op, src, q, trg, g, grad_fwd, need_q, need_s, need_t):
    import torch
    self_t = trg is None
    tr = src if self_t else trg
    ns, nt = src.shape[1], tr.shape[1]
    g = g.contiguous()
    _check_tensor("grad of the output", g, (op.nrhs, 2, nt) if op.kernel in _VEC else (op.nrhs, nt), src.device)
    dq = torch.empty_like(q) if need_q else None
    dsrc = torch.empty_like(src) if need_s else None
    if self_t and need_s and need_t:
        dtrg = dsrc  # one array receives both roles
    else:
        dtrg = torch.empty_like(tr) if (need_t and not self_t) else None
    ws = op.workspace()
    st = torch.cuda.current_stream(src.device).cuda_stream
    _lib.check(_lib.lib().pfmm_execute_adjoint(op._h, _ptr(ws), ws.numel(), ns, _ptr(src), _ptr(q), nt, _ptr(tr),
                                               _ptr(g), _ptr(grad_fwd), _ptr(dq), _ptr(dsrc), _ptr(dtrg),
                                               ctypes.c_void_p(st)))
    return dq, dsrc, (None if self_t else dtrg)


def _make_function():
    import torch

    class PeriodicFunction(torch.autograd.Function):
        """u = K^(p) q as a differentiable function of (src, q, trg).  Backward
        runs pfmm_execute_adjoint (the operator with sources and targets swapped,
        derivative-kernel evaluation for positions); nothing but the inputs and
        the forward gradient is stored.  Derivatives through the gradient output
        (second derivatives of G) are not provided."""

        @staticmethod
        def forward(ctx, op, src, q, trg):
            pot, grad = op(src, q, trg, grad=op.kernel not in _VEC)
            ctx.op = op
            ctx.self_t = trg is None
            ctx.save_for_backward(src, q, trg if trg is not None else src, grad if grad is not None else pot)
            if grad is not None:
                ctx.mark_non_differentiable(grad)
                return pot, grad
            return pot

        @staticmethod
        def backward(ctx, g_pot, *rest):
            src, q, trg, grad = ctx.saved_tensors
            op = ctx.op
            need_s, need_q, need_t = ctx.needs_input_grad[1], ctx.needs_input_grad[2], ctx.needs_input_grad[3]
            if ctx.self_t:
                need_t = need_s
            vec = op.kernel in _VEC  # Stokes kernels: strengths only
            dq, dsrc, dtrg = _adjoint(op, src, q, None if ctx.self_t else trg, g_pot, None if vec else grad,
                                      need_q, need_s and not vec, need_t and not vec)
            return None, dsrc, dq, dtrg

    return PeriodicFunction


_FN = None


def periodic(op, src, q, trg=None):
    """Differentiable application of a PeriodicOp: returns pot (and, for the
    scalar kernels, the gradient as a non-differentiable second output)."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(op, src, q, trg)
