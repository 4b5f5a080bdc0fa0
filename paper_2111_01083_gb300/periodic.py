"""Python front end of the C ABI (argument marshalling only; PyTorch supplies
device memory and the current CUDA stream).

    op = PeriodicOp("laplace", e1=(16, 0), e2=(0, 1), tol=1e-6, precision="mixed",
                    ns_max=N, nt_max=N)
    pot, grad = op(src, q)            # targets = sources
    vel, _ = stokes_op(src, f, trg)   # Stokes: velocity

Tensors: src/trg [2, n] float64 (CUDA), q [nrhs, n] or [nrhs, 2, n] (Stokes).
Outputs: pot [nrhs, nt] (Stokes: [nrhs, 2, nt]), grad [nrhs, 2, nt] or None.
Every step of the computation runs in the CUDA library; nothing here
computes.
"""
import ctypes

import numpy as np

from . import _lib

_KER = {"laplace": _lib.PFMM_LAPLACE, "modhelm": _lib.PFMM_MODHELM, "stokes": _lib.PFMM_STOKES}
_PREC = {"fp64": _lib.PFMM_FP64, "mixed": _lib.PFMM_MIXED}
_PATH = {"auto": _lib.PFMM_PATH_AUTO, "direct": _lib.PFMM_PATH_DIRECT, "nufft": _lib.PFMM_PATH_NUFFT}
_PART = {"total": 0, "far": _lib.PFMM_FAR_ONLY, "near": _lib.PFMM_NEAR_ONLY}


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class PeriodicOp:
    def __init__(self, kernel, e1, e2, beta=0.0, tol=1e-6, precision="mixed", path="auto", nufft_w=0, n_gl=0,
                 nrhs=1, part="total", ns_max=0, nt_max=0, device=None):
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
        o.flags = _PART[part]
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
        return {k: (list(getattr(d, k)) if k == "rot" else getattr(d, k)) for k, _ in d._fields_}

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
        assert src.dtype == torch.float64 and src.is_cuda and src.is_contiguous()
        self_t = trg is None
        if self_t:
            trg = src
        ns, nt = src.shape[1], trg.shape[1]
        stokes = self.kernel == "stokes"
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
        stokes = self.kernel == "stokes"
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

    def phase_ms(self):
        """Milliseconds of [prep, far field, near P2P] of the last execute."""
        ms = (ctypes.c_float * 3)()
        _lib.check(_lib.lib().pfmm_profile_read(self._h, ms, 3))
        return list(ms)

    def status(self, stream=None):
        """Synchronise and return the device status of the last execute (raises on error)."""
        import torch
        ws = self.workspace()
        st = stream if stream is not None else torch.cuda.current_stream(ws.device).cuda_stream
        _lib.check(_lib.lib().pfmm_get_status(self._h, _ptr(ws), ctypes.c_void_p(st)))
