"""ctypes binding of include/pfmm.h (argument marshalling only).

Loads the in-tree libpfmm.so.  There is no fallback: if the library is
missing or fails to load, every call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# PFMM_LIB overrides the library path (profiling experiments only)
LIB_PATH = os.environ.get("PFMM_LIB") or os.path.join(HERE, "libpfmm.so")

PFMM_LAPLACE, PFMM_MODHELM, PFMM_STOKES, PFMM_MSTOKES = 0, 1, 2, 3
PFMM_FP64, PFMM_MIXED = 0, 1
PFMM_PATH_AUTO, PFMM_PATH_DIRECT, PFMM_PATH_NUFFT = 0, 1, 2
PFMM_FAR_ONLY, PFMM_NEAR_ONLY, PFMM_NO_GRAD, PFMM_PROJECT_NEUTRAL, PFMM_SINGLY_PERIODIC = 1, 2, 4, 8, 16
PFMM_WE_ROTATED, PFMM_WE_AXIS = 32, 64
PFMM_NEAR_DIRECT, PFMM_NEAR_FMM, PFMM_DETERMINISTIC = 128, 256, 512

STATUS = {0: "PFMM_OK", 1: "PFMM_ERR_INVALID_ARG", 2: "PFMM_ERR_LATTICE", 3: "PFMM_ERR_NOT_NEUTRAL",
          4: "PFMM_ERR_TOLERANCE", 5: "PFMM_ERR_WORKSPACE", 6: "PFMM_ERR_CUDA", 7: "PFMM_ERR_NONFINITE",
          8: "PFMM_ERR_TIMEOUT", 9: "PFMM_ERR_INTERNAL"}

# Every symbol declared in include/pfmm.h (checked by the CPU test suite).
EXPORTS = ["pfmm_plan_create", "pfmm_workspace_size", "pfmm_workspace_size_host", "pfmm_plan_describe",
           "pfmm_execute", "pfmm_execute_host", "pfmm_get_status", "pfmm_last_error", "pfmm_plan_destroy",
           "pfmm_version", "pfmm_profile_enable", "pfmm_profile_read", "pfmm_profile_pairs", "pfmm_execute_static",
           "pfmm_batch_create", "pfmm_batch_workspace_size", "pfmm_batch_execute", "pfmm_batch_get_status",
           "pfmm_batch_destroy", "pfmm_batch_profile_enable", "pfmm_batch_profile_read", "pfmm_execute_adjoint",
           "pfmm_stokes_pressure", "pfmm_near_stats"]


class Opts(ctypes.Structure):
    _fields_ = [("e1", ctypes.c_double * 2), ("e2", ctypes.c_double * 2), ("kernel", ctypes.c_int),
                ("beta", ctypes.c_double), ("tol", ctypes.c_double), ("precision", ctypes.c_int),
                ("path", ctypes.c_int), ("nufft_w", ctypes.c_int), ("n_gl", ctypes.c_int),
                ("nrhs", ctypes.c_int), ("flags", ctypes.c_uint), ("near_order", ctypes.c_int),
                ("near_leaf", ctypes.c_int)]


class PlanDesc(ctypes.Structure):
    _fields_ = [("d", ctypes.c_double), ("xi", ctypes.c_double), ("eta", ctypes.c_double),
                ("rot", ctypes.c_double * 4), ("m0", ctypes.c_int), ("M", ctypes.c_int), ("mode0", ctypes.c_int),
                ("Nq", ctypes.c_int), ("path", ctypes.c_int), ("n_gl", ctypes.c_int), ("nf", ctypes.c_int),
                ("nufft_w", ctypes.c_int), ("es_beta", ctypes.c_double), ("nlaunch", ctypes.c_int),
                ("npairs", ctypes.c_int64), ("we_rotated", ctypes.c_int), ("we_dir", ctypes.c_double * 2),
                ("near_fmm", ctypes.c_int), ("near_order", ctypes.c_int), ("near_leaf", ctypes.c_int),
                ("near_theta", ctypes.c_double),
                ("p1_nufft_nodes", ctypes.c_int)]


class PfmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpfmm.so not built ({LIB_PATH}); run paper_2111_01083_gb300.build.build_library()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    L.pfmm_plan_create.argtypes = [ctypes.POINTER(Opts), i64, i64, ctypes.POINTER(vp)]
    L.pfmm_plan_create.restype = ctypes.c_int
    L.pfmm_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
    L.pfmm_workspace_size.restype = ctypes.c_int
    L.pfmm_workspace_size_host.argtypes = [vp, ctypes.POINTER(sz)]
    L.pfmm_workspace_size_host.restype = ctypes.c_int
    L.pfmm_plan_describe.argtypes = [vp, ctypes.POINTER(PlanDesc)]
    L.pfmm_plan_describe.restype = ctypes.c_int
    L.pfmm_execute.argtypes = [vp, vp, sz, i64, vp, vp, i64, vp, vp, vp, vp]
    L.pfmm_execute.restype = ctypes.c_int
    L.pfmm_execute_host.argtypes = [vp, vp, sz, i64, vp, vp, i64, vp, vp, vp, vp]
    L.pfmm_execute_host.restype = ctypes.c_int
    L.pfmm_execute_static.argtypes = [vp, i64, vp, vp, i64, vp, vp, vp, vp]
    L.pfmm_execute_static.restype = ctypes.c_int
    L.pfmm_batch_create.argtypes = [ctypes.POINTER(Opts), ctypes.c_int, ctypes.POINTER(i64), ctypes.POINTER(i64),
                                    ctypes.c_int, ctypes.POINTER(vp)]
    L.pfmm_batch_create.restype = ctypes.c_int
    L.pfmm_batch_workspace_size.argtypes = [vp, ctypes.POINTER(sz)]
    L.pfmm_batch_workspace_size.restype = ctypes.c_int
    L.pfmm_batch_execute.argtypes = [vp, vp, sz, vp, vp, vp, vp, vp, vp]
    L.pfmm_batch_execute.restype = ctypes.c_int
    L.pfmm_batch_get_status.argtypes = [vp, vp, vp]
    L.pfmm_batch_get_status.restype = ctypes.c_int
    L.pfmm_batch_profile_enable.argtypes = [vp, ctypes.c_int]
    L.pfmm_batch_profile_enable.restype = ctypes.c_int
    L.pfmm_batch_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_double)]
    L.pfmm_batch_profile_read.restype = ctypes.c_int
    L.pfmm_batch_destroy.argtypes = [vp]
    L.pfmm_batch_destroy.restype = None
    L.pfmm_execute_adjoint.argtypes = [vp, vp, sz, i64, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp]
    L.pfmm_execute_adjoint.restype = ctypes.c_int
    L.pfmm_stokes_pressure.argtypes = [vp, vp, sz, i64, vp, vp, i64, vp, vp, vp]
    L.pfmm_stokes_pressure.restype = ctypes.c_int
    L.pfmm_get_status.argtypes = [vp, vp, vp]
    L.pfmm_get_status.restype = ctypes.c_int
    L.pfmm_last_error.argtypes = []
    L.pfmm_last_error.restype = ctypes.c_char_p
    L.pfmm_plan_destroy.argtypes = [vp]
    L.pfmm_plan_destroy.restype = None
    L.pfmm_profile_enable.argtypes = [vp, ctypes.c_int]
    L.pfmm_profile_enable.restype = ctypes.c_int
    L.pfmm_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    L.pfmm_profile_read.restype = ctypes.c_int
    L.pfmm_profile_pairs.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_double)]
    L.pfmm_profile_pairs.restype = ctypes.c_int
    L.pfmm_near_stats.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_int64)]
    L.pfmm_near_stats.restype = ctypes.c_int
    L.pfmm_version.argtypes = []
    L.pfmm_version.restype = ctypes.c_char_p
    _lib = L
    return L


def check(code):
    if code != 0:
        raise PfmmError(code, lib().pfmm_last_error().decode())
