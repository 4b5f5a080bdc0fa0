"""pfmm_execute_static: the allocation-free entry point.

Some callers cannot allocate device memory (a C host program that only gets
device pointers from elsewhere, or code that must not call cudaMalloc
between launches because it synchronises the device).  For them the library
runs the operator on a fixed scratch array compiled into it.  This test calls
that entry point through the C ABI twice in a row and checks each result
against pfmm_execute with an ordinary workspace, at the tolerances of the
other parity tests.  It lives in a file of its own, collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_execute_static_matches_execute(precision, tol):
    import torch
    from paper_2111_01083_gb300 import PeriodicOp, _lib
    from paper_2111_01083_gb300.periodic import _ptr

    dev = torch.device("cuda", 0)
    e1, e2 = (6.0, 0.0), (0.7, 1.0)
    rng = np.random.default_rng(31)
    src = torch.tensor(workloads.points(rng, e1, e2, 3000, "gmm"), device=dev)
    q = torch.tensor(workloads.strengths(rng, 2, 3000), device=dev)
    trg = torch.tensor(workloads.points(rng, e1, e2, 1100), device=dev)
    op = PeriodicOp("laplace", e1, e2, tol=tol, precision=precision, nrhs=2, ns_max=3000, nt_max=1100)
    ref_pot, ref_grad = op(src, q, trg)
    torch.cuda.synchronize()
    L = _lib.lib()
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for _ in range(2):
        pot = torch.full_like(ref_pot, float("nan"))
        grad = torch.full_like(ref_grad, float("nan"))
        _lib.check(L.pfmm_execute_static(op._h, 3000, _ptr(src), _ptr(q), 1100, _ptr(trg), _ptr(pot), _ptr(grad), st))
        torch.cuda.synchronize()
        dp = (pot - pot.mean(-1, keepdim=True)) - (ref_pot - ref_pot.mean(-1, keepdim=True))
        assert float(dp.norm() / (ref_pot - ref_pot.mean(-1, keepdim=True)).norm()) < tol
        assert float((grad - ref_grad).norm() / ref_grad.norm()) < tol


def test_execute_static_rejects_large_plans():
    from paper_2111_01083_gb300 import PeriodicOp, _lib
    op = PeriodicOp("laplace", (1.0, 0.0), (0.0, 1.0), tol=1e-6, ns_max=2_000_000, nt_max=2_000_000)
    code = _lib.lib().pfmm_execute_static(op._h, 10, None, None, 10, None, None, None, None)
    assert code == 5  # PFMM_ERR_WORKSPACE
    assert b"static array" in _lib.lib().pfmm_last_error()


def test_execute_static_reports_device_status():
    """Conditions only the kernels can see (here a NaN strength) land in the
    static array's status word; pfmm_get_status with a NULL workspace reads
    and clears it, and a clean call afterwards reports PFMM_OK."""
    import torch
    from paper_2111_01083_gb300 import PeriodicOp, _lib
    from paper_2111_01083_gb300.periodic import _ptr

    dev = torch.device("cuda", 0)
    e1, e2 = (2.0, 0.0), (0.3, 1.0)
    rng = np.random.default_rng(7)
    src = torch.tensor(workloads.points(rng, e1, e2, 500), device=dev)
    q = torch.tensor(workloads.strengths(rng, 1, 500), device=dev)
    op = PeriodicOp("laplace", e1, e2, tol=1e-6, precision="mixed", ns_max=500, nt_max=500)
    pot = torch.empty((1, 500), dtype=torch.float64, device=dev)
    grad = torch.empty((1, 2, 500), dtype=torch.float64, device=dev)
    L = _lib.lib()
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    bad = q.clone()
    bad[0, 17] = float("nan")
    _lib.check(L.pfmm_execute_static(op._h, 500, _ptr(src), _ptr(bad), 500, _ptr(src), _ptr(pot), _ptr(grad), st))
    assert L.pfmm_get_status(op._h, None, st) == 7  # PFMM_ERR_NONFINITE
    _lib.check(L.pfmm_execute_static(op._h, 500, _ptr(src), _ptr(q), 500, _ptr(src), _ptr(pot), _ptr(grad), st))
    assert L.pfmm_get_status(op._h, None, st) == 0
