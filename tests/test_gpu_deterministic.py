"""PFMM_DETERMINISTIC: two executes on the same inputs give bit-identical
outputs (no order-dependent atomics on the path), and the results still meet
the parity tolerances against the oracle."""
import numpy as np
import pytest

import workloads
from gpu_util import oracle, run_lib
from oracle import api as oapi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel,e1,e2,ns,nt,beta,precision,tol", [
    ("laplace", (16.0, 0.0), (0.0, 1.0), 6000, None, 0.0, "mixed", 1e-6),
    ("stokes", (1.0, 0.0), (0.3, 0.8), 3000, 2000, 0.0, "mixed", 1e-6),
    ("modhelm", (8.0, 0.0), (0.0, 1.0), 3000, None, 2.0, "mixed", 1e-6),
    ("laplace", (2.0, 0.0), (0.4, 1.0), 1500, 1200, 0.0, "fp64", 1e-10),
])
def test_deterministic_repeat(kernel, e1, e2, ns, nt, beta, precision, tol):
    rng = np.random.default_rng(ns)
    src = workloads.points(rng, e1, e2, ns, "gmm")
    q = workloads.strengths(rng, 2, ns, stokes=kernel == "stokes", neutral=kernel != "modhelm")
    trg = None if nt is None else workloads.points(rng, e1, e2, nt)
    grad = kernel != "stokes"
    kw = dict(beta=beta, tol=tol, precision=precision, path="auto", grad=grad, deterministic=True)
    a = run_lib(kernel, e1, e2, src, q, trg, **kw)
    b = run_lib(kernel, e1, e2, src, q, trg, **kw)
    assert np.array_equal(a[0], b[0])
    if grad:
        assert np.array_equal(a[1], b[1])
    tt = src if trg is None else trg
    idx = rng.choice(tt.shape[1], 200, replace=False)
    ref = oracle(kernel, e1, e2, src, q, tt[:, idx], beta=beta, grad=grad)
    mc = kernel != "modhelm"
    assert oapi.rel_err(a[0][..., idx], ref[0], modconst=mc) < tol
    if grad:
        assert oapi.rel_err(a[1][..., idx], ref[1]) < tol
