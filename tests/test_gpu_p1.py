"""GPU parity of the singly periodic operator P1 (PFMM_SINGLY_PERIODIC)
against the P1 oracle (oracle/p1.py: near images |m| <= 1 plus the row-0
west/east factorization, itself pinned to the closed forms, series and image
sums), all kernels, FP64 (1e-10) and mixed (1e-6), on tall, skewed and
rotated strips; and the status for a point outside the strip."""
import numpy as np
import pytest

import workloads
from gpu_util import errs, run_lib
from oracle import p1

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "mixed": 1e-6}
STRIPS = {
    "tall": ((1.0, 0.0), (0.0, 2.5)),
    "skew": ((2.0, 0.0), (0.7, 0.5)),
    "rotated": ((1.2, 0.5), (-0.3, 1.9)),
}


def _points(e1, e2, n, rng, frac=0.98):
    """Input-frame points inside the strip: u1 any, |u2| < frac / 2."""
    u1 = rng.uniform(-0.5, 0.5, n)
    u2 = rng.uniform(-0.5, 0.5, n) * frac
    e1, e2 = np.asarray(e1), np.asarray(e2)
    return u1[None, :] * e1[:, None] + u2[None, :] * e2[:, None]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("strip", ["tall", "skew", "rotated"])
@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 1.5), ("stokes", 0.0)])
def test_p1_total(precision, strip, kernel, beta):
    e1, e2 = STRIPS[strip]
    rng = np.random.default_rng(71)
    ns, nt = 700, 300
    src = _points(e1, e2, ns, rng)
    trg = _points(e1, e2, nt, rng)
    stokes = kernel == "stokes"
    q = workloads.strengths(rng, 2, ns, stokes=stokes, neutral=kernel != "modhelm")
    got = run_lib(kernel, e1, e2, src, q, trg, beta=beta, tol=TOL[precision], precision=precision,
                  grad=not stokes, singly=True)
    ref = p1.evaluate(kernel, beta, e1, e2, src, q, trg, want_grad=not stokes)
    ep, eg = errs(kernel, got, ref)
    assert ep < TOL[precision], ep
    if eg is not None:
        assert eg < TOL[precision], eg


def test_p1_laplace_matches_closed_form_self():
    """Targets = sources (self pairs excluded) against the closed-form kernel."""
    e1, e2 = (1.5, 0.0), (0.0, 3.0)
    rng = np.random.default_rng(72)
    n = 900
    src = _points(e1, e2, n, rng)
    q = workloads.strengths(rng, 1, n)
    pot, grad, _ = run_lib("laplace", e1, e2, src, q, None, tol=1e-10, precision="fp64", singly=True)
    cell = p1.canonical_strip(e1, e2)
    s = p1.wrap_strip(src, cell)
    rp, rg = p1.laplace_closed(cell, s, s, q)
    ep, eg = errs("laplace", (pot, grad), (rp, np.einsum("ij,rjn->rin", cell["rot"].T, rg)))
    assert ep < 1e-10 and eg < 1e-10, (ep, eg)


def test_p1_point_outside_strip_is_reported():
    from paper_2111_01083_gb300._lib import PfmmError
    e1, e2 = (1.0, 0.0), (0.0, 1.0)
    rng = np.random.default_rng(73)
    src = _points(e1, e2, 50, rng)
    src[1, 7] = 0.7  # beyond eta / 2
    q = workloads.strengths(rng, 1, 50)
    with pytest.raises(PfmmError):
        run_lib("laplace", e1, e2, src, q, None, tol=1e-6, precision="mixed", singly=True)


TALL = {
    "1x16": ((1.0, 0.0), (0.0, 16.0)),
    "rot1x12": ((0.8, 0.6), (-7.2, 9.6)),
    "skew1x10": ((1.0, 0.0), (0.4, 10.0)),
}


_TALL_CACHE = {}


def _tall_case(strip, kernel, beta):
    """Seeded input and its oracle field, shared by both precisions."""
    key = (strip, kernel, beta)
    if key not in _TALL_CACHE:
        e1, e2 = TALL[strip]
        rng = np.random.default_rng(81)
        ns, nt = 2000, 300
        src = _points(e1, e2, ns, rng)
        trg = _points(e1, e2, nt, rng)
        stokes = kernel == "stokes"
        q = workloads.strengths(rng, 2, ns, stokes=stokes, neutral=kernel != "modhelm")
        ref = p1.evaluate(kernel, beta, e1, e2, src, q, trg, want_grad=not stokes)
        _TALL_CACHE[key] = (src, q, trg, ref)
    return _TALL_CACHE[key]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("strip", list(TALL))
@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 1.5), ("stokes", 0.0)])
def test_p1_nufft_total(precision, strip, kernel, beta):
    """Tall strips on the NUFFT path (the west/east sums through GL lines in
    x, a type-1 transform in y and ES interpolation onto the nodes) against
    the P1 oracle."""
    e1, e2 = TALL[strip]
    src, q, trg, ref = _tall_case(strip, kernel, beta)
    stokes = kernel == "stokes"
    pot, g, op = run_lib(kernel, e1, e2, src, q, trg, beta=beta, tol=TOL[precision], precision=precision,
                         grad=not stokes, singly=True, path="nufft")
    d = op.describe()
    assert d["path"] == 2 and d["p1_nufft_nodes"] > 0, d
    ep, eg = errs(kernel, (pot, g), ref)
    assert ep < TOL[precision], ep
    if eg is not None:
        assert eg < TOL[precision], eg


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 0.5), ("stokes", 0.0)])
def test_p1_nufft_far_matches_direct(precision, kernel, beta):
    """The far part alone (1 x 24 strip, targets = sources) through the
    transforms and through the direct kernels on the same input: equal to
    the tolerance relative to the far part itself (modulo the constant the
    two Laplace/Stokes gauges differ by)."""
    e1, e2 = (1.0, 0.0), (0.0, 24.0)
    rng = np.random.default_rng(82)
    n = 5000
    src = _points(e1, e2, n, rng)
    stokes = kernel == "stokes"
    q = workloads.strengths(rng, 1, n, stokes=stokes, neutral=kernel != "modhelm")
    kw = dict(beta=beta, tol=TOL[precision], precision=precision, grad=not stokes, singly=True, part="far")
    pn, gn, op = run_lib(kernel, e1, e2, src, q, None, path="nufft", **kw)
    assert op.describe()["p1_nufft_nodes"] > 0
    pd, gd, _ = run_lib(kernel, e1, e2, src, q, None, path="direct", **kw)
    ep, eg = errs(kernel, (pn, gn), (pd, gd))
    assert ep < TOL[precision], ep
    if eg is not None:
        assert eg < TOL[precision], eg
