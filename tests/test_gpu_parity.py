"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Tolerances (relative l2 over all targets and rhs; Laplace potentials and
Stokes velocities modulo the best-fit constant):
  FP64 path : 1e-10 (tol = 1e-10 requested)
  mixed path: 1e-6  (tol = 1e-6 requested)
Sizes span several 128-wide P2P tiles and the 64-wide formation sub-tiles
with ragged tails.
"""
import numpy as np
import pytest

import workloads
from gpu_util import errs, oracle, run_lib

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}
LAT = {
    "square": ((1.0, 0.0), (0.0, 1.0)),
    "rect4": ((4.0, 0.0), (0.0, 1.0)),
    "skew": ((1.0, 0.0), (0.3, 0.8)),
    "rotated": ((1.2, 0.4), (-0.5, 0.9)),
    "aspect16": ((16.0, 0.0), (0.0, 1.0)),
}


def _case(kernel, lat, ns, nt=None, seed=0, dist="uniform", nrhs=1):
    e1, e2 = LAT[lat]
    rng = np.random.default_rng(seed)
    src = workloads.points(rng, e1, e2, ns, dist)
    q = workloads.strengths(rng, nrhs, ns, stokes=kernel == "stokes", neutral=kernel != "modhelm")
    trg = None if nt is None else workloads.points(rng, e1, e2, nt)
    return e1, e2, src, q, trg


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("lat", ["square", "skew", "rotated", "aspect16"])
def test_laplace_total(precision, lat):
    e1, e2, src, q, trg = _case("laplace", lat, 700, seed=1)
    got = run_lib("laplace", e1, e2, src, q, trg, tol=TOL[precision], precision=precision)
    ref = oracle("laplace", e1, e2, src, q, trg)
    ep, eg = errs("laplace", got, ref)
    assert ep < TOL[precision] and eg < TOL[precision], (ep, eg)


def test_laplace_square_n1000_fp64():
    """The 1000-charge square-cell workload (seed 0), potential + gradient."""
    w = workloads.make("laplace_square_n1000")
    got = run_lib("laplace", w["e1"], w["e2"], w["src"], w["q"], None, tol=1e-10, precision="fp64")
    ref = oracle("laplace", w["e1"], w["e2"], w["src"], w["q"], None)
    ep, eg = errs("laplace", got, ref)
    assert ep < 1e-10 and eg < 1e-10, (ep, eg)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("lat", ["square", "skew", "rotated"])
def test_stokes_total_separate_targets(precision, lat):
    e1, e2, src, f, trg = _case("stokes", lat, 600, nt=333, seed=2)
    got = run_lib("stokes", e1, e2, src, f, trg, tol=TOL[precision], precision=precision, grad=False)
    ref = oracle("stokes", e1, e2, src, f, trg, grad=False)
    ep, _ = errs("stokes", got, ref)
    assert ep < TOL[precision], ep


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("beta,lat", [(1.0, "square"), (1.0, "rect4"), (10.0, "skew"), (3.0, "rotated")])
def test_modhelm_total_multi_rhs(precision, beta, lat):
    e1, e2, src, q, trg = _case("modhelm", lat, 500, seed=3, nrhs=3)
    got = run_lib("modhelm", e1, e2, src, q, trg, beta=beta, tol=TOL[precision], precision=precision)
    ref = oracle("modhelm", e1, e2, src, q, trg, beta=beta)
    ep, eg = errs("modhelm", got, ref)
    assert ep < TOL[precision] and eg < TOL[precision], (ep, eg)


@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 2.0), ("stokes", 0.0)])
@pytest.mark.parametrize("part", ["far", "near"])
def test_parts_fp64(kernel, beta, part):
    e1, e2, src, q, trg = _case(kernel, "skew", 400, nt=257, seed=4)
    g = kernel != "stokes"
    got = run_lib(kernel, e1, e2, src, q, trg, beta=beta, tol=1e-10, precision="fp64", part=part, grad=g)
    ref = oracle(kernel, e1, e2, src, q, trg, beta=beta, part=part, grad=g)
    ep, eg = errs(kernel, got, ref)
    scale = 1e-10 if part == "near" else 1e-9  # far part alone is small: relative to itself
    assert ep < scale, ep
    if g:
        assert eg < scale, eg


def test_coincident_target_is_skipped():
    """A target placed exactly on a source: the zero-distance pair is skipped
    (the oracle uses the regular limit on the periodic side and skips it in the
    near sum; both give the same total)."""
    e1, e2, src, q, _ = _case("laplace", "rect4", 300, seed=5)
    trg = np.concatenate([src[:, :7], workloads.points(np.random.default_rng(9), e1, e2, 50)], axis=1)
    got = run_lib("laplace", e1, e2, src, q, trg, tol=1e-10, precision="fp64")
    ref = oracle("laplace", e1, e2, src, q, trg)
    ep, eg = errs("laplace", got, ref)
    assert ep < 1e-10 and eg < 1e-10


@pytest.mark.parametrize("ns,nt", [(1, 5), (2, 1), (129, 1), (300, 0)])
def test_tiny_and_empty(ns, nt):
    e1, e2 = LAT["rotated"]
    rng = np.random.default_rng(6)
    src = workloads.points(rng, e1, e2, ns)
    q = rng.standard_normal((1, ns))
    trg = workloads.points(rng, e1, e2, nt)
    got = run_lib("modhelm", e1, e2, src, q, trg, beta=1.5, tol=1e-10, precision="fp64")
    if nt == 0:
        assert got[0].shape == (1, 0)
        return
    ref = oracle("modhelm", e1, e2, src, q, trg, beta=1.5)
    ep, eg = errs("modhelm", got, ref)
    assert ep < 1e-10 and eg < 1e-10


def test_mixed_matches_fp64_gpu():
    """Mixed vs FP64 GPU path on the same input (aspect-16 Gaussian mixture)."""
    e1, e2, src, q, _ = _case("laplace", "aspect16", 3000, seed=7, dist="gmm")
    a = run_lib("laplace", e1, e2, src, q, None, tol=1e-6, precision="mixed")
    b = run_lib("laplace", e1, e2, src, q, None, tol=1e-10, precision="fp64")
    ep, eg = errs("laplace", a, b)
    assert ep < 1e-6 and eg < 1e-6, (ep, eg)


def test_nonfinite_input_reported():
    from paper_2111_01083_gb300._lib import PfmmError
    e1, e2, src, q, _ = _case("laplace", "square", 64, seed=8)
    q = q.copy()
    q[0, 5] = np.nan
    with pytest.raises(PfmmError, match="NONFINITE"):
        run_lib("laplace", e1, e2, src, q, None, tol=1e-6)


def test_not_neutral_reported():
    from paper_2111_01083_gb300._lib import PfmmError
    e1, e2, src, q, _ = _case("laplace", "square", 64, seed=8)
    with pytest.raises(PfmmError, match="NOT_NEUTRAL"):
        run_lib("laplace", e1, e2, src, q + 0.1, None, tol=1e-6)


# ---------------------------------------------------------------------------
# NUFFT path (Sec. 6, Eqs. fastanterp / fastinterp)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("e1,e2", [((8.0, 0.0), (0.0, 1.0)), ((16.0, 0.0), (3.0, 1.0)), ((40.0, 0.0), (0.0, 1.0))])
def test_laplace_nufft_path(precision, e1, e2):
    rng = np.random.default_rng(11)
    src = workloads.points(rng, e1, e2, 1500, "gmm")
    q = workloads.strengths(rng, 2, 1500)
    trg = workloads.points(rng, e1, e2, 400)
    tol = TOL[precision]
    for part in ("far", "total"):
        got = run_lib("laplace", e1, e2, src, q, trg, tol=tol, precision=precision, part=part, path="nufft")
        assert got[2].describe()["path"] == 2
        ref = oracle("laplace", e1, e2, src, q, trg, part=part)
        if part == "far":
            # far part alone, measured against the total field's scale (the quantity the tolerance is for)
            tot = oracle("laplace", e1, e2, src, q, trg, part="total")
            sc_p = np.linalg.norm(tot[0] - tot[0].mean(-1, keepdims=True))
            d = (got[0] - got[0].mean(-1, keepdims=True)) - (ref[0] - ref[0].mean(-1, keepdims=True))
            assert np.linalg.norm(d) / sc_p < tol
            assert np.linalg.norm(got[1] - ref[1]) / np.linalg.norm(tot[1]) < tol
        else:
            ep, eg = errs("laplace", got, ref)
            assert ep < tol and eg < tol, (ep, eg)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kernel,beta", [("modhelm", 0.5), ("modhelm", 3.0), ("stokes", 0.0)])
@pytest.mark.parametrize("e1,e2", [((40.0, 0.0), (0.0, 1.0)), ((48.0, 0.0), (0.5, 1.0))])
def test_nufft_path_modhelm_stokes(precision, kernel, beta, e1, e2):
    """Modified Helmholtz (m = 0 mode included, chi = sqrt(alpha^2 + beta^2))
    and Stokes (four spread channels, 2 x 2 weight blocks) through the NUFFT
    south/north path; far part against the total field's scale, and the total."""
    stokes = kernel == "stokes"
    mc = kernel != "modhelm"
    rng = np.random.default_rng(13)
    src = workloads.points(rng, e1, e2, 1500, "gmm")
    q = workloads.strengths(rng, 2, 1500, stokes=stokes, neutral=mc)
    trg = workloads.points(rng, e1, e2, 400)
    tol = TOL[precision]
    tot = oracle(kernel, e1, e2, src, q, trg, beta=beta, part="total", grad=not stokes)
    cen = (lambda a: a - a.mean(-1, keepdims=True)) if mc else (lambda a: a)
    for part in ("far", "total"):
        got = run_lib(kernel, e1, e2, src, q, trg, beta=beta, tol=tol, precision=precision, part=part,
                      path="nufft", grad=not stokes)
        desc = got[2].describe()
        assert desc["path"] == 2 and desc["M"] >= 48
        ref = tot if part == "total" else oracle(kernel, e1, e2, src, q, trg, beta=beta, part=part,
                                                 grad=not stokes)
        assert np.linalg.norm(cen(got[0]) - cen(ref[0])) / np.linalg.norm(cen(tot[0])) < tol
        if not stokes:
            assert np.linalg.norm(got[1] - ref[1]) / np.linalg.norm(tot[1]) < tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 1.0), ("stokes", 0.0)])
def test_nufft_matches_direct(precision, kernel, beta):
    e1, e2 = (24.0, 0.0), (1.5, 1.0)
    stokes = kernel == "stokes"
    mc = kernel != "modhelm"
    rng = np.random.default_rng(12)
    src = workloads.points(rng, e1, e2, 2500, "gmm")
    q = workloads.strengths(rng, 1, 2500, stokes=stokes, neutral=mc)
    tol = TOL[precision]
    kw = dict(beta=beta, tol=tol, precision=precision, grad=not stokes)
    a = run_lib(kernel, e1, e2, src, q, None, part="far", path="nufft", **kw)
    b = run_lib(kernel, e1, e2, src, q, None, part="far", path="direct", **kw)
    tot = run_lib(kernel, e1, e2, src, q, None, part="total", path="direct", **kw)
    cen = (lambda x: x - x.mean(-1, keepdims=True)) if mc else (lambda x: x)
    assert np.linalg.norm(cen(a[0]) - cen(b[0])) / np.linalg.norm(cen(tot[0])) < tol
    if not stokes:
        assert np.linalg.norm(a[1] - b[1]) / np.linalg.norm(tot[1]) < tol


# ---------------------------------------------------------------------------
# Stokes pressure (pfmm_stokes_pressure: Laplace gradients of the force components)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
@pytest.mark.parametrize("lat", ["square", "skew", "rotated", "aspect16"])
def test_stokes_pressure(precision, tol, lat):
    import torch
    from oracle import api as oapi
    from paper_2111_01083_gb300 import StokesPressure
    e1, e2, src, f, trg = _case("stokes", lat, 900, nt=400, seed=5, nrhs=2)
    dev = torch.device("cuda", 0)
    op = StokesPressure(e1, e2, tol=tol, precision=precision, nrhs=2, ns_max=900, nt_max=900)
    S = torch.tensor(src, device=dev)
    F = torch.tensor(f, device=dev)
    T = torch.tensor(trg, device=dev)
    p = op(S, F, T)
    torch.cuda.synchronize()
    op.status()
    ref = oapi.stokes_pressure(e1, e2, src, f, trg)
    err = np.linalg.norm(p.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < tol, err
