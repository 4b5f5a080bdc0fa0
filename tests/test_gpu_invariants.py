"""GPU checks against properties the exact periodic field has at any size
(no oracle evaluation needed, so they run at sizes beyond the oracle's reach):

* periodicity, the paper's own accuracy measure (Sec. 7): the potential
  (velocity) and gradient just inside one edge of the cell equal those just
  inside the opposite edge (the same points across the periodic boundary);
* the Stokes velocity is divergence free: central differences of the FP64
  velocity on a small stencil;
* the mixed path does not depend on the input order of the points (the
  spatial sort is internal): permuted inputs give permuted outputs.
"""
import numpy as np
import pytest

import workloads
from gpu_util import run_lib

pytestmark = pytest.mark.gpu


def _edge_pairs(desc, n, which, rng, eps=1e-13):
    """n pairs of points just inside opposite edges of the canonical cell
    (fractional coordinate -1/2 + eps and 1/2 - eps along e_which, the same
    random position along the other vector), returned in the input frame.
    The two points of a pair are 2 eps |e_which| apart across the periodic
    boundary, but the method treats them very differently (opposite sides of
    the near block, opposite ends of the plane-wave expansions), so the field
    agrees there only if the decomposition is consistent (Sec. 7)."""
    d, xi, eta = desc["d"], desc["xi"], desc["eta"]
    rot = np.array(desc["rot"]).reshape(2, 2)
    c1, c2 = np.array([d, 0.0]), np.array([xi, eta])
    ew, eo = (c1, c2) if which == 1 else (c2, c1)
    s = rng.uniform(-0.45, 0.45, n)
    a = (-0.5 + eps) * ew[:, None] + s[None, :] * eo[:, None]
    b = (0.5 - eps) * ew[:, None] + s[None, :] * eo[:, None]
    return rot.T @ a, rot.T @ b


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 2.0), ("stokes", 0.0)])
@pytest.mark.parametrize("e1,e2", [((1.0, 0.0), (0.3, 0.8)), ((16.0, 0.0), (0.0, 1.0)),
                                   ((1.0, 0.0), (0.5, 0.8660254037844386))])
def test_periodicity(precision, tol, kernel, beta, e1, e2):
    from paper_2111_01083_gb300 import PeriodicOp
    rng = np.random.default_rng(31)
    n = 3000 if precision == "mixed" else 1200
    src = workloads.points(rng, e1, e2, n, "gmm")
    stokes = kernel == "stokes"
    q = workloads.strengths(rng, 2, n, stokes=stokes, neutral=kernel != "modhelm")
    desc = PeriodicOp(kernel, e1, e2, beta=beta, tol=tol, precision=precision, ns_max=8, nt_max=8).describe()
    inner = workloads.points(rng, e1, e2, 500)
    for which in (1, 2):
        a, b = _edge_pairs(desc, 250, which, rng)
        trg = np.concatenate([a, b, inner], axis=1)
        pot, grad, _ = run_lib(kernel, e1, e2, src, q, trg, beta=beta, tol=tol, precision=precision,
                               grad=not stokes)
        # both halves come from one evaluation (one gauge constant), so they agree
        # to the method's accuracy (plus 2 eps |grad|, negligible), measured
        # against the field's spread over the cell (edge and interior points)
        pa, pb = pot[..., :250], pot[..., 250:500]
        ref = pot - pot.mean(-1, keepdims=True) if kernel != "modhelm" else pot
        err = np.linalg.norm(pa - pb) / np.linalg.norm(ref)
        assert err < 2 * tol, (which, err)
        if grad is not None:
            gerr = np.linalg.norm(grad[..., :250] - grad[..., 250:500]) / np.linalg.norm(grad)
            assert gerr < 2 * tol, (which, gerr)


def _div_points(e1, e2, src, rng, dist=0.05, m=48):
    """Points at least `dist` from every source image."""
    cand = workloads.points(rng, e1, e2, 4000)
    E = np.array([e1, e2]).T
    dmin = np.full(cand.shape[1], np.inf)
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            sh = E @ np.array([a, b])
            d = np.hypot(cand[0][:, None] - src[0][None, :] - sh[0], cand[1][:, None] - src[1][None, :] - sh[1])
            dmin = np.minimum(dmin, d.min(axis=1))
    return cand[:, dmin > dist][:, :m]


def test_stokes_velocity_divergence_free():
    """div u = 0 away from the sources: 4th-order central differences
    (h = 1e-3, 5 points per axis) of the FP64 velocity at points at least 0.05
    from every source image, against the largest velocity derivative."""
    rng = np.random.default_rng(32)
    e1, e2 = (1.0, 0.0), (0.3, 0.8)
    n = 400
    src = workloads.points(rng, e1, e2, n)
    f = workloads.strengths(rng, 1, n, stokes=True)
    c = _div_points(e1, e2, src, rng)
    nc = c.shape[1]
    assert nc >= 16
    h = 1e-3
    w = np.array([1.0, -8.0, 0.0, 8.0, -1.0]) / (12 * h)
    sh = np.arange(-2, 3) * h
    pts = [c + np.array([[s_], [0.0]]) for s_ in sh] + [c + np.array([[0.0], [s_]]) for s_ in sh]
    u, _, _ = run_lib("stokes", e1, e2, src, f, np.concatenate(pts, axis=1), tol=1e-12, precision="fp64",
                      grad=False)
    u = u[0].reshape(2, 2, 5, nc)  # component, direction, stencil, point
    dxx = np.einsum("s,sp->p", w, u[0, 0])
    dyy = np.einsum("s,sp->p", w, u[1, 1])
    scale = max(np.abs(dxx).max(), np.abs(dyy).max())
    assert np.abs(dxx + dyy).max() / scale < 1e-6


@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 5.0), ("stokes", 0.0)])
def test_mixed_path_independent_of_input_order(kernel, beta):
    rng = np.random.default_rng(33)
    e1, e2 = (8.0, 0.0), (0.5, 1.0)
    n = 4000
    stokes = kernel == "stokes"
    src = workloads.points(rng, e1, e2, n, "gmm")
    q = workloads.strengths(rng, 1, n, stokes=stokes, neutral=kernel != "modhelm")
    perm = rng.permutation(n)
    a = run_lib(kernel, e1, e2, src, q, None, beta=beta, tol=1e-6, precision="mixed", grad=not stokes)
    b = run_lib(kernel, e1, e2, src[:, perm], q[..., perm], None, beta=beta, tol=1e-6, precision="mixed",
                grad=not stokes)
    inv = np.argsort(perm)
    for x, y in ((a[0], b[0][..., inv]), (a[1], None if b[1] is None else b[1][..., inv])):
        if x is None:
            continue
        mc = kernel != "modhelm" and x is a[0]
        if mc:
            x = x - x.mean(-1, keepdims=True)
            y = y - y.mean(-1, keepdims=True)
        assert np.linalg.norm(x - y) / np.linalg.norm(x) < 1e-6
