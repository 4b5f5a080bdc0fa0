"""Pins of the singly periodic (P1) oracle, oracle/p1.py, against what the
mathematics fixes, independently of the factorization:

* Laplace: the closed-form kernel -(1/4pi) log(cosh(2 pi y/d) - cos(2 pi x/d))
  against the image sum over |m| <= M (zero net charge, Richardson in M);
* modified Helmholtz: the Poisson-summed spectral series against the image
  sum (absolutely convergent);
* Stokes: the image sum (zero net force, Richardson in M), and the flow
  equations -Lap u + grad p = 0, div u = 0 with p from the Laplace closed form;
* the paper's method (near images + the row-0 west/east factorization of the
  far images) against the closed forms and series to ~1e-12.
"""
import numpy as np
import pytest

from oracle import p1


def _strip_points(cell, n, rng, frac=0.98):
    u = rng.uniform(-0.5, 0.5, (2, n))
    return np.stack([u[0] * cell["d"], u[1] * cell["eta"] * frac])


def _cen(a):
    return a - a.mean(-1, keepdims=True)


STRIPS = [((1.0, 0.0), (0.0, 2.5)), ((2.0, 0.0), (0.7, 0.5)), ((1.2, 0.5), (-0.3, 1.9))]


@pytest.mark.parametrize("e1,e2", STRIPS)
def test_laplace_closed_form_is_the_image_sum(e1, e2):
    rng = np.random.default_rng(1)
    cell = p1.canonical_strip(e1, e2)
    src, trg = _strip_points(cell, 16, rng), _strip_points(cell, 6, rng)
    q = rng.standard_normal((1, 16))
    q -= q.mean()
    pc, gc = p1.laplace_closed(cell, trg, src, q)
    pb, gb = p1.brute_extrapolated("laplace", 0.0, cell, trg, src, q, 2000)
    assert np.abs(_cen(pb) - _cen(pc)).max() < 2e-7 * np.abs(_cen(pc)).max()
    assert np.abs(gb - gc).max() < 2e-7 * np.abs(gc).max()


@pytest.mark.parametrize("beta", [0.5, 2.0])
def test_modhelm_series_is_the_image_sum(beta):
    rng = np.random.default_rng(2)
    cell = p1.canonical_strip((1.5, 0.0), (0.0, 2.0))
    src, trg = _strip_points(cell, 16, rng), _strip_points(cell, 6, rng)
    q = rng.standard_normal((2, 16))
    ps = p1.modhelm_spectral(cell, beta, trg, src, q)
    M = int(np.ceil(60.0 / (beta * cell["d"]))) + 2  # K0(beta M d) < 1e-25
    pb, _ = p1.brute("modhelm", beta, cell, trg, src, q, M, want_grad=False)
    assert np.abs(ps - pb).max() < 1e-13 * np.abs(pb).max()


@pytest.mark.parametrize("e1,e2", STRIPS)
@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 1.0)])
def test_method_matches_closed_forms(e1, e2, kernel, beta):
    rng = np.random.default_rng(3)
    cell = p1.canonical_strip(e1, e2)
    src, trg = _strip_points(cell, 24, rng), _strip_points(cell, 9, rng)
    rot = cell["rot"]
    src_in, trg_in = rot.T @ src, rot.T @ trg
    q = rng.standard_normal((2, 24))
    if kernel == "laplace":
        q -= q.mean(-1, keepdims=True)
        ref, rg = p1.laplace_closed(cell, trg, src, q)
        got, gg = p1.evaluate(kernel, beta, e1, e2, src_in, q, trg_in)
        assert np.abs(_cen(got) - _cen(ref)).max() < 1e-12 * np.abs(_cen(ref)).max()
        rg_in = np.einsum("ij,rjn->rin", rot.T, rg)
        assert np.abs(gg - rg_in).max() < 1e-12 * np.abs(rg_in).max()
    else:
        ref = p1.modhelm_spectral(cell, beta, trg, src, q)
        got, _ = p1.evaluate(kernel, beta, e1, e2, src_in, q, trg_in, want_grad=False)
        assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_stokes_method_is_the_image_sum():
    rng = np.random.default_rng(4)
    cell = p1.canonical_strip((1.0, 0.0), (0.0, 1.5))
    src, trg = _strip_points(cell, 16, rng), _strip_points(cell, 6, rng)
    f = rng.standard_normal((1, 2, 16))
    f -= f.mean(-1, keepdims=True)
    vb, _ = p1.brute_extrapolated("stokes", 0.0, cell, trg, src, f, 2000)
    vm, _ = p1.evaluate("stokes", 0.0, (1.0, 0.0), (0.0, 1.5), src, f, trg)
    assert np.abs(_cen(vm) - _cen(vb)).max() < 3e-7 * np.abs(_cen(vb)).max()


def test_stokes_solves_the_flow_equations():
    """-Lap u + grad p = 0 and div u = 0 away from the sources (4th-order
    differences), p = -(d/dx phi[f_x] + d/dy phi[f_y]) from the Laplace closed
    form: pins the P1 Stokes velocity up to a constant."""
    rng = np.random.default_rng(5)
    e1, e2 = (1.0, 0.0), (0.0, 2.0)
    cell = p1.canonical_strip(e1, e2)
    src = _strip_points(cell, 10, rng, frac=0.6)
    f = rng.standard_normal((1, 2, 10))
    f -= f.mean(-1, keepdims=True)
    pts = []
    while len(pts) < 4:
        c = _strip_points(cell, 1, rng, frac=0.8)[:, 0]
        dd = np.min(np.hypot(c[0] - src[0][None, :] - np.array([[-1.0], [0.0], [1.0]]), c[1] - src[1]))
        if dd > 0.15:
            pts.append(c)
    h = 2e-3
    sh = np.arange(-2, 3) * h
    d1 = np.array([1, -8, 0, 8, -1]) / (12 * h)
    d2 = np.array([-1, 16, -30, 16, -1]) / (12 * h * h)
    P = []
    for c in pts:
        for s_ in sh:
            P.append(c + [s_, 0.0])
        for s_ in sh:
            P.append(c + [0.0, s_])
    P = np.array(P).T
    u, _ = p1.evaluate("stokes", 0.0, e1, e2, src, f, P)
    _, g = p1.laplace_closed(cell, P, src, f[0])  # charges f_x, f_y as two rhs
    p = -(g[0, 0] + g[1, 1])
    u = u[0].reshape(2, -1, 2, 5)
    p = p.reshape(-1, 2, 5)
    lap = u[:, :, 0, :] @ d2 + u[:, :, 1, :] @ d2
    gradp = np.stack([p[:, 0, :] @ d1, p[:, 1, :] @ d1])
    assert np.abs(lap - gradp).max() / np.abs(gradp).max() < 2e-6
    div = u[0, :, 0, :] @ d1 + u[1, :, 1, :] @ d1
    assert np.abs(div).max() / np.abs(u[:, :, 0, :] @ d1).max() < 1e-7


def test_planted_mistake_is_caught():
    """A method with all three image rows (the doubly periodic factor) in the
    singly periodic far part must disagree with the closed form."""
    from oracle import method
    rng = np.random.default_rng(6)
    cell = p1.canonical_strip((1.0, 0.0), (0.0, 1.0))
    src, trg = _strip_points(cell, 12, rng), _strip_points(cell, 5, rng)
    q = rng.standard_normal((1, 12))
    q -= q.mean()
    ref, _ = p1.laplace_closed(cell, trg, src, q)
    near, _ = p1.near_sum("laplace", 0.0, cell, trg, src, q)
    wrong, _ = method.far_field("laplace", 0.0, cell, trg, src, q, parts=("west", "east"), rows=(-1, 0, 1))
    assert np.abs(_cen(near + wrong) - _cen(ref)).max() > 1e-3 * np.abs(_cen(ref)).max()
