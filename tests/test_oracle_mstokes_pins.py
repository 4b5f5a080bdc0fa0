"""Pins of the modified Stokes oracle (Eq. msgreen, Theorems south_thm_ms,
west_thm_ms) against things other than itself:

* the free-space kernel (1/2pi)(A I - B rr) against 4th-order differences of
  the paper's G_MB = -(1/(2 pi beta^2))(K0(beta r) - log(1/r)) under
  (grad grad^T - Lap I), and its small/large-argument limits (Stokeslet,
  (1/beta^2) grad grad^T G_L);
* each far part against exact image sums in the paper's order (image rows):
  G^MS = H + (1/beta^2) grad grad^T G_L with H = G_MH I - (1/beta^2) grad
  grad^T G_MH exponentially decaying (plain truncated sums), and the row sums
  of grad grad^T G_L in closed form, the Hessian of
  -(1/4pi) log(cosh(2 pi y/d) - cos(2 pi x/d));
* planted mistakes (the Laplace family's m = 0 term kept as its lambda -> 0
  limit, the west/east beta-family block transposed) are caught.
"""
import math

import numpy as np
import pytest
from scipy import special

from oracle import greens, lattice, method
import workloads


def _H(beta, dx, dy):
    """(G_MH I - (1/beta^2) grad grad^T G_MH)(r): (1/2pi)[(K0 + K1/x) I - (K0 + 2 K1/x) rr]."""
    r = np.hypot(dx, dy)
    x = beta * r
    k0, k1x = special.k0(x), special.k1(x) / x
    a, b = k0 + k1x, k0 + 2 * k1x
    c = 1 / (2 * np.pi)
    return c * (a - b * dx * dx / r ** 2), -c * b * dx * dy / r ** 2, c * (a - b * dy * dy / r ** 2)


def _hess_row(d, dx, dy):
    """Row sum over m of grad grad^T G_L(r - m d e_x), G_L = -(1/2pi) log r.
    sum_m log(z - m d) = log sin(pi z/d) + const (z = x + i y), so G_L's row
    sum is Re f with f = -(1/2pi) log sin(pi z/d) and its Hessian is
    (Re f'', -Im f'', -Re f''), f'' = (pi/(2 d^2)) / sin^2(pi z/d).  1/sin^2 w
    = -4 q/(1 - q)^2 with q = e^{2 i w sgn(Im w)} (|q| < 1: no overflow)."""
    w = np.pi * (dx + 1j * dy) / d
    sg = np.where(dy >= 0, 1.0, -1.0)
    q = np.exp(2j * w * sg)
    F = (np.pi / (2 * d * d)) * (-4 * q / (1 - q) ** 2)
    return F.real, -F.imag, -F.real


def _hess_L(dx, dy):
    r2 = dx * dx + dy * dy
    c = 1 / (2 * np.pi * r2)
    return c * (2 * dx * dx / r2 - 1), c * 2 * dx * dy / r2, c * (2 * dy * dy / r2 - 1)


def _apply(t, s, f, fn, offs):
    out = np.zeros((f.shape[0], 2, t.shape[1]))
    for o in offs:
        dx = t[0][:, None] - s[0][None, :] - o[0]
        dy = t[1][:, None] - s[1][None, :] - o[1]
        g11, g12, g22 = fn(dx, dy)
        out[:, 0] += f[:, 0] @ g11.T + f[:, 1] @ g12.T
        out[:, 1] += f[:, 0] @ g12.T + f[:, 1] @ g22.T
    return out


def exact_part(beta, cell, t, s, f, part):
    """The far part as an exact image-row sum (see module docstring)."""
    d, xi, eta, m0 = cell["d"], cell["xi"], cell["eta"], cell["m0"]
    reach = 40.0 / beta + 2 * (d + eta)  # K0, K1 < 1e-17 beyond
    N = int(reach / eta) + 2
    M = int((reach + N * abs(xi)) / d) + 2
    if part == "south":
        rows = range(-N, -1)
    elif part == "north":
        rows = range(2, N + 1)
    else:
        rows = (-1, 0, 1)
    hoffs, loffs, rowsh = [], [], []
    for n in rows:
        rowsh.append((n * xi, n * eta))
        for m in range(-M, M + 1):
            if part == "we" and abs(m) <= m0:
                loffs.append((m * d + n * xi, n * eta))  # near columns: removed from the row sums
                continue
            hoffs.append((m * d + n * xi, n * eta))
    out = _apply(t, s, f, lambda a, b: _H(beta, a, b), hoffs)
    out += _apply(t, s, f, lambda a, b: _hess_row(d, a, b), rowsh) / beta ** 2
    if loffs:
        out -= _apply(t, s, f, _hess_L, loffs) / beta ** 2
    return out


CELLS = [((1.0, 0.0), (0.0, 1.0), "auto"), ((1.0, 0.0), (0.3, 0.8), "auto"),
         ((1.0, 0.0), (0.5, math.sqrt(3) / 2), "rotated"), ((2.0, 0.0), (0.4, 1.0), "auto"),
         ((1.0, 0.0), (0.5, math.sqrt(3) / 2), "axis")]


@pytest.mark.parametrize("e1,e2,we", CELLS)
@pytest.mark.parametrize("beta", [0.7, 3.0])
def test_parts_match_exact_row_sums(e1, e2, we, beta):
    rng = np.random.default_rng(61)
    src = workloads.points(rng, e1, e2, 12)
    trg = workloads.points(rng, e1, e2, 7)
    f = rng.standard_normal((2, 2, 12))
    cell, s, t = lattice.to_canonical(e1, e2, src, trg, we=we)
    for part, parts in (("south", ("south",)), ("north", ("north",)), ("we", ("west", "east"))):
        ref = exact_part(beta, cell, t, s, f, part)
        got, _ = method.far_field("mstokes", beta, cell, t, s, f, parts=parts)
        assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max(), part


def test_kernel_is_the_paper_definition():
    """(grad grad^T - Lap I) G_MB by 4th-order central differences."""
    beta = 1.3
    h = 1e-3
    d1 = np.array([1, -8, 0, 8, -1]) / (12 * h)
    d2 = np.array([-1, 16, -30, 16, -1]) / (12 * h * h)
    sh = np.arange(-2, 3) * h

    def gmb(x, y):
        r = np.hypot(x, y)
        return -(special.k0(beta * r) + np.log(r)) / (2 * np.pi * beta ** 2)

    for (x, y) in ((0.4, 0.3), (-1.1, 0.7), (0.05, -0.2), (2.5, 3.0)):
        gxx = gmb(x + sh, y) @ d2
        gyy = gmb(x, y + sh) @ d2
        gxy = np.array([gmb(x + a, y + sh) @ d1 for a in sh]) @ d1
        ref = np.array([[-gyy, gxy], [gxy, -gxx]])
        g11, g12, g22 = greens._pair_terms("mstokes", beta, np.array([x]), np.array([y]), False)
        got = np.array([[g11[0], g12[0]], [g12[0], g22[0]]])
        assert np.abs(got - ref).max() < 1e-7 * np.abs(ref).max(), (x, y)


def test_kernel_limits():
    """Small beta r: the Stokeslet -(1/4pi)(log r I - rr) up to a constant
    times I; large beta r: (1/beta^2) grad grad^T G_L."""
    dx, dy = np.array([3e-4, -2e-4]), np.array([1e-4, 2.5e-4])
    beta = 1.0
    m = greens._pair_terms("mstokes", beta, dx, dy, False)
    st = greens._pair_terms("stokes", 0.0, dx, dy, False)
    # A -> -(1/2) log(x/2) - gamma/2 - 1/4 and B -> -1/2 as x -> 0, so the
    # difference tends to c I with c = (1/4pi)(log(2/beta) - gamma - 1/2)
    c = (math.log(2 / beta) - np.euler_gamma - 0.5) / (4 * np.pi)
    for a, b, diag in zip(m, st, (True, False, True)):
        assert np.abs(a - b - (c if diag else 0.0)).max() < 1e-6
    dx, dy = np.array([40.0, -30.0]), np.array([25.0, 33.0])
    beta = 2.0
    m = greens._pair_terms("mstokes", beta, dx, dy, False)
    hl = _hess_L(dx, dy)
    for a, b in zip(m, hl):
        assert np.abs(a - b / beta ** 2).max() < 1e-14


@pytest.mark.parametrize("mistake", ["laplace_m0_limit", "we_block_transposed"])
def test_planted_mistakes_are_caught(mistake, monkeypatch):
    e1, e2 = (1.0, 0.0), (0.3, 0.8)
    beta = 1.5
    rng = np.random.default_rng(62)
    src = workloads.points(rng, e1, e2, 10)
    trg = workloads.points(rng, e1, e2, 6)
    f = rng.standard_normal((1, 2, 10))
    cell, s, t = lattice.to_canonical(e1, e2, src, trg)
    if mistake == "laplace_m0_limit":
        part, parts = "south", ("south",)
        good = method._mstokes_sn

        def bad(beta_, cell_, trg_, src_, f_, eps_, part_):
            # add the lambda -> 0 limit of the Laplace family as an m = 0 term:
            # diag(-1, 1) / (eta * 2 beta^2 d) (row sums taken after the
            # lattice sum instead of per row)
            out = good(beta_, cell_, trg_, src_, f_, eps_, part_)
            k = 1.0 / (cell_["eta"] * 2 * beta_ ** 2 * cell_["d"])
            out[:, 0] += -k * f_[:, 0].sum(-1)[:, None]
            out[:, 1] += k * f_[:, 1].sum(-1)[:, None]
            return out

        monkeypatch.setattr(method, "_mstokes_sn", bad)
    else:
        part, parts = "we", ("west", "east")
        good = method._mstokes_we

        def bad(beta_, cell_, trg_, src_, f_, eps_, part_):
            # swap the force components on input: a transposed 2 x 2 block
            return good(beta_, cell_, trg_, src_, f_[:, ::-1], eps_, part_)

        monkeypatch.setattr(method, "_mstokes_we", bad)
    ref = exact_part(beta, cell, t, s, f, part)
    got, _ = method.far_field("mstokes", beta, cell, t, s, f, parts=parts)
    assert np.abs(got - ref).max() > 1e-3 * np.abs(ref).max()


def test_total_independent_of_split_and_basis():
    """near + far is one lattice sum: the same for either west/east direction
    (3 x 3 or 5 x 3 near block), for another basis of the lattice, and
    periodic in the targets."""
    from oracle import api
    rng = np.random.default_rng(63)
    e1, e2 = (1.0, 0.0), (0.5, math.sqrt(3) / 2)
    src = workloads.points(rng, e1, e2, 25)
    trg = workloads.points(rng, e1, e2, 9)
    f = rng.standard_normal((2, 2, 25))
    a, _ = api.evaluate("mstokes", 1.7, e1, e2, src, f, trg, how="plain", we="rotated")
    b, _ = api.evaluate("mstokes", 1.7, e1, e2, src, f, trg, how="plain", we="axis")
    c, _ = api.evaluate("mstokes", 1.7, (e1[0] + e2[0], e1[1] + e2[1]), (-e1[0], -e1[1]), src, f, trg,
                        how="plain")
    d, _ = api.evaluate("mstokes", 1.7, e1, e2, src, f, trg + np.array(e2)[:, None], how="plain")
    for x in (b, c, d):
        assert api.rel_err(x, a) < 1e-12


def test_solves_the_pde():
    """(beta^2 - Lap) u + grad p = 0 and div u = 0 away from the sources
    (4th-order differences), zero net force, p = -(d/dx phi[f_x] + d/dy phi[f_y])
    from the periodic Laplace potential (the modified Stokeslet shares the
    Stokes pressurelet): pins the whole periodic sum, constant included (the
    beta^2 u term leaves no free constant)."""
    from oracle import api
    rng = np.random.default_rng(81)
    e1, e2 = (1.0, 0.0), (0.3, 0.8)
    beta = 1.7
    src = workloads.points(rng, e1, e2, 12)
    f = rng.standard_normal((1, 2, 12))
    f -= f.mean(-1, keepdims=True)
    E = np.array([e1, e2]).T
    pts = []
    while len(pts) < 4:
        c = workloads.points(rng, e1, e2, 1)[:, 0]
        dmin = min(np.hypot(*(c[:, None] - src - (E @ np.array([a, b]))[:, None])).min()
                   for a in (-1, 0, 1) for b in (-1, 0, 1))
        if dmin > 0.12:
            pts.append(c)
    h = 2e-3
    sh = np.arange(-2, 3) * h
    d1 = np.array([1, -8, 0, 8, -1]) / (12 * h)
    d2 = np.array([-1, 16, -30, 16, -1]) / (12 * h * h)
    P = np.array([c + [s_, 0] for c in pts for s_ in sh] + [c + [0, s_] for c in pts for s_ in sh]).T
    # reorder to [point][direction][stencil]
    n = len(pts)
    P = P.reshape(2, 2, n, 5).transpose(0, 2, 1, 3).reshape(2, -1)
    u, _ = api.evaluate("mstokes", beta, e1, e2, src, f, P, how="plain")
    p = api.stokes_pressure(e1, e2, src, f, P, how="plain")
    u = u[0].reshape(2, n, 2, 5)
    p = p[0].reshape(n, 2, 5)
    lap = u[:, :, 0, :] @ d2 + u[:, :, 1, :] @ d2
    gp = np.stack([p[:, 0, :] @ d1, p[:, 1, :] @ d1])
    res = beta ** 2 * u[:, :, 0, 2] - lap + gp
    assert np.abs(res).max() < 1e-7 * np.abs(gp).max()
    div = u[0, :, 0, :] @ d1 + u[1, :, 1, :] @ d1
    assert np.abs(div).max() < 1e-6 * np.abs(u[:, :, 0, :] @ d1).max()
