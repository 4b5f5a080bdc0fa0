"""Pins of the FP64 oracle against things other than itself.

* Laplace: Ewald sum vs the Jacobi-theta closed form (oracle.theta).
* modified Helmholtz: Ewald vs absolutely convergent brute-force image sums,
  and each far-field part S/N/W/E of the plain method vs its own brute-force
  image sum (Eq. ksplitting2).
* Stokes: the periodic velocity solves -Lap u + grad p = 0 and div u = 0 away
  from the sources, with p built from the (theta-pinned) Laplace gradient
  (pressurelet p = (1/2pi) f.r/|r|^2 = -f.grad G_Laplace, Sec. 5.2).
* Rotated west/east direction (App. A): each rotated part vs its brute-force
  image sum (modified Helmholtz), Laplace and Stokes vs Ewald, planted
  mistakes (column phase dropped, rotation transposed) caught.
* Ewald: independence of the splitting parameter tau.
* Method invariants: periodicity across cell edges (the paper's own error
  metric, Sec. 7), symmetry of P2, gradient = derivative of potential,
  invariance under a change of lattice basis, truncation error below the
  precision (Eq. esbound1).
* Special-function values against textbook values.
"""
import math

import numpy as np
import pytest
from scipy import special

from oracle import api, brute, ewald, greens, lattice, method, nufft, theta
import workloads

R = np.random.default_rng(12345)


def _cell_pts(e1, e2, n, seed):
    rng = np.random.default_rng(seed)
    return workloads.points(rng, e1, e2, n)


def _q(n, nrhs=2, seed=0, stokes=False):
    return workloads.strengths(np.random.default_rng(seed), nrhs, n, stokes=stokes)


def test_special_function_values():
    # Abramowitz & Stegun tables: K0(1), K1(1), E1(1).
    assert abs(special.k0(1.0) - 0.4210244382407083) < 1e-15
    assert abs(special.k1(1.0) - 0.6019072301972346) < 1e-15
    assert abs(special.exp1(1.0) - 0.2193839343955203) < 1e-15


@pytest.mark.parametrize("e1,e2", [((1, 0), (0, 1)), ((1, 0), (0.3, 0.8)), ((4, 0), (0, 1)),
                                   ((2, 0.5), (-0.4, 1.7))])
def test_laplace_ewald_matches_theta(e1, e2):
    src = _cell_pts(e1, e2, 50, 1)
    trg = _cell_pts(e1, e2, 30, 2)
    q = _q(50)
    cell, s, t = lattice.to_canonical(e1, e2, src, trg)
    pe, ge = ewald.periodic_sum("laplace", 0.0, cell, t, s, q)
    pt, gt = theta.laplace_periodic(cell, t, s, q)
    assert api.rel_err(pe, pt, modconst=True) < 1e-12
    assert api.rel_err(ge, gt) < 1e-11


def test_laplace_ewald_theta_self_targets():
    e1, e2 = (1.0, 0.0), (0.2, 1.1)
    src = _cell_pts(e1, e2, 40, 3)
    q = _q(40)
    cell, s, t = lattice.to_canonical(e1, e2, src, src)
    pe, ge = ewald.periodic_sum("laplace", 0.0, cell, t, s, q)
    pt, gt = theta.laplace_periodic(cell, t, s, q)
    assert api.rel_err(pe, pt, modconst=True) < 1e-12
    assert api.rel_err(ge, gt) < 1e-11


def test_single_charge_pair_rectangular_closed_form():
    # +1 at the origin, -1 elsewhere: theta form vs Ewald at a few targets.
    e1, e2 = (1.5, 0.0), (0.0, 1.0)
    src = np.array([[0.0, 0.3], [0.0, -0.2]])
    q = np.array([[1.0, -1.0]])
    trg = np.array([[0.1, -0.6, 0.7], [0.25, 0.4, -0.45]])
    cell, s, t = lattice.to_canonical(e1, e2, src, trg)
    pe, _ = ewald.periodic_sum("laplace", 0.0, cell, t, s, q)
    pt, _ = theta.laplace_periodic(cell, t, s, q)
    assert api.rel_err(pe, pt, modconst=True) < 1e-13


@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 2.0), ("modhelm", 0.3), ("stokes", 0.0)])
def test_ewald_tau_independent(kernel, beta):
    e1, e2 = (2.0, 0.0), (0.5, 1.0)
    src = _cell_pts(e1, e2, 30, 4)
    trg = _cell_pts(e1, e2, 20, 5)
    q = _q(30, stokes=kernel == "stokes")
    cell, s, t = lattice.to_canonical(e1, e2, src, trg)
    a, ga = ewald.periodic_sum(kernel, beta, cell, t, s, q, tau=0.01)
    b, gb = ewald.periodic_sum(kernel, beta, cell, t, s, q, tau=0.07)
    mc = kernel != "modhelm"
    assert api.rel_err(a, b, modconst=mc) < 1e-12
    if ga is not None:
        assert api.rel_err(ga, gb) < 1e-12


@pytest.mark.parametrize("beta", [1.0, 4.0])
def test_modhelm_ewald_matches_brute(beta):
    e1, e2 = (1.0, 0.0), (0.3, 0.8)
    src = _cell_pts(e1, e2, 25, 6)
    trg = _cell_pts(e1, e2, 15, 7)
    q = np.random.default_rng(1).standard_normal((2, 25))  # beta > 0: no neutrality needed
    cell, s, t = lattice.to_canonical(e1, e2, src, trg)
    pe, ge = ewald.far_sum("modhelm", beta, cell, t, s, q)
    pb, gb = brute.modhelm_part(cell, beta, t, s, q, "far")
    assert api.rel_err(pe, pb) < 1e-11
    assert api.rel_err(ge, gb) < 1e-11


@pytest.mark.parametrize("e1,e2", [((1, 0), (0, 1)), ((1, 0), (0.3, 0.8)), ((6, 0), (0, 1))])
@pytest.mark.parametrize("part", brute.PARTS)
def test_method_parts_match_brute_modhelm(e1, e2, part):
    beta = 1.5
    src = _cell_pts(e1, e2, 30, 8)
    trg = _cell_pts(e1, e2, 20, 9)
    q = np.random.default_rng(2).standard_normal((2, 30))  # no neutrality needed for beta > 0
    cell, s, t = lattice.to_canonical(e1, e2, src, trg)
    pb, gb = brute.modhelm_part(cell, beta, t, s, q, part)
    pm, gm = method.far_field("modhelm", beta, cell, t, s, q, parts=(part,))
    scale = np.linalg.norm(pb) + 1e-300
    assert np.linalg.norm(pm - pb) / scale < 1e-11
    assert np.linalg.norm(gm - gb) / (np.linalg.norm(gb) + 1e-300) < 1e-11


@pytest.mark.parametrize("e1,e2", [((1, 0), (0, 1)), ((1, 0), (0.3, 0.8)), ((5, 0), (0, 1)),
                                   ((1.2, 0.4), (-0.5, 0.9))])
def test_method_matches_ewald_laplace(e1, e2):
    src = _cell_pts(e1, e2, 40, 10)
    trg = _cell_pts(e1, e2, 25, 11)
    q = _q(40)
    pe, ge = api.evaluate("laplace", 0.0, e1, e2, src, q, trg, part="far", how="ewald")
    pm, gm = api.evaluate("laplace", 0.0, e1, e2, src, q, trg, part="far", how="plain")
    assert api.rel_err(pm, pe, modconst=True) < 1e-12
    assert api.rel_err(gm, ge) < 1e-12


@pytest.mark.parametrize("e1,e2", [((1, 0), (0, 1)), ((1, 0), (0.3, 0.8)), ((5, 0), (0, 1)),
                                   ((1.2, 0.4), (-0.5, 0.9))])
def test_method_matches_ewald_stokes(e1, e2):
    src = _cell_pts(e1, e2, 40, 12)
    trg = _cell_pts(e1, e2, 25, 13)
    f = _q(40, stokes=True)
    ve, _ = api.evaluate("stokes", 0.0, e1, e2, src, f, trg, part="far", how="ewald")
    vm, _ = api.evaluate("stokes", 0.0, e1, e2, src, f, trg, part="far", how="plain")
    assert api.rel_err(vm, ve, modconst=True) < 1e-12


HEX = ((1.0, 0.0), (0.5, math.sqrt(3) / 2))
ROT_CELLS = [HEX, ((1, 0), (0.42, 0.5)), ((2, 0), (0.9, 1.1)), ((1, 0), (0.3, 0.8))]


@pytest.mark.parametrize("e1,e2", ROT_CELLS)
@pytest.mark.parametrize("part", ["west", "east"])
def test_rotated_we_parts_match_brute_modhelm(e1, e2, part):
    """App. A (Eq. k0west2): west/east plane waves decaying along e2-perp with
    m0 = 1, each part against its own absolutely convergent image sum over
    m <= -2 (m >= 2), |n| <= 1."""
    beta = 1.5
    src = _cell_pts(e1, e2, 30, 40)
    trg = _cell_pts(e1, e2, 20, 41)
    q = np.random.default_rng(4).standard_normal((2, 30))
    cell, s, t = lattice.to_canonical(e1, e2, src, trg, we="rotated")
    assert cell["we_rot"] and cell["m0"] == 1
    pb, gb = brute.modhelm_part(cell, beta, t, s, q, part)
    pm, gm = method.far_field("modhelm", beta, cell, t, s, q, parts=(part,))
    assert np.linalg.norm(pm - pb) / np.linalg.norm(pb) < 1e-11
    assert np.linalg.norm(gm - gb) / np.linalg.norm(gb) < 1e-11


@pytest.mark.parametrize("e1,e2", ROT_CELLS)
def test_rotated_method_matches_ewald(e1, e2):
    """Laplace (potential up to a constant, gradient) and Stokes with the
    rotated west/east direction against the Ewald definition of P2 for the
    3 x 3 near block."""
    src = _cell_pts(e1, e2, 40, 42)
    trg = _cell_pts(e1, e2, 25, 43)
    q = _q(40, seed=5)
    f = _q(40, seed=6, stokes=True)
    pe, ge = api.evaluate("laplace", 0.0, e1, e2, src, q, trg, part="far", how="ewald", we="rotated")
    pm, gm = api.evaluate("laplace", 0.0, e1, e2, src, q, trg, part="far", how="plain", we="rotated")
    assert api.rel_err(pm, pe, modconst=True) < 1e-12
    assert api.rel_err(gm, ge) < 1e-12
    ve, _ = api.evaluate("stokes", 0.0, e1, e2, src, f, trg, part="far", how="ewald", we="rotated")
    vm, _ = api.evaluate("stokes", 0.0, e1, e2, src, f, trg, part="far", how="plain", we="rotated")
    assert api.rel_err(vm, ve, modconst=True) < 1e-12


def test_rotated_direction_rule():
    d, xi = 1.0, 0.5  # hexagonal cell: the axis direction needs m0 = 2
    assert lattice.choose_we(d, xi, "axis") == (False, 2)
    assert lattice.choose_we(d, xi, "auto") == (True, 1)
    assert lattice.choose_we(d, 0.3, "auto") == (False, 1)
    assert lattice.choose_we(d, 0.0, "rotated") == (True, 1)
    fr = method.we_frame(dict(d=1.0, xi=0.5, eta=math.sqrt(3) / 2, m0=1, we_rot=True))
    # e2 maps to (0, |e2|), e1 to (d eta/|e2|, d xi/|e2|)
    assert abs(fr["c"] * 0.5 - fr["s"] * math.sqrt(3) / 2) < 1e-15
    assert abs(fr["dx"] - math.sqrt(3) / 2) < 1e-15 and abs(fr["dy"] - 0.5) < 1e-15


@pytest.mark.parametrize("mistake", ["no_column_phase", "transposed_rotation"])
def test_rotated_planted_mistakes_are_caught(mistake, monkeypatch):
    """A west part that drops the y~ shift of the image columns, or rotates
    the wrong way, must disagree with the brute image sum."""
    e1, e2 = HEX
    src = _cell_pts(e1, e2, 20, 44)
    trg = _cell_pts(e1, e2, 12, 45)
    q = np.random.default_rng(7).standard_normal((1, 20))
    cell, s, t = lattice.to_canonical(e1, e2, src, trg, we="rotated")
    pb, _ = brute.modhelm_part(cell, 1.5, t, s, q, "west")
    good = method.we_frame

    def bad(c):
        fr = dict(good(c))
        if mistake == "no_column_phase":
            fr["dy"] = 0.0
        else:
            fr["s"] = -fr["s"]
        return fr

    monkeypatch.setattr(method, "we_frame", bad)
    pm, _ = method.far_field("modhelm", 1.5, cell, t, s, q, parts=("west",))
    assert np.linalg.norm(pm - pb) / np.linalg.norm(pb) > 1e-3


def _away_points(e1, e2, src, n, dmin, seed):
    rng = np.random.default_rng(seed)
    cell = lattice.canonicalize(e1, e2)
    out = []
    offs = []
    for a in (-1, 0, 1):
        for b in (-1, 0, 1):
            offs.append(a * np.array(e1, float) + b * np.array(e2, float))
    while len(out) < n:
        p = workloads.points(rng, e1, e2, 1)[:, 0]
        dist = min(np.min(np.hypot(*(p[:, None] - src - o[:, None]))) for o in offs)
        if dist > dmin:
            out.append(p)
    return np.array(out).T


def _fd_stencil(h):
    # 4th-order central differences: first and second derivative weights on -2..2
    d1 = np.array([1, -8, 0, 8, -1]) / (12 * h)
    d2 = np.array([-1, 16, -30, 16, -1]) / (12 * h * h)
    return d1, d2


@pytest.mark.parametrize("how", ["ewald", "plain"])
def test_stokes_solves_pde(how):
    """-Lap u + grad p = 0 and div u = 0 away from sources, p from Laplace theta."""
    e1, e2 = (1.0, 0.0), (0.3, 0.8)
    n = 12
    src = _cell_pts(e1, e2, n, 14)
    f = _q(n, nrhs=1, stokes=True)
    pts = _away_points(e1, e2, src, 4, 0.12, 15)
    h = 2e-3
    d1, d2 = _fd_stencil(h)
    sh = np.arange(-2, 3) * h
    # stencil points: along x and along y
    P = []
    for p in pts.T:
        for s_ in sh:
            P.append(p + [s_, 0.0])
        for s_ in sh:
            P.append(p + [0.0, s_])
    P = np.array(P).T
    # evaluate at points without wrapping (stay in the cell: dmin >> 2h)
    cell = lattice.canonicalize(e1, e2)
    cell["m0"] = lattice.choose_m0(cell["d"], cell["xi"])
    rot = cell["rot"]
    s = lattice.wrap(rot @ src, cell["d"], cell["xi"], cell["eta"])
    t = rot @ P
    fc = np.einsum("ij,rjn->rin", rot, f)
    if how == "ewald":
        u, _ = ewald.periodic_sum("stokes", 0.0, cell, t, s, fc)
    else:
        u0, _ = ewald.near_sum("stokes", 0.0, cell, t, s, fc)
        u1, _ = method.far_field("stokes", 0.0, cell, t, s, fc)
        u = u0 + u1
    # pressure from the theta-pinned Laplace gradient, charges f_x and f_y
    _, gx = theta.laplace_periodic(cell, t, s, fc[:, 0])
    _, gy = theta.laplace_periodic(cell, t, s, fc[:, 1])
    p = -(gx[:, 0] + gy[:, 1])  # [1, npts]
    u = u[0].reshape(2, -1, 2, 5)  # comp, point, dir, stencil
    p = p[0].reshape(-1, 2, 5)
    lap = u[:, :, 0, :] @ d2 + u[:, :, 1, :] @ d2  # [comp, point]
    gradp = np.stack([p[:, 0, :] @ d1, p[:, 1, :] @ d1])  # [comp, point]
    div = u[0, :, 0, :] @ d1 + u[1, :, 1, :] @ d1
    scale = np.abs(gradp).max()
    assert np.abs(lap - gradp).max() / scale < 2e-6
    gscale = np.abs(u[:, :, 0, :] @ d1).max()
    assert np.abs(div).max() / gscale < 1e-7  # 4th-order FD truncation ~h^4


def _boundary_targets(e1, e2, n):
    """(left, right, bottom, top) canonical-frame targets with right = left + e1
    and top = bottom + e2, both on the closed cell boundary (not wrapped)."""
    cell = lattice.canonicalize(e1, e2)
    d, xi, eta = cell["d"], cell["xi"], cell["eta"]
    u = (np.arange(n) + 0.5) / n - 0.5
    A = np.array([[d, xi], [0, eta]])
    left = A @ np.stack([-0.5 * np.ones(n), u])
    bottom = A @ np.stack([u, -0.5 * np.ones(n)])
    return cell, left, left + A[:, :1], bottom, bottom + A[:, 1:]




def test_stokes_pressure_closes_the_pde():
    """oracle.api.stokes_pressure (Laplace gradients of the force components)
    is the pressure of the periodic Stokes flow: with it, -Lap u + grad p = 0
    away from the sources (4th-order differences), and it is periodic."""
    e1, e2 = (1.0, 0.0), (0.3, 0.8)
    n = 12
    src = _cell_pts(e1, e2, n, 14)
    f = _q(n, nrhs=1, stokes=True)
    pts = _away_points(e1, e2, src, 4, 0.12, 15)
    h = 2e-3
    d1, d2 = _fd_stencil(h)
    sh = np.arange(-2, 3) * h
    P = []
    for p in pts.T:
        for s_ in sh:
            P.append(p + [s_, 0.0])
        for s_ in sh:
            P.append(p + [0.0, s_])
    P = np.array(P).T
    u, _ = api.evaluate("stokes", 0.0, e1, e2, src, f, P, want_grad=False)
    p = api.stokes_pressure(e1, e2, src, f, P)
    u = u[0].reshape(2, -1, 2, 5)
    p = p[0].reshape(-1, 2, 5)
    lap = u[:, :, 0, :] @ d2 + u[:, :, 1, :] @ d2
    gradp = np.stack([p[:, 0, :] @ d1, p[:, 1, :] @ d1])
    assert np.abs(lap - gradp).max() / np.abs(gradp).max() < 2e-6
    # periodic: p(t + e1) = p(t), p(t + e2) = p(t)
    t = pts
    p0 = api.stokes_pressure(e1, e2, src, f, t)
    for e in (e1, e2):
        pe = api.stokes_pressure(e1, e2, src, f, t + np.array(e, float)[:, None])
        assert np.abs(pe - p0).max() < 1e-10 * np.abs(p0).max()


@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 1.0), ("stokes", 0.0)])
@pytest.mark.parametrize("e1,e2", [((1, 0), (0, 1)), ((1, 0), (0.3, 0.8)), ((8, 0), (0, 1))])
def test_method_periodicity(kernel, beta, e1, e2):
    """The paper's accuracy check (Sec. 7): relative l2 of the difference of the
    full field (near + far) between opposite cell sides."""
    n = 40
    src = _cell_pts(e1, e2, n, 16)
    q = _q(n, stokes=kernel == "stokes")
    cell, left, right, bottom, top = _boundary_targets(e1, e2, 50)
    cell["m0"] = lattice.choose_m0(cell["d"], cell["xi"])
    rot = cell["rot"]
    s = lattice.wrap(rot @ src, cell["d"], cell["xi"], cell["eta"])
    if kernel == "stokes":
        q = np.einsum("ij,rjn->rin", rot, q)
    T = np.concatenate([left, right, bottom, top], axis=1)
    u0, g0 = ewald.near_sum(kernel, beta, cell, T, s, q)
    u1, g1 = method.far_field(kernel, beta, cell, T, s, q)
    u = u0 + u1
    k = 50
    diff = np.concatenate([u[..., k:2 * k] - u[..., :k], u[..., 3 * k:] - u[..., 2 * k:3 * k]], -1)
    ref = u - u.mean(-1, keepdims=True)
    assert np.linalg.norm(diff) / np.linalg.norm(ref) < 1e-12
    if g0 is not None:
        g = g0 + g1
        gd = np.concatenate([g[..., k:2 * k] - g[..., :k], g[..., 3 * k:] - g[..., 2 * k:3 * k]], -1)
        assert np.linalg.norm(gd) / np.linalg.norm(g) < 1e-12


@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 2.0), ("stokes", 0.0)])
def test_far_operator_symmetric(kernel, beta):
    e1, e2 = (3.0, 0.0), (0.4, 1.0)
    n = 35
    src = _cell_pts(e1, e2, n, 17)
    st = kernel == "stokes"
    a = _q(n, nrhs=1, seed=1, stokes=st)
    b = _q(n, nrhs=1, seed=2, stokes=st)
    pa, _ = api.evaluate(kernel, beta, e1, e2, src, a, src, part="far", how="plain")
    pb, _ = api.evaluate(kernel, beta, e1, e2, src, b, src, part="far", how="plain")
    lhs = np.sum(a * pb)
    rhs = np.sum(pa * b)
    assert abs(lhs - rhs) / (abs(lhs) + abs(rhs)) < 1e-12


@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 0.7)])
def test_gradient_is_derivative_of_potential(kernel, beta):
    e1, e2 = (2.0, 0.0), (0.0, 1.0)
    src = _cell_pts(e1, e2, 30, 18)
    q = _q(30, nrhs=1)
    pts = _away_points(e1, e2, src, 3, 0.1, 19)
    h = 1e-3
    d1, _ = _fd_stencil(h)
    sh = np.arange(-2, 3) * h
    P = np.array([p + [s_, 0] for p in pts.T for s_ in sh] + [p + [0, s_] for p in pts.T for s_ in sh]).T
    pot, grad = api.evaluate(kernel, beta, e1, e2, src, q, P, part="far", how="plain")
    k = 5 * pts.shape[1]
    fx = pot[0, :k].reshape(-1, 5) @ d1
    fy = pot[0, k:].reshape(-1, 5) @ d1
    gx = grad[0, 0, :k].reshape(-1, 5)[:, 2]
    gy = grad[0, 1, k:].reshape(-1, 5)[:, 2]
    scale = np.abs(np.concatenate([gx, gy])).max()
    assert np.abs(fx - gx).max() / scale < 1e-7
    assert np.abs(fy - gy).max() / scale < 1e-7


@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 1.0), ("stokes", 0.0)])
def test_basis_invariance(kernel, beta):
    e1, e2 = (1.0, 0.0), (0.25, 0.9)
    f1, f2 = (1.25, 0.9), (-1.0, 0.0)  # same lattice: e1 + e2, -e1
    src = _cell_pts(e1, e2, 30, 20)
    trg = _cell_pts(e1, e2, 20, 21)
    q = _q(30, stokes=kernel == "stokes")
    a, ga = api.evaluate(kernel, beta, e1, e2, src, q, trg, part="total", how="plain")
    b, gb = api.evaluate(kernel, beta, f1, f2, src, q, trg, part="total", how="plain")
    assert api.rel_err(a, b, modconst=(kernel != "modhelm")) < 1e-12
    if ga is not None:
        assert api.rel_err(ga, gb) < 1e-12


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_truncation_error_within_precision(eps):
    """Theorem south_thm: with M from Eq. mpk0s each entry of P^south is
    approximated to O(eps); check |u_M - u| <= eps * sum|q| at every target."""
    e1, e2 = (10.0, 0.0), (0.0, 1.0)
    cell = lattice.canonicalize(e1, e2)
    cell["m0"] = 1
    src = _cell_pts(e1, e2, 30, 22)
    trg = _cell_pts(e1, e2, 20, 23)
    q = np.random.default_rng(3).standard_normal((1, 30))
    rot = cell["rot"]
    s = lattice.wrap(rot @ src, cell["d"], cell["xi"], cell["eta"])
    t = lattice.wrap(rot @ trg, cell["d"], cell["xi"], cell["eta"])
    ex, _ = brute.modhelm_part(cell, 0.5, t, s, q, "south")
    ap, _ = method.far_field("modhelm", 0.5, cell, t, s, q, eps=eps, parts=("south",))
    err = np.abs(ap - ex).max()
    assert err <= eps * np.abs(q).sum()
    assert err > 0  # the truncation is real


def test_canonicalization_rules():
    c = lattice.canonicalize((0.0, 2.0), (1.0, 0.0))
    assert abs(c["d"] - 2.0) < 1e-15 and abs(c["eta"] - 1.0) < 1e-15 and abs(c["xi"]) < 1e-15
    c = lattice.canonicalize((1.0, 0.0), (0.3, 0.8))
    assert (c["d"], c["xi"], c["eta"]) == (1.0, 0.3, 0.8)
    assert lattice.choose_m0(1.0, 0.3) == 1 and lattice.choose_m0(16.0, 0.0) == 1
    assert lattice.choose_m0(1.0, 0.4) == 2 and lattice.choose_m0(1.0, 0.3, margin_frac=1.0) == 2
    c = lattice.canonicalize((1.0, 0.0), (5.3, 0.8))  # reduces xi to 0.3
    assert abs(c["xi"] - 0.3) < 1e-12 and abs(c["eta"] - 0.8) < 1e-12
    w = lattice.wrap(np.array([[0.5, -0.5, 1.7], [0.0, 0.0, 0.2]]), 1.0, 0.0, 1.0)
    assert np.allclose(w[0], [-0.5, -0.5, -0.3])


def test_nufft_definitions():
    n = 16
    x = 2 * np.pi * np.arange(n) / n
    c = np.random.default_rng(4).standard_normal(n)
    f = nufft.nufft1(x, c, 7)
    ref = np.fft.ifft(c) * n  # sum_j c_j e^{+2 pi i k j/n}
    k = np.arange(-7, 8)
    assert np.allclose(f, ref[k % n], atol=1e-12)
    # type 2 is the adjoint of type 1: <N c, g> = <c, N* g>
    xr = np.random.default_rng(5).uniform(-np.pi, np.pi, 23)
    cr = np.random.default_rng(6).standard_normal(23) + 1j * np.random.default_rng(7).standard_normal(23)
    g = np.random.default_rng(8).standard_normal(15) + 0j
    lhs = np.vdot(g, nufft.nufft1(xr, cr, 7))
    rhs = np.vdot(nufft.nufft2(xr, g, 7), cr)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_barycentric_reproduces_polynomials():
    nodes = nufft.legendre_nodes(8)
    assert np.allclose(np.polynomial.legendre.legval(nodes, [0] * 8 + [1]), 0, atol=1e-14)
    t = np.linspace(-1, 1, 41)
    g = nufft.gamma_matrix(t, nodes)
    for deg in range(8):
        assert np.allclose(g @ nodes ** deg, t ** deg, atol=1e-12)
    assert np.allclose(g.sum(1), 1.0)
