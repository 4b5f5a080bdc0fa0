"""The definition of the periodic and periodizing operators, by Ewald splitting.

Sec. 1 (Eq. psum and the K^(p) definition): u = sum_j K^(p)(t, s_j) q_j with
K^(p)(t, s) = sum over all lattice vectors l_mn of G(t, s + l_mn); Eq.
nearfarsplit: K^(p) = K^near + K^far; Definition "periodizing operators":
P2(l, j) = K^far(t_l, s_j).  The oracle therefore computes

    P2 q = K^(p) q - K^near q,

with K^near q the plain direct sum over Lambda_near (``greens.image_sum``)
and K^(p) q the conditionally/absolutely convergent lattice sum evaluated by
Ewald's splitting (Sec. 1 attributes the spectral approach to Ewald).  The
split comes from writing the Fourier symbol as an integral over t and cutting
it at t = tau:

  1/k^2          = int_0^tau e^{-k^2 t} dt + e^{-k^2 tau}/k^2
  1/(k^2+b^2)    = int_0^tau e^{-(k^2+b^2) t} dt + e^{-(k^2+b^2) tau}/(k^2+b^2)
  1/k^4          = int_0^tau t e^{-k^2 t} dt + e^{-k^2 tau}(tau/k^2 + 1/k^4)

The first pieces become rapidly decaying real-space image sums (heat kernel
(4 pi t)^-1 exp(-r^2/4t), Poisson summation), the second rapidly decaying
reciprocal-lattice sums.  Real-space pieces, with s = r^2/(4 tau):

  Laplace   (1/4pi) E1(s)
  modhelm   (1/4pi) int_1^inf u^-1 exp(-s u - beta^2 tau / u) du
  Stokes    G_ij = (1/4pi) e^-s r_i r_j / r^2 + [(1/8pi) E1(s) - (1/4pi) e^-s] delta_ij
            (G = (-Lap I + grad grad) B, B-hat = 1/k^4)

Reciprocal pieces (cell area |C|, k over the reciprocal lattice):

  Laplace   (1/|C|) sum_{k != 0} e^{ik.r} e^{-k^2 tau} / k^2
  modhelm   (1/|C|) sum_k        e^{ik.r} e^{-(k^2+b^2) tau} / (k^2+b^2)
  Stokes    (1/|C|) sum_{k != 0} e^{ik.r} (k^2 I - k k^T) e^{-k^2 tau} (tau/k^2 + 1/k^4)

Dropping k = 0 for Laplace/Stokes is the zero-mean gauge and requires net
charge / net force zero (Eq. chargeneutral).  A pair at zero distance (the
self pair) takes the regular limit of K^(p) - G there:
  Laplace (1/4pi)(ln 4tau - gamma), modhelm -(1/4pi) E1(beta^2 tau),
  Stokes (1/8pi)(ln 4tau - gamma - 2) I
(plus the other images' real-space terms and the reciprocal sum at r = 0).
"""
import math
import numpy as np
from scipy import special

from .greens import image_sum
from .lattice import near_offsets

EULER_GAMMA = 0.57721566490153286061
_CUT = 40.0  # exp(-40) ~ 4e-18


def _gl(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def _incbessel(c, b):
    """I0 = int_1^inf u^-1 exp(-c u - b/u) du and I1 = int_1^inf exp(-c u - b/u) du
    for arrays c > 0 and scalar b > 0, by composite Gauss-Legendre in s = ln u
    (for c >= b) or via the full-line closed forms 2 K0(2 sqrt(bc)),
    2 sqrt(b/c) K1(2 sqrt(bc)) minus the integral over (0, 1) (for c < b)."""
    c = np.asarray(c, np.float64)
    I0 = np.empty_like(c)
    I1 = np.empty_like(c)
    smax = max(2.0, math.log(60.0 / min(b, 1.0)) + 2.0)
    npan = int(math.ceil(smax / 0.5))
    gx, gw = _gl(16)
    nodes = (np.arange(npan)[:, None] * 0.5 + 0.25 * (gx[None, :] + 1.0)).ravel()
    wts = np.tile(0.25 * gw, npan)
    es, ems = np.exp(nodes), np.exp(-nodes)
    direct = c >= b
    if np.any(direct):
        cd = c[direct][:, None]
        f = np.exp(-cd * es[None, :] - b * ems[None, :])
        I0[direct] = f @ wts
        I1[direct] = (f * es[None, :]) @ wts
    comp = ~direct
    if np.any(comp):
        cc = c[comp]
        z = 2.0 * np.sqrt(b * cc)
        f = np.exp(-cc[:, None] * ems[None, :] - b * es[None, :])
        I0[comp] = 2.0 * special.k0(z) - f @ wts
        I1[comp] = 2.0 * np.sqrt(b / cc) * special.k1(z) - (f * ems[None, :]) @ wts
    return I0, I1


def default_tau(d, eta, n):
    area = d * eta
    return float(np.clip(0.12 * area / math.sqrt(max(n, 1)), 2e-4 * area, 0.05 * area)) * 1.0


def _real_space(kernel, beta, cell, trg, src, q, tau, want_grad, chunk=128):
    d, xi, eta = cell["d"], cell["xi"], cell["eta"]
    rcut = math.sqrt(4.0 * tau * _CUT)
    diam = max(math.hypot(d + xi, eta), math.hypot(d - xi, eta))
    R = rcut + diam
    nmax = int(R / eta) + 2
    lat = []
    for n in range(-nmax, nmax + 1):
        mmax = int((R + abs(n * xi)) / d) + 2
        for m in range(-mmax, mmax + 1):
            L = (m * d + n * xi, n * eta)
            if math.hypot(*L) <= R:
                lat.append(L)
    nt = trg.shape[1]
    nrhs = q.shape[0]
    stokes = kernel == "stokes"
    pot = np.zeros((nrhs, 2, nt)) if stokes else np.zeros((nrhs, nt))
    grad = np.zeros((nrhs, 2, nt)) if (want_grad and not stokes) else None
    b = beta * beta * tau
    for l0 in range(0, nt, chunk):
        l1 = min(nt, l0 + chunk)
        tx, ty = trg[0, l0:l1, None], trg[1, l0:l1, None]
        for L in lat:
            dx = tx - (src[0][None, :] + L[0])
            dy = ty - (src[1][None, :] + L[1])
            rho = dx * dx + dy * dy
            s = rho / (4.0 * tau)
            act = s < _CUT
            if not np.any(act):
                continue
            zero = act & (rho == 0.0)
            nz = act & (rho > 0.0)
            sn = s[nz]
            if kernel == "laplace":
                g = np.zeros_like(rho)
                g[nz] = special.exp1(sn) / (4 * np.pi)
                g[zero] = (math.log(4 * tau) - EULER_GAMMA) / (4 * np.pi)
                pot[:, l0:l1] += q @ g.T
                if want_grad:
                    f = np.zeros_like(rho)
                    f[nz] = -np.exp(-sn) / (2 * np.pi * rho[nz])
                    grad[:, 0, l0:l1] += q @ (f * dx).T
                    grad[:, 1, l0:l1] += q @ (f * dy).T
            elif kernel == "modhelm":
                I0, I1 = _incbessel(sn, b)
                g = np.zeros_like(rho)
                g[nz] = I0 / (4 * np.pi)
                g[zero] = -special.exp1(b) / (4 * np.pi)
                pot[:, l0:l1] += q @ g.T
                if want_grad:
                    f = np.zeros_like(rho)
                    f[nz] = -I1 / (8 * np.pi * tau)
                    grad[:, 0, l0:l1] += q @ (f * dx).T
                    grad[:, 1, l0:l1] += q @ (f * dy).T
            else:
                es = np.exp(-sn)
                diag = np.zeros_like(rho)
                diag[nz] = special.exp1(sn) / (8 * np.pi) - es / (4 * np.pi)
                diag[zero] = (math.log(4 * tau) - EULER_GAMMA - 2.0) / (8 * np.pi)
                h = np.zeros_like(rho)
                h[nz] = es / (4 * np.pi * rho[nz])
                g11 = diag + h * dx * dx
                g12 = h * dx * dy
                g22 = diag + h * dy * dy
                pot[:, 0, l0:l1] += q[:, 0] @ g11.T + q[:, 1] @ g12.T
                pot[:, 1, l0:l1] += q[:, 0] @ g12.T + q[:, 1] @ g22.T
    return pot, grad


def _reciprocal(kernel, beta, cell, trg, src, q, tau, want_grad):
    d, xi, eta = cell["d"], cell["xi"], cell["eta"]
    area = d * eta
    b1 = np.array([2 * np.pi / d, -2 * np.pi * xi / (d * eta)])
    b2 = np.array([0.0, 2 * np.pi / eta])
    kmax = math.sqrt(_CUT / tau)
    rmax = int(kmax / (2 * np.pi / eta)) + 2
    ks = []
    for r in range(-rmax, rmax + 1):
        # |p b1 + r b2| <= kmax  ->  p range from the x component
        pmax = int(kmax / (2 * np.pi / d)) + 2
        for p in range(-pmax, pmax + 1):
            k = p * b1 + r * b2
            k2 = k @ k
            if k2 * tau >= _CUT:
                continue
            if (p, r) == (0, 0) and kernel != "modhelm":
                continue
            ks.append(k)
    ks = np.array(ks)
    kx, ky = ks[:, 0], ks[:, 1]
    k2 = kx * kx + ky * ky
    Es = np.exp(-1j * (kx[:, None] * src[0][None, :] + ky[:, None] * src[1][None, :]))  # [nk, ns]
    Et = np.exp(1j * (kx[:, None] * trg[0][None, :] + ky[:, None] * trg[1][None, :]))  # [nk, nt]
    if kernel == "stokes":
        w = np.exp(-k2 * tau) * (tau / k2 + 1.0 / (k2 * k2)) / area
        S1 = q[:, 0] @ Es.T  # [nrhs, nk]
        S2 = q[:, 1] @ Es.T
        a1 = w * ((k2 - kx * kx) * S1 - kx * ky * S2)
        a2 = w * (-kx * ky * S1 + (k2 - ky * ky) * S2)
        vel = np.stack([(a1 @ Et).real, (a2 @ Et).real], axis=1)
        return vel, None
    if kernel == "laplace":
        w = np.exp(-k2 * tau) / k2 / area
    else:
        kb = k2 + beta * beta
        w = np.exp(-kb * tau) / kb / area
    S = (q @ Es.T) * w  # [nrhs, nk]
    pot = (S @ Et).real
    grad = None
    if want_grad:
        grad = np.stack([((S * (1j * kx)) @ Et).real, ((S * (1j * ky)) @ Et).real], axis=1)
    return pot, grad


def periodic_sum(kernel, beta, cell, trg, src, q, want_grad=True, tau=None):
    """K^(p) q at the targets (canonical frame, wrapped points).  Zero-distance
    pairs take the regular limit.  Laplace/Stokes: zero-mean gauge."""
    trg = np.asarray(trg, np.float64)
    src = np.asarray(src, np.float64)
    q = np.asarray(q, np.float64)
    if tau is None:
        tau = default_tau(cell["d"], cell["eta"], max(trg.shape[1], src.shape[1]))
    p1, g1 = _real_space(kernel, beta, cell, trg, src, q, tau, want_grad)
    p2, g2 = _reciprocal(kernel, beta, cell, trg, src, q, tau, want_grad)
    pot = p1 + p2
    grad = (g1 + g2) if (g1 is not None and g2 is not None) else None
    return pot, grad


def near_sum(kernel, beta, cell, trg, src, q, want_grad=True):
    """K^near q: direct sum over Lambda_near with self pairs skipped."""
    offs = near_offsets(cell["d"], cell["xi"], cell["eta"], cell["m0"])
    return image_sum(kernel, beta, trg, src, q, offs, want_grad)


def far_sum(kernel, beta, cell, trg, src, q, want_grad=True, tau=None):
    """P2 q = K^(p) q - K^near q (the periodizing potential)."""
    p, g = periodic_sum(kernel, beta, cell, trg, src, q, want_grad, tau)
    pn, gn = near_sum(kernel, beta, cell, trg, src, q, want_grad)
    return p - pn, (g - gn) if g is not None else None
