"""Singly periodic operator P1 (periodic along e1 only), FP64.  Test
infrastructure: only tests/ and bench.py's reference and CPU-baseline legs
use it; the library never does.

Geometry.  e1 is the period; e2 spans the strip: after the rotation that
takes e1 to (d, 0), points are wrapped along x by multiples of d into
[-d/2, d/2) and must lie in |y| < eta/2 with eta = |e1 x e2| / d (the
component of e2 across the strip).  The near images are m e1, |m| <= 1.

Definitions (each pinned independently in tests/test_oracle_pins.py):

* Laplace, zero net charge: sum_m log|z - m d| = log|sin(pi z/d)| + const
  for z = x + i y, so the P1 kernel is
      G1(x, y) = -(1/4 pi) log( cosh(2 pi y/d) - cos(2 pi x/d) )
  up to a constant that multiplies sum q = 0.  A self pair keeps the regular
  limit of G1 - G, -(1/4 pi) log(2 pi^2 / d^2).
* modified Helmholtz: by Poisson summation of the image sum of (1/2pi) K0,
      G1(x, y) = (1/(2d)) sum_k e^{i alpha_k x} e^{-chi_k |y|} / chi_k,
  alpha_k = 2 pi k / d, chi_k = sqrt(alpha_k^2 + beta^2) (|y| > 0).
* every kernel: the image sum over |m| <= M (symmetric truncation), with a
  Richardson step in M for the conditionally convergent Laplace / Stokes sums.
* the paper's method for the far images |m| >= 2: the west/east parts of the
  doubly periodic factorization restricted to the row n = 0 (Theorems
  west_thm, west_thm_lap, west_thm_s with the three-row factor replaced by
  its middle row), no south/north parts.
"""
import math

import numpy as np
from scipy import special

from . import greens, method


def canonical_strip(e1, e2):
    """Rotation and strip sizes: rot @ e1 = (d, 0); eta across the strip."""
    e1 = np.asarray(e1, np.float64)
    e2 = np.asarray(e2, np.float64)
    d = float(np.hypot(*e1))
    c, s = e1 / d
    rot = np.array([[c, s], [-s, c]])
    eta = abs(float(e1[0] * e2[1] - e1[1] * e2[0])) / d
    return {"d": d, "xi": 0.0, "eta": eta, "rot": rot, "m0": 1}


def wrap_strip(pts, cell):
    """Canonical coordinates: rotate, wrap x into [-d/2, d/2); y must be in the strip."""
    c = cell["rot"] @ np.asarray(pts, np.float64)
    d = cell["d"]
    u = c[0] / d
    u = u - np.floor(u + 0.5)
    out = np.stack([u * d, c[1]])
    if np.any(np.abs(out[1]) >= 0.5 * cell["eta"]):
        raise ValueError("points outside the strip |y| < eta/2")
    return out


def near_offsets(cell):
    d = cell["d"]
    return np.array([[-d, 0.0], [0.0, 0.0], [d, 0.0]])


def laplace_closed(cell, trg, src, q, want_grad=True):
    """Sum over all images with the closed-form P1 kernel (canonical frame)."""
    d = cell["d"]
    k = 2 * np.pi / d
    nrhs, nt = q.shape[0], trg.shape[1]
    pot = np.zeros((nrhs, nt))
    grad = np.zeros((nrhs, 2, nt)) if want_grad else None
    for l0 in range(0, nt, 256):
        t = trg[:, l0:l0 + 256]
        dx = t[0][:, None] - src[0][None, :]
        dy = t[1][:, None] - src[1][None, :]
        # reduce dx to [-d/2, d/2) (the kernel is d-periodic in x)
        dx = dx - d * np.floor(dx / d + 0.5)
        zero = (dx == 0.0) & (dy == 0.0)
        den = np.cosh(k * dy) - np.cos(k * dx)
        den = np.where(zero, 1.0, den)
        g = -np.log(den) / (4 * np.pi)
        g = np.where(zero, -math.log(2 * np.pi ** 2 / d ** 2) / (4 * np.pi), g)
        pot[:, l0:l0 + 256] = q @ g.T
        if want_grad:
            fx = np.where(zero, 0.0, -(k / (4 * np.pi)) * np.sin(k * dx) / den)
            fy = np.where(zero, 0.0, -(k / (4 * np.pi)) * np.sinh(k * dy) / den)
            grad[:, 0, l0:l0 + 256] = q @ fx.T
            grad[:, 1, l0:l0 + 256] = q @ fy.T
    return pot, grad


def modhelm_spectral(cell, beta, trg, src, q, kmax=None):
    """Potential by the spectral sum (pairs with |dy| > 0 only; tail < 1e-16)."""
    d = cell["d"]
    dx = trg[0][:, None] - src[0][None, :]
    dy = np.abs(trg[1][:, None] - src[1][None, :])
    dy_min = dy.min()
    if kmax is None:
        # e^{-|alpha_k| dy_min} < 1e-18 beyond kmax
        kmax = int(math.ceil(d * 42.0 / (2 * np.pi * max(dy_min, 1e-3)))) + 2
    pot = np.zeros((q.shape[0], trg.shape[1]))
    for kk in range(-kmax, kmax + 1):
        a = 2 * np.pi * kk / d
        chi = math.sqrt(a * a + beta * beta)
        g = np.cos(a * dx) * np.exp(-chi * dy) / (2 * d * chi)
        pot += q @ g.T
    return pot


def brute(kernel, beta, cell, trg, src, q, M, want_grad=True):
    """Image sum over |m| <= M, symmetric, in blocks of images."""
    d = cell["d"]
    offs = np.stack([np.arange(-M, M + 1) * d, np.zeros(2 * M + 1)], axis=1)
    return greens.image_sum(kernel, beta, trg, src, q, offs, want_grad)


def brute_extrapolated(kernel, beta, cell, trg, src, q, M, want_grad=True):
    """Richardson step in M for the conditionally convergent sums (zero net
    charge / force): the symmetric tail is c/M + O(1/M^2)."""
    a = brute(kernel, beta, cell, trg, src, q, M, want_grad)
    b = brute(kernel, beta, cell, trg, src, q, 2 * M, want_grad)
    pot = 2 * b[0] - a[0]
    grad = None if a[1] is None else 2 * b[1] - a[1]
    return pot, grad


def far_field(kernel, beta, cell, trg, src, q, eps=1e-14, want_grad=True):
    """The paper's method for the far images |m| >= 2 (row n = 0 of the
    west/east factorization)."""
    return method.far_field(kernel, beta, cell, trg, src, q, eps=eps, parts=("west", "east"),
                            want_grad=want_grad, rows=(0,))


def near_sum(kernel, beta, cell, trg, src, q, want_grad=True):
    return greens.image_sum(kernel, beta, trg, src, q, near_offsets(cell), want_grad)


def evaluate(kernel, beta, e1, e2, src, q, trg, part="total", how="method", eps=1e-14, want_grad=True):
    """Input-frame P1 field: part total/near/far; how: "method" (near images
    + the factorized far images) or "closed" (Laplace closed form / modified
    Helmholtz spectral sum, total only)."""
    cell = canonical_strip(e1, e2)
    rot = cell["rot"]
    s = wrap_strip(src, cell)
    t = wrap_strip(trg, cell)
    q = np.asarray(q, np.float64)
    stokes = kernel == "stokes"
    if stokes:
        q = np.einsum("ij,rjn->rin", rot, q)
        want_grad = False
    if how == "closed":
        if kernel == "laplace":
            pot, grad = laplace_closed(cell, t, s, q, want_grad)
        else:
            pot, grad = modhelm_spectral(cell, beta, t, s, q), None
    else:
        pot = 0.0
        grad = 0.0 if want_grad else None
        if part in ("total", "near"):
            p, g = near_sum(kernel, beta, cell, t, s, q, want_grad)
            pot = pot + p
            if want_grad:
                grad = grad + g
        if part in ("total", "far"):
            p, g = far_field(kernel, beta, cell, t, s, q, eps=eps, want_grad=want_grad)
            pot = pot + p
            if want_grad:
                grad = grad + g
    if stokes:
        return np.einsum("ij,rjn->rin", rot.T, pot), None
    return pot, (None if grad is None else np.einsum("ij,rjn->rin", rot.T, grad))
