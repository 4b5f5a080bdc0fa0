"""Free-space Green's functions and plain image sums (oracle, FP64).

Sec. 1: G = (1/2pi) log(1/|t-s|) (Poisson) and G = (1/2pi) K0(beta |t-s|)
(modified Helmholtz); Sec. 5.2, Eq. stokeslet: the Stokeslet
G = -(1/4pi) (log|r| I - r r^T / |r|^2).  The sign convention is u = sum G q
(the sign of Eq. govpde is not used).

``image_sum`` is the plain double loop sum_{images o} sum_j G(t - s_j - o) q_j
with pairs at exactly zero distance skipped (self-exclusion), vectorised over
chunks of targets.  With o running over Lambda_near it is K^near q
(Eq. nearfarsplit).
"""
import numpy as np
from scipy import special

KERNELS = ("laplace", "modhelm", "stokes")


def _pair_terms(kernel, beta, dx, dy, want_grad):
    """Return per-pair kernel values for displacement (dx, dy) (t - s).
    scalar: (g, gx, gy); stokes: (g11, g12, g22).  Zero-distance pairs give 0."""
    r2 = dx * dx + dy * dy
    zero = r2 == 0.0
    r2s = np.where(zero, 1.0, r2)
    if kernel == "laplace":
        g = -np.log(r2s) / (4 * np.pi)
        g = np.where(zero, 0.0, g)
        if not want_grad:
            return g, None, None
        f = np.where(zero, 0.0, -1.0 / (2 * np.pi * r2s))
        return g, f * dx, f * dy
    if kernel == "modhelm":
        r = np.sqrt(r2s)
        g = np.where(zero, 0.0, special.k0(beta * r) / (2 * np.pi))
        if not want_grad:
            return g, None, None
        f = np.where(zero, 0.0, -beta * special.k1(beta * r) / (2 * np.pi * r))
        return g, f * dx, f * dy
    if kernel == "stokes":
        lg = -np.log(r2s) / (8 * np.pi)  # -(1/4pi) log r
        inv = 1.0 / (4 * np.pi * r2s)
        g11 = np.where(zero, 0.0, lg + dx * dx * inv)
        g12 = np.where(zero, 0.0, dx * dy * inv)
        g22 = np.where(zero, 0.0, lg + dy * dy * inv)
        return g11, g12, g22
    raise ValueError(kernel)


def image_sum(kernel, beta, trg, src, q, offsets, want_grad=True, chunk=256):
    """sum over offsets o and sources j of G(t_l - (s_j + o)) q_j.

    trg [2, nt], src [2, ns]; q [nrhs, ns] (scalar) or [nrhs, 2, ns] (stokes).
    Returns (pot, grad) for scalar kernels, (vel, None) for stokes."""
    trg = np.asarray(trg, np.float64)
    src = np.asarray(src, np.float64)
    q = np.asarray(q, np.float64)
    nt = trg.shape[1]
    nrhs = q.shape[0]
    if kernel == "stokes":
        out = np.zeros((nrhs, 2, nt))
        grad = None
    else:
        out = np.zeros((nrhs, nt))
        grad = np.zeros((nrhs, 2, nt)) if want_grad else None
    for l0 in range(0, nt, chunk):
        l1 = min(nt, l0 + chunk)
        tx = trg[0, l0:l1, None]
        ty = trg[1, l0:l1, None]
        for o in offsets:
            dx = tx - (src[0][None, :] + o[0])
            dy = ty - (src[1][None, :] + o[1])
            a, b, c = _pair_terms(kernel, beta, dx, dy, want_grad)
            if kernel == "stokes":
                out[:, 0, l0:l1] += q[:, 0, :] @ a.T + q[:, 1, :] @ b.T
                out[:, 1, l0:l1] += q[:, 0, :] @ b.T + q[:, 1, :] @ c.T
            else:
                out[:, l0:l1] += q @ a.T
                if want_grad:
                    grad[:, 0, l0:l1] += q @ b.T
                    grad[:, 1, l0:l1] += q @ c.T
    return out, grad
