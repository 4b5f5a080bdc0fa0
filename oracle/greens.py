"""Free-space Green's functions and plain image sums (oracle, FP64).

Sec. 1: G = (1/2pi) log(1/|t-s|) (Poisson) and G = (1/2pi) K0(beta |t-s|)
(modified Helmholtz); Sec. 5.2, Eq. stokeslet: the Stokeslet
G = -(1/4pi) (log|r| I - r r^T / |r|^2).  The sign convention is u = sum G q
(the sign of Eq. govpde is not used).

Modified Stokeslet (Eq. msgreen): G = (grad grad^T - Lap I) G_MB with
G_MB = -(1/(2 pi beta^2)) (K0(beta r) - log(1/r)).  For a radial h(r),
grad grad^T h = h'' rr + (h'/r)(I - rr) (rr = r r^T / r^2); with
h = (1/beta^2)(G_L - G_MH) (since 1/(k^2 (k^2 + beta^2)) =
(1/beta^2)(1/k^2 - 1/(k^2 + beta^2))) and Lap h = -G_MH away from 0 this
gives, with x = beta r,
    G = (1/2pi) [ A(x) I - B(x) rr ],  A = K0 + E,  B = K0 + 2 E,
    E(x) = K1(x)/x - 1/x^2.
E is summed from the ascending series of K1 for x < 2 (the two terms of the
difference cancel to O(log x) there):
    E = (I1(x)/x) ln(x/2) - (1/4) sum_k [psi(k+1) + psi(k+2)] t^k / (k! (k+1)!),
    I1(x)/x = (1/2) sum_k t^k / (k! (k+1)!),  t = x^2/4.

``image_sum`` is the plain double loop sum_{images o} sum_j G(t - s_j - o) q_j
with pairs at exactly zero distance skipped (self-exclusion), vectorised over
chunks of targets.  With o running over Lambda_near it is K^near q
(Eq. nearfarsplit).
"""
import numpy as np
from scipy import special

KERNELS = ("laplace", "modhelm", "stokes", "mstokes")
VECTOR = ("stokes", "mstokes")


def ms_E(x):
    """E(x) = K1(x)/x - 1/x^2 for x > 0 (FP64)."""
    x = np.asarray(x, np.float64)
    out = np.empty_like(x)
    small = x < 2.0
    xs = x[small]
    t = xs * xs / 4.0
    # ascending series: terms t^k / (k! (k+1)!) with psi(k+1) + psi(k+2)
    term = np.ones_like(t)
    i1x = np.zeros_like(t)
    ssum = np.zeros_like(t)
    psi1 = -np.euler_gamma  # psi(k+1)
    for k in range(0, 30):
        psi2 = psi1 + 1.0 / (k + 1)  # psi(k+2)
        i1x += 0.5 * term
        ssum += (psi1 + psi2) * term
        term = term * t / ((k + 1) * (k + 2))
        psi1 = psi2
    out[small] = i1x * np.log(xs / 2.0) - 0.25 * ssum
    xl = x[~small]
    out[~small] = special.k1(xl) / xl - 1.0 / (xl * xl)
    return out


def ms_AB(x):
    """A(x), B(x) of the modified Stokeslet (1/2pi)(A I - B rr)."""
    k0 = special.k0(x)
    e = ms_E(x)
    return k0 + e, k0 + 2.0 * e


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
    if kernel == "mstokes":
        A, B = ms_AB(beta * np.sqrt(r2s))
        c = 1.0 / (2 * np.pi)
        g11 = np.where(zero, 0.0, c * (A - B * dx * dx / r2s))
        g12 = np.where(zero, 0.0, -c * B * dx * dy / r2s)
        g22 = np.where(zero, 0.0, c * (A - B * dy * dy / r2s))
        return g11, g12, g22
    raise ValueError(kernel)


def image_sum(kernel, beta, trg, src, q, offsets, want_grad=True, chunk=256):
    """sum over offsets o and sources j of G(t_l - (s_j + o)) q_j.

    trg [2, nt], src [2, ns]; q [nrhs, ns] (scalar) or [nrhs, 2, ns] (stokes,
    mstokes).  Returns (pot, grad) for scalar kernels, (vel, None) for the
    vector kernels."""
    trg = np.asarray(trg, np.float64)
    src = np.asarray(src, np.float64)
    q = np.asarray(q, np.float64)
    nt = trg.shape[1]
    nrhs = q.shape[0]
    if kernel in VECTOR:
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
            if kernel in VECTOR:
                out[:, 0, l0:l1] += q[:, 0, :] @ a.T + q[:, 1, :] @ b.T
                out[:, 1, l0:l1] += q[:, 0, :] @ b.T + q[:, 1, :] @ c.T
            else:
                out[:, l0:l1] += q @ a.T
                if want_grad:
                    grad[:, 0, l0:l1] += q @ b.T
                    grad[:, 1, l0:l1] += q @ c.T
    return out, grad
