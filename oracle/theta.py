"""Closed form of the doubly periodic Laplace Green's function (oracle pin).

For the lattice {m d + n (xi + i eta)} the function
    G(z) = -(1/2pi) ln|theta1(pi z/d | tau_c)| + y^2/(2 d eta),
    tau_c = (xi + i eta)/d,  theta1(w) = 2 sum_{n>=0} (-1)^n q^{(n+1/2)^2} sin((2n+1) w),
    q = exp(i pi tau_c),
is periodic in both lattice directions (theta1(w+pi) = -theta1(w),
theta1(w + pi tau_c) = -q^-1 e^{-2iw} theta1(w)), has the singularity
(1/2pi) log(1/|z|) at z = 0 (the Green's function of Sec. 1) and
-Laplacian G = delta - 1/|C|.  With zero net charge (Eq. chargeneutral) the
background term drops out, so sum_j G(t - s_j) q_j equals the periodic
potential K^(p) q up to a constant.  This is derived here from the standard
theta-function identities; it shares nothing with the Ewald oracle and pins
it for Laplace.
"""
import math
import numpy as np


def _theta1_and_deriv(w, qn, n):
    """theta1(w) and theta1'(w) for complex array w."""
    k = 2 * np.arange(n) + 1
    coef = 2.0 * ((-1.0) ** np.arange(n)) * qn  # [n]
    kw = k[None, :] * w[..., None]
    th = (coef * np.sin(kw)).sum(-1)
    dth = (coef * k * np.cos(kw)).sum(-1)
    return th, dth


def laplace_periodic(cell, trg, src, q, want_grad=True):
    d, xi, eta = cell["d"], cell["xi"], cell["eta"]
    tau_c = (xi + 1j * eta) / d
    nterm = int(math.sqrt(45.0 * d / (math.pi * eta))) + 6
    ns = np.arange(nterm)
    qn = np.exp(1j * math.pi * tau_c * (ns + 0.5) ** 2)
    trg = np.asarray(trg, np.float64)
    src = np.asarray(src, np.float64)
    q = np.asarray(q, np.float64)
    nt = trg.shape[1]
    nrhs = q.shape[0]
    pot = np.zeros((nrhs, nt))
    grad = np.zeros((nrhs, 2, nt))
    _, dth0 = _theta1_and_deriv(np.zeros(1, complex), qn, nterm)
    self_val = -(math.log(abs(dth0[0])) + math.log(math.pi / d)) / (2 * math.pi)
    for l in range(nt):
        zx = trg[0, l] - src[0]
        zy = trg[1, l] - src[1]
        zero = (zx == 0.0) & (zy == 0.0)
        w = math.pi * (zx + 1j * zy) / d
        th, dth = _theta1_and_deriv(np.where(zero, 0.1, w), qn, nterm)
        g = -np.log(np.abs(th)) / (2 * math.pi) + zy * zy / (2 * d * eta)
        g = np.where(zero, self_val, g)
        ratio = (math.pi / d) * dth / th
        gx = np.where(zero, 0.0, -ratio.real / (2 * math.pi))
        gy = np.where(zero, 0.0, ratio.imag / (2 * math.pi) + zy / (d * eta))
        pot[:, l] = q @ g
        if want_grad:
            grad[:, 0, l] = q @ gx
            grad[:, 1, l] = q @ gy
    return pot, (grad if want_grad else None)
