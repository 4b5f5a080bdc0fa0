"""Direct-sum definitions used by the NUFFT path (oracle, FP64).

Sec. 2.3, Eqs. nufft1/nufft2: type 1  f_k = sum_j c_j e^{i k x_j},
type 2  v_j = sum_k f_k e^{-i k x_j} (k = -M..M).
Sec. 2.4, Eq. baryweights: Legendre nodes t_i (roots of P_n), weights
sigma_i = 1/prod_{j != i}(t_i - t_j), second barycentric form.
Sec. 6, Eqs. fastanterp/fastinterp: gamma(t, n) = (sigma_n/(t - ybar_n)) /
sum_l sigma_l/(t - ybar_l) on the scaled nodes ybar in [-eta/2, eta/2].
"""
import numpy as np


def nufft1(x, c, M):
    k = np.arange(-M, M + 1)
    return np.exp(1j * k[:, None] * x[None, :]) @ c


def nufft2(x, f, M):
    k = np.arange(-M, M + 1)
    return np.exp(-1j * x[:, None] * k[None, :]) @ f


def legendre_nodes(n):
    return np.polynomial.legendre.leggauss(n)[0]


def bary_weights(t):
    n = t.size
    s = np.empty(n)
    for i in range(n):
        s[i] = 1.0 / np.prod(t[i] - np.delete(t, i))
    return s


def gamma_matrix(tq, nodes):
    """gamma(tq_j, n) for points tq (any) and interpolation nodes; rows sum to 1.
    A point equal to a node gets the unit vector."""
    sig = bary_weights(nodes)
    diff = tq[:, None] - nodes[None, :]
    hit = diff == 0.0
    diff = np.where(hit, 1.0, diff)
    r = sig[None, :] / diff
    g = r / r.sum(1, keepdims=True)
    rows = hit.any(1)
    g[rows] = hit[rows].astype(float)
    return g
