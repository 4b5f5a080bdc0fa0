"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers (numpy default_rng(seed)); it holds
none of the method's arithmetic and is shared by the tests, the benchmark and
the oracle checks.  The paper measures on uniform random sources in the unit
cell (Sec. 7); no dataset is involved.

Point recipes are in FRACTIONAL lattice coordinates u in [-1/2, 1/2)^2,
mapped to the plane by x = u1 e1 + u2 e2:
  "uniform": u ~ U[-1/2, 1/2)^2
  "gmm"    : 8-component Gaussian mixture, centres uniform, sigma 0.02 per
             fractional axis, wrapped back into [-1/2, 1/2)
Strengths: N(0, 1) per entry, then the mean over sources removed per rhs (and
per component for Stokes forces), i.e. zero net charge / net force.
"""
import math
import numpy as np


def points(rng, e1, e2, n, dist="uniform", ncomp=8, sigma=0.02):
    if dist == "uniform":
        u = rng.uniform(-0.5, 0.5, size=(2, n))
    elif dist == "gmm":
        cen = rng.uniform(-0.5, 0.5, size=(2, ncomp))
        lab = rng.integers(0, ncomp, size=n)
        u = cen[:, lab] + sigma * rng.standard_normal((2, n))
        u = u - np.floor(u + 0.5)
    else:
        raise ValueError(dist)
    e1 = np.asarray(e1, np.float64)
    e2 = np.asarray(e2, np.float64)
    return np.ascontiguousarray(e1[:, None] * u[0][None, :] + e2[:, None] * u[1][None, :])


def strengths(rng, nrhs, n, stokes=False, neutral=True):
    q = rng.standard_normal((nrhs, 2, n) if stokes else (nrhs, n))
    if neutral:
        q = q - q.mean(-1, keepdims=True)
    return np.ascontiguousarray(q)


def single_cell(kernel, e1, e2, ns, nt=None, seed=0, dist="uniform", nrhs=1, beta=0.0):
    """One cell. nt=None means targets = sources (same array)."""
    rng = np.random.default_rng(seed)
    src = points(rng, e1, e2, ns, dist)
    # forces for the Stokes kernels; zero mean except for modified Stokes
    # (which needs no net-force condition)
    q = strengths(rng, nrhs, ns, stokes=kernel in ("stokes", "mstokes"), neutral=kernel != "mstokes")
    trg = src if nt is None else points(rng, e1, e2, nt, "uniform")
    return dict(kernel=kernel, beta=beta, e1=tuple(e1), e2=tuple(e2), src=src, q=q, trg=trg,
                self_targets=nt is None)


# Named configurations (full size).  Each is a dict of generator arguments.
CONFIGS = {
    "laplace_square_n1000": dict(kernel="laplace", e1=(1.0, 0.0), e2=(0.0, 1.0), ns=1000,
                                 seed=0, dist="uniform", tol=1e-10, precision="fp64"),
    "laplace_aspect16_gmm_n1e5": dict(kernel="laplace", e1=(16.0, 0.0), e2=(0.0, 1.0), ns=100000,
                                      seed=1, dist="gmm", tol=1e-6, precision="mixed",
                                      path="nufft", nufft_w=8, n_gl=8),
    "stokes_skew_n2e5": dict(kernel="stokes", e1=(1.0, 0.0), e2=(0.3, 0.8), ns=200000, nt=200000,
                             seed=2, dist="uniform", tol=1e-6, precision="mixed"),
    # hexagonal lattice (|xi| = d/2): the axis west/east direction needs a 5 x 3
    # near block, the rotated one (e2-perp) a 3 x 3 block
    "stokes_hex_n2e5": dict(kernel="stokes", e1=(1.0, 0.0), e2=(0.5, 0.8660254037844386), ns=200000,
                            nt=200000, seed=7, dist="uniform", tol=1e-6, precision="mixed"),
    # modified Stokeslet (Brinkman) with beta = 1 on the skew cell: 1e5 sources
    # with N(0,1) forces (no zero-net-force condition), 1e5 separate targets
    "mstokes_skew_beta1_n1e5": dict(kernel="mstokes", beta=1.0, e1=(1.0, 0.0), e2=(0.3, 0.8), ns=100000,
                                    nt=100000, seed=8, dist="uniform", tol=1e-6, precision="mixed"),
    "laplace_adjoint_4x1_n5e4": dict(kernel="laplace", e1=(4.0, 0.0), e2=(0.0, 1.0), ns=50000,
                                     seed=4, dist="uniform", tol=1e-6, precision="mixed"),
    # singly periodic (P1): period e1, 1e5 uniform sources in the strip segment
    # [-1/2, 1/2) x [-2, 2), targets = sources (the paper's P1 rectangle cases)
    "laplace_p1_strip4_n1e5": dict(kernel="laplace", e1=(1.0, 0.0), e2=(0.0, 4.0), ns=100000,
                                   seed=6, dist="uniform", tol=1e-6, precision="mixed", singly=True),
    # one long cell of the batched workload's shape (aspect 64, beta = 1, 8 rhs):
    # the far-field kernels (NUFFT spread/interpolation, direct formation and
    # evaluation) at the size where the batch's per-cell phases are largest
    "modhelm_aspect64_beta1_n5e4_r8": dict(kernel="modhelm", beta=1.0, e1=(64.0, 0.0), e2=(0.0, 1.0), ns=50000,
                                           seed=9, dist="uniform", tol=1e-6, precision="mixed", nrhs=8),
}


def make(name, scale=1.0, seed=None):
    """Generate a named configuration, optionally with point counts scaled."""
    c = dict(CONFIGS[name])
    ns = max(1, int(round(c["ns"] * scale)))
    nt = c.get("nt")
    if nt is not None:
        nt = max(1, int(round(nt * scale)))
    w = single_cell(c["kernel"], c["e1"], c["e2"], ns, nt, seed if seed is not None else c["seed"],
                    c.get("dist", "uniform"), nrhs=c.get("nrhs", 1), beta=c.get("beta", 0.0))
    for k in ("tol", "precision", "path", "nufft_w", "n_gl", "singly"):
        if k in c:
            w[k] = c[k]
    return w


def batch_cells(ncell=256, seed=3, nmin=500, nmax=50000, amin=1.0, amax=64.0, nrhs=8, scale=1.0):
    """Batched modified-Helmholtz cells: eta = 1, d = A with A log-uniform in
    [amin, amax] (rectangular), N log-uniform in [nmin, nmax] (times scale),
    nrhs strength vectors N(0,1) per cell, targets = sources."""
    rng = np.random.default_rng(seed)
    cells = []
    for _ in range(ncell):
        A = math.exp(rng.uniform(math.log(amin), math.log(amax)))
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax))) * scale))
        n = max(n, 2)
        e1, e2 = (A, 0.0), (0.0, 1.0)
        src = points(rng, e1, e2, n)
        q = rng.standard_normal((nrhs, n))
        cells.append(dict(e1=e1, e2=e2, src=src, q=q))
    return cells
