"""Input-frame entry points of the oracle.

The library takes lattice vectors e1, e2 in any orientation, points anywhere
in the plane (wrapped into the cell), and returns potentials, gradients and
velocities in the input frame.  These helpers do the same for the oracle:
canonicalise (``lattice``), evaluate in the canonical frame, rotate vectors
back (canonical = rot @ input, so input = rot^T @ canonical).

part: "total" (K^(p) q = K^near q + P2 q), "far" (P2 q), "near" (K^near q).
how : "ewald" (the definition), "plain" (the paper's direct L D R method).
The modified Stokeslet ("mstokes") has no Ewald form here: its periodic sum
is defined in the paper's order (image rows), which the plain method follows
and tests/test_oracle_mstokes_pins.py pins against exact row sums; "ewald"
is refused for it.
"""
import numpy as np

from . import ewald, lattice, method


def _rot_vec(rotT, v):
    # v[..., 2, n] -> rotT @ v
    return np.einsum("ij,...jn->...in", rotT, v)


def evaluate(kernel, beta, e1, e2, src, q, trg, part="total", how="ewald", eps=1e-14,
             want_grad=True, margin_frac=0.25, we="auto"):
    """we: west/east plane-wave direction, "axis", "rotated" (App. A) or
    "auto" (lattice.choose_we); it sets m0 and so the near/far split."""
    src = np.asarray(src, np.float64)
    trg = np.asarray(trg, np.float64)
    q = np.asarray(q, np.float64)
    cell, s, t = lattice.to_canonical(e1, e2, src, trg, margin_frac, we)
    rot = cell["rot"]
    if kernel == "mstokes" and how == "ewald" and part != "near":
        raise ValueError("mstokes: use how='plain' (no Ewald form)")
    if kernel in ("stokes", "mstokes"):
        q = np.einsum("ij,rjn->rin", rot, q)
        want_grad = False
    pot = 0.0
    grad = 0.0 if want_grad else None
    if part in ("total", "near"):
        p, g = ewald.near_sum(kernel, beta, cell, t, s, q, want_grad)
        pot = pot + p
        if want_grad:
            grad = grad + g
    if part in ("total", "far"):
        if how == "ewald":
            p, g = ewald.far_sum(kernel, beta, cell, t, s, q, want_grad)
        else:
            p, g = method.far_field(kernel, beta, cell, t, s, q, eps=eps, want_grad=want_grad)
        pot = pot + p
        if want_grad:
            grad = grad + g
    if kernel in ("stokes", "mstokes"):
        return _rot_vec(rot.T, pot), None
    return pot, (_rot_vec(rot.T, grad) if want_grad else None)


def stokes_pressure(e1, e2, src, f, trg, how="ewald", eps=1e-14, margin_frac=0.25, we="auto"):
    """Pressure of the periodic Stokeslet sum, input frame, [nrhs][nt].

    The free-space Stokeslet of this normalisation, u = (1/4pi)(-log r I +
    r r^T / r^2) f, has pressure p = (1/2pi) f . r / r^2 = -f . grad G_L with
    G_L = -(1/2pi) log r the Laplace kernel; summed over the lattice (zero net
    force) this is p = -(d/dx phi[f_x] + d/dy phi[f_y]), phi[c] the periodic
    Laplace potential of charges c.  Evaluated with the Laplace field of this
    oracle (part="total": near images plus the periodizing part).
    """
    f = np.asarray(f, np.float64)
    nrhs = f.shape[0]
    q = f.reshape(2 * nrhs, -1)  # [r][c][n] -> rows (r, c)
    _, g = evaluate("laplace", 0.0, e1, e2, src, q, trg, how=how, eps=eps, margin_frac=margin_frac, we=we)
    g = g.reshape(nrhs, 2, 2, -1)  # [r][c][component][n]
    return -(g[:, 0, 0] + g[:, 1, 1])


def rel_err(a, b, modconst=False):
    """Relative l2 error over all entries; modconst removes the best-fit
    constant per rhs (per component) along the last axis first."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if modconst:
        a = a - a.mean(-1, keepdims=True)
        b = b - b.mean(-1, keepdims=True)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
