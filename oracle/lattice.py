"""Unit cell conventions of the paper, restated for the oracle.

Sec. 1: the cell is C = {x1 e1 + x2 e2 : x1, x2 in [-1/2, 1/2]} with
e1 = (d, 0), e2 = (xi, eta), d, eta > 0 and d >= |e2|.  Any input basis is
brought to that form by (i) Lagrange-Gauss reduction (a change of basis of
the same lattice, so the periodic sum is unchanged), (ii) taking the longer
reduced vector as e1, (iii) rotating e1 onto +x and (iv) flipping e2 so that
eta > 0.  After reduction |xi| <= d/2.

Definition of Lambda_near (Sec. 1): m in [-m0, m0], n in {-1, 0, 1}.  The
west/east plane-wave integrals need x - x' - m d - n xi >= margin > 0 for every
far image in the three middle rows (proof after Eq. pylw02); with points in
the parallelogram the smallest such gap is m0 d - 2|xi|, which gives the rule
m0 = max(1, ceil((margin + 2|xi|)/d)).  margin = d reproduces the paper's
choice (m0 = 1 for rectangles, m0 = 2 for 0 < |xi| <= d/2).  The default here
is margin = d/4 (reading: any positive gap keeps the west/east integrands
exponentially decaying; a smaller gap only needs more quadrature nodes), so
m0 = 1 unless |xi| > 3d/8, which keeps the near block at 3 x 3 cells for most
parallelograms.
"""
import math
import numpy as np


def _round_half_up(v):
    return math.floor(v + 0.5)


def canonicalize(e1, e2):
    """Return dict(d, xi, eta, rot) with rot the 2x2 rotation taking input
    coordinates to the canonical frame (canonical = rot @ input)."""
    b1 = np.array(e1, dtype=np.float64)
    b2 = np.array(e2, dtype=np.float64)
    cross = b1[0] * b2[1] - b1[1] * b2[0]
    if not np.all(np.isfinite(b1)) or not np.all(np.isfinite(b2)) or abs(cross) <= 1e-14 * (
        np.dot(b1, b1) + np.dot(b2, b2)
    ):
        raise ValueError("degenerate lattice")
    # Lagrange-Gauss reduction
    for _ in range(200):
        if np.dot(b1, b1) > np.dot(b2, b2):
            b1, b2 = b2, b1
        mu = _round_half_up(np.dot(b1, b2) / np.dot(b1, b1))
        if mu == 0:
            break
        b2 = b2 - mu * b1
    a, b = b2, b1  # a: longer (becomes e1), b: shorter (becomes e2)
    d = math.hypot(a[0], a[1])
    c, s = a[0] / d, a[1] / d
    rot = np.array([[c, s], [-s, c]])
    bb = rot @ b
    if bb[1] < 0:
        bb = -bb
    return dict(d=d, xi=float(bb[0]), eta=float(bb[1]), rot=rot)


def choose_m0(d, xi, margin_frac=0.25):
    """Smallest m0 >= 1 with m0 d - 2|xi| >= margin_frac * d."""
    return max(1, int(math.ceil((margin_frac * d + 2.0 * abs(xi)) / d - 1e-12)))


def wrap(pts, d, xi, eta):
    """Wrap canonical-frame points [2, n] into the cell: fractional coordinate
    u -> u - floor(u + 1/2), i.e. u in [-1/2, 1/2)."""
    x, y = np.asarray(pts[0], np.float64), np.asarray(pts[1], np.float64)
    u2 = y / eta
    u1 = (x - u2 * xi) / d
    u1 = u1 - np.floor(u1 + 0.5)
    u2 = u2 - np.floor(u2 + 0.5)
    return np.stack([u1 * d + u2 * xi, u2 * eta])


def near_offsets(d, xi, eta, m0):
    """Image offsets l_mn = m e1 + n e2 for (m, n) in Lambda_near."""
    out = []
    for n in (-1, 0, 1):
        for m in range(-m0, m0 + 1):
            out.append((m * d + n * xi, n * eta))
    return np.array(out)


def choose_we(d, xi, we="auto", margin_frac=0.25):
    """West/east plane-wave direction and m0.  "axis": decay along e1 with m0
    from choose_m0; "rotated": decay along e2-perp (App. A), m0 = 1 for any
    cell; "auto": rotated exactly when the axis direction would need m0 >= 2.
    Returns (we_rot, m0)."""
    if we not in ("axis", "rotated", "auto"):
        raise ValueError("we must be axis, rotated or auto")
    m0 = choose_m0(d, xi, margin_frac)
    rot = we == "rotated" or (we == "auto" and m0 >= 2)
    return rot, (1 if rot else m0)


def to_canonical(e1, e2, src, trg, margin_frac=0.25, we="auto"):
    """Canonicalise the lattice and wrap sources/targets given in the input
    frame ([2, n] arrays).  Returns (cell dict incl. m0 and we_rot, src_c,
    trg_c)."""
    cell = canonicalize(e1, e2)
    cell["we_rot"], cell["m0"] = choose_we(cell["d"], cell["xi"], we, margin_frac)
    R = cell["rot"]
    s = wrap(R @ np.asarray(src, np.float64), cell["d"], cell["xi"], cell["eta"])
    t = wrap(R @ np.asarray(trg, np.float64), cell["d"], cell["xi"], cell["eta"])
    return cell, s, t
