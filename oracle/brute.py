"""Brute-force image sums for the modified Helmholtz kernel (oracle pin).

For beta > 0 the Green's function (1/2pi) K0(beta r) decays exponentially, so
every sum over image cells in Sec. 3 converges absolutely and can be
truncated at a radius R with K0(beta R) below 1e-18.  This gives each of the
four far-field parts of Eq. ksplitting2 separately (m0 taken from the cell):

  south: n <= -2 (all m)      north: n >= 2 (all m)
  west : |n| <= 1, m <= -(m0+1)   east : |n| <= 1, m >= m0+1

and their sum, the whole far field P2 q.  It checks each low-rank
factorization on its own, not only their total.
"""
import math
import numpy as np

from .greens import image_sum

PARTS = ("south", "north", "west", "east")


def part_offsets(cell, beta, part, rmax=None):
    d, xi, eta, m0 = cell["d"], cell["xi"], cell["eta"], cell["m0"]
    if rmax is None:
        rmax = 41.0 / beta
    diam = max(math.hypot(d + xi, eta), math.hypot(d - xi, eta))
    R = rmax + diam
    nmax = int(R / eta) + 2
    out = []
    for n in range(-nmax, nmax + 1):
        mmax = int((R + abs(n * xi)) / d) + 2
        for m in range(-mmax, mmax + 1):
            if part == "south" and not n <= -2:
                continue
            if part == "north" and not n >= 2:
                continue
            if part == "west" and not (abs(n) <= 1 and m <= -(m0 + 1)):
                continue
            if part == "east" and not (abs(n) <= 1 and m >= m0 + 1):
                continue
            if part == "far" and (abs(n) <= 1 and abs(m) <= m0):
                continue
            L = (m * d + n * xi, n * eta)
            if math.hypot(*L) <= R:
                out.append(L)
    return np.array(out).reshape(-1, 2)


def modhelm_part(cell, beta, trg, src, q, part="far", want_grad=True):
    offs = part_offsets(cell, beta, part)
    if len(offs) == 0:
        nrhs, nt = q.shape[0], trg.shape[1]
        return np.zeros((nrhs, nt)), np.zeros((nrhs, 2, nt))
    return image_sum("modhelm", beta, trg, src, q, offs, want_grad)
