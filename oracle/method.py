"""The paper's plain method: direct application P q = L (D (R q)) of the
low-rank factorizations of the four far-field parts (Sec. 6, direct
application, O(r (N_S + N_T)) work), in FP64, for targets and sources
already in the canonical cell.

Per part and kernel (theorem / equation labels of the paper):

modhelm  south/north: Theorem south_thm (Eqs. mpk0s, chialphadef,
         lowranksouth3) and its corollary (Eq. lowranknorth).
         west/east: Eq. pylw02 / tk0west and Theorem west_thm (Eq. lowrankwest)
         with its corollary (Eq. lowrankeast), general m0 (App. A, Eq. k0west2:
         the geometric sum over m <= -(m0+1) gives e^{-(m0+1)kd}/(1-e^{-kd})).
laplace  south/north: Theorem south_thm_lap, corollary north_thm_lap (m = 0
         term -(1/(2 d eta)) y sum q y' each, Eq. phis3).  west/east: Theorem
         west_thm_lap.  Potential gauge (reading of Eq. k1lap/k2lap): the
         source factor is used as (R - 1) (exact under sum q = 0) and the
         target factor as (L - 1), which moves the result by a
         target-independent constant only and removes the 1/lambda
         non-integrable term of the potential integrand.
stokes   south: Theorem south_thm_s (Eqs. pssm, pss0, lowranksouth3s),
         north: the remark after it; west/east: Eq. pssw0 (general m0: the
         factor (P - (P-1) z)/(1-z), P = m0+1, from summing p z^p),
         Theorem west_thm_s and the east remark.  The west/east integrals over
         the whole real line are written as 2 Re of the half line, so the
         half-line prefactor is 1/(4 pi).  Same (L - 1)/(R - 1) gauge.

West/east frame (App. A).  By default the west/east plane waves decay
along x (e1).  With cell["we_rot"] they decay along x~ = e2-perp instead:
coordinates (x~, y~) = (c x - s y, s x + c y) with c = eta/|e2|, s = xi/|e2|,
in which e2 = (0, |e2|) and e1 = (d c, d s) (Eq. k0west2).  The geometric sum
over the image columns m <= -(m0+1) then has the complex ratio
e^{-(kappa d c - i lambda d s)}, the rows n = -1, 0, 1 shift only y~, and
m0 = 1 suffices for every parallelogram (smallest gap d c).  Stokes: forces
are rotated into the frame and velocities back; scalar gradients likewise.

mstokes  (modified Stokeslet, beta > 0) south/north: Theorem south_thm_ms
         (Eqs. pmss1, chialphadefms, lowranksouth3ms): per mode m a beta
         family (decay chi_m, block [[chi, i alpha], [i alpha, -alpha^2/chi]])
         and a Laplace family (decay |alpha_m|, block [[-|a|, -i a], [-i a, |a|]]),
         each with the scalar lattice factor e^{-2Q}/(1 - e^{-Q}) / (2 beta^2 d);
         north: conjugate blocks.  The Laplace family has no m = 0 term: each
         image row is Poisson-summed on its own, and the row's zero mode of
         grad grad^T log r vanishes (its integral over x is 0).
         west/east: Theorem west_thm_ms (Eq. pmsw0, general m0): blocks
         [[-lambda^2/kappa, i lambda], [i lambda, kappa]] (kappa = sqrt(lambda^2 +
         beta^2)) and [[|l|, -i l], [-i l, -|l|]] (kappa = |lambda|), 2 Re of the
         half line, prefactor 1/(2 pi beta^2); east: conjugate blocks.  No gauge
         and no coordinate channels: both families are integrable at lambda = 0.

Modes: M from Eq. mpk0s.  West/east quadrature: this oracle's own,
deliberately over-resolved composite Gauss-Legendre rule in lambda' = lambda d
(panels of width 1/2, narrower when the oscillation span exceeds 2d, 20
points each, dyadic panels toward 0 when beta d < 1, truncated where
exp(-kappa' x_min') < eps e^-8 with x_min' the smallest scaled west/east gap).
The paper's precomputed GGQ tables are not printed, so any accurate rule is a
valid reading.
"""
import math
import numpy as np

PARTS = ("south", "north", "west", "east")


def mpk0s(d, eta, eps):
    """Eq. mpk0s: number of modes M for precision eps."""
    r = 2 * math.pi * eta / d
    return int(math.ceil((d / (2 * math.pi * eta)) * math.log(1.0 / ((1.0 - math.exp(-r)) * eps))))


def we_frame(cell):
    """West/east frame: rotation (c, s) to (x~, y~), the image-column step
    (dx, dy) and row step (xr, yr) in that frame, the smallest gap x - x' -
    (image x) over the far columns, and the largest lambda-frequency of the
    integrand (|y~ - y~'| + row shifts + the phase of the first far column)."""
    d, xi, eta, m0 = cell["d"], cell["xi"], cell["eta"], cell["m0"]
    if not cell.get("we_rot", False):
        return dict(c=1.0, s=0.0, dx=d, dy=0.0, xr=xi, yr=eta, gap=m0 * d - 2 * abs(xi), freq=2 * eta)
    h = math.hypot(xi, eta)
    c, s = eta / h, xi / h
    dx, dy = d * c, d * s
    # x~ of a point in the cell spans exactly dx (e2 has no x~ part)
    return dict(c=c, s=s, dx=dx, dy=dy, xr=0.0, yr=h, gap=m0 * dx,
                freq=2 * h + (m0 + 2) * abs(dy))


def _to_frame(fr, pts):
    return np.stack([fr["c"] * pts[0] - fr["s"] * pts[1], fr["s"] * pts[0] + fr["c"] * pts[1]])


def _from_frame(fr, v):
    # v[..., 2, n] in the frame -> canonical (the transpose rotation)
    c, s = fr["c"], fr["s"]
    return np.stack([c * v[..., 0, :] + s * v[..., 1, :], -s * v[..., 0, :] + c * v[..., 1, :]], axis=-2)


def we_quadrature(cell, beta, eps, width=0.5, npts=20):
    """Nodes lambda_n > 0 and weights w_n for int_0^inf (.) d lambda."""
    d = cell["d"]
    fr = we_frame(cell)
    xmin = fr["gap"] / d
    width = width * min(1.0, 2.0 * d / fr["freq"])
    bt = beta * d
    top = (math.log(1.0 / eps) + 8.0) / xmin
    if top <= bt:
        return np.zeros(0), np.zeros(0)
    lam_max = math.sqrt(top * top - bt * bt)
    edges = [0.0]
    if 0 < bt < 1:
        e = bt / 16
        while e < 0.5:
            edges.append(e)
            e *= 2
    e = edges[-1]
    while e < lam_max:
        e = min(lam_max, (math.floor(e / width + 1e-9) + 1) * width)
        edges.append(e)
    gx, gw = np.polynomial.legendre.leggauss(npts)
    nodes, wts = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        nodes.append(0.5 * (b - a) * (gx + 1) + a)
        wts.append(0.5 * (b - a) * gw)
    return np.concatenate(nodes) / d, np.concatenate(wts) / d


def _scalar_sn(kernel, beta, cell, trg, src, q, eps, part, want_grad):
    d, xi, eta = cell["d"], cell["xi"], cell["eta"]
    M = mpk0s(d, eta, eps)
    m = np.arange(-M, M + 1)
    if kernel == "laplace":
        m = m[m != 0]
    al = 2 * np.pi * m / d
    chi = np.sqrt(al * al + beta * beta) if kernel == "modhelm" else np.abs(al)
    Q = chi * eta - 1j * al * xi
    D = np.exp(-2 * Q) / (2 * d * chi * (1 - np.exp(-Q)))
    sgn = 1.0 if part == "south" else -1.0
    if part == "north":
        D = np.conj(D)
    R = np.exp(sgn * chi[:, None] * src[1][None, :] - 1j * al[:, None] * src[0][None, :])
    w = (q.astype(complex) @ R.T) * D  # [nrhs, nm]
    L = np.exp(-sgn * chi[None, :] * trg[1][:, None] + 1j * al[None, :] * trg[0][:, None])
    pot = (w @ L.T).real
    grad = None
    if want_grad:
        gx = ((w * (1j * al)) @ L.T).real
        gy = ((w * (-sgn * chi)) @ L.T).real
        grad = np.stack([gx, gy], axis=1)
    if kernel == "laplace":
        s1 = q @ src[1]  # [nrhs]
        c0 = -1.0 / (2 * d * eta)
        pot = pot + c0 * s1[:, None] * trg[1][None, :]
        if want_grad:
            grad[:, 1, :] += c0 * s1[:, None]
    return pot, grad


def _scalar_we(kernel, beta, cell, trg, src, q, eps, part, want_grad, rows=(-1, 0, 1)):
    m0 = cell["m0"]
    fr = we_frame(cell)
    lam, w = we_quadrature(cell, beta if kernel == "modhelm" else 0.0, eps)
    nrhs, nt = q.shape[0], trg.shape[1]
    if lam.size == 0:
        return np.zeros((nrhs, nt)), np.zeros((nrhs, 2, nt)) if want_grad else None
    trg, src = _to_frame(fr, trg), _to_frame(fr, src)
    kap = np.sqrt(lam * lam + beta * beta) if kernel == "modhelm" else lam
    P = m0 + 1
    # rows n of image columns m <= -(m0+1): sum_n e^{n (kappa xr - i lambda yr)}
    B = sum(np.exp(n * (kap * fr["xr"] - 1j * lam * fr["yr"])) for n in rows)
    # columns: sum_{p >= P} e^{-p g}, g = kappa dx - i lambda dy
    g = kap * fr["dx"] - 1j * lam * fr["dy"]
    F = np.exp(-P * g) / (1 - np.exp(-g))
    D = w / (2 * np.pi * kap) * F * B
    s = 1.0 if part == "west" else -1.0  # east: x -> -x, D -> conj
    if part == "east":
        D = np.conj(D)
    R = np.exp(s * kap[:, None] * src[0][None, :] - 1j * lam[:, None] * src[1][None, :])
    L = np.exp(-s * kap[None, :] * trg[0][:, None] + 1j * lam[None, :] * trg[1][:, None])
    if kernel == "laplace":
        R = R - 1.0
    wv = (q.astype(complex) @ R.T) * D
    Lp = (L - 1.0) if kernel == "laplace" else L
    pot = (wv @ Lp.T).real
    grad = None
    if want_grad:
        gx = ((wv * (-s * kap)) @ L.T).real
        gy = ((wv * (1j * lam)) @ L.T).real
        grad = _from_frame(fr, np.stack([gx, gy], axis=1))
    return pot, grad


def _stokes_sn(cell, trg, src, f, eps, part):
    d, xi, eta = cell["d"], cell["xi"], cell["eta"]
    M = mpk0s(d, eta, eps)
    m = np.arange(-M, M + 1)
    m = m[m != 0]
    al = 2 * np.pi * m / d
    a = np.abs(al)
    sg = np.sign(m)
    Q = a * eta - 1j * al * xi
    north = part == "north"
    if north:
        Q = np.conj(Q)
    z = np.exp(-Q)
    S = np.zeros((m.size, 2, 2), complex)
    S[:, 0, 0] = 1
    S[:, 0, 1] = S[:, 1, 0] = 1j * sg
    S[:, 1, 1] = -1
    if north:
        S = np.conj(S)
    pre = (z * z / (1 - z)) / (4 * d)
    I2 = np.eye(2)[None]
    Db = pre[:, None, None] * S
    Da = pre[:, None, None] * (I2 / a[:, None, None] - (eta * (2 - z) / (1 - z))[:, None, None] * S)
    sy = -1.0 if north else 1.0
    R = np.exp(sy * a[:, None] * src[1][None, :] - 1j * al[:, None] * src[0][None, :])  # [nm, ns]
    L = np.exp(-sy * a[None, :] * trg[1][:, None] + 1j * al[None, :] * trg[0][:, None])  # [nt, nm]
    fc = f.astype(complex)
    ca = np.einsum("rcj,mj->rcm", fc, R)
    cb = np.einsum("rcj,mj->rcm", fc * src[1][None, None, :], R)
    wa = np.einsum("mij,rjm->rim", Da, ca) + sy * np.einsum("mij,rjm->rim", Db, cb)
    wb = np.einsum("mij,rjm->rim", Db, ca)
    vel = np.einsum("lm,rim->ril", L, wa).real - sy * trg[1][None, None, :] * np.einsum("lm,rim->ril", L, wb).real
    c0 = -1.0 / (2 * d * eta)
    vel[:, 0, :] += c0 * (f[:, 0, :] @ src[1])[:, None] * trg[1][None, :]
    return vel


def _stokes_we(cell, trg, src, f, eps, part, rows=(-1, 0, 1)):
    m0 = cell["m0"]
    fr = we_frame(cell)
    lam, w = we_quadrature(cell, 0.0, eps)
    trg, src = _to_frame(fr, trg), _to_frame(fr, src)
    f = _to_frame(fr, f.transpose(1, 0, 2)).transpose(1, 0, 2)  # [r][c][n] forces in the frame
    d = fr["dx"]
    P = m0 + 1
    # column ratio (complex when the columns also shift y~)
    z = np.exp(-lam * fr["dx"] + 1j * lam * fr["dy"])
    ph = {n: np.exp(n * (lam * fr["xr"] - 1j * lam * fr["yr"])) for n in rows}
    B = sum(ph.values())
    # the x-shift n xr of row n enters the coordinate factor: sum_n n xr phi_n
    dph = fr["xr"] * sum(n * ph[n] for n in rows)
    Sp = np.zeros((lam.size, 2, 2), complex)
    Sp[:, 0, 0] = -1
    Sp[:, 0, 1] = Sp[:, 1, 0] = 1j
    Sp[:, 1, 1] = 1
    pref = w / (4 * np.pi) * z ** P / (1 - z)
    I2 = np.eye(2)[None]
    Db = (pref * B)[:, None, None] * Sp
    Da = pref[:, None, None] * (
        B[:, None, None] * (I2 / lam[:, None, None] - (P * d + d * z / (1 - z))[:, None, None] * Sp)
        + dph[:, None, None] * Sp
    )
    east = part == "east"
    s = -1.0 if east else 1.0
    if east:
        Da, Db = np.conj(Da), np.conj(Db)
    R = np.exp(s * lam[:, None] * src[0][None, :] - 1j * lam[:, None] * src[1][None, :])
    L = np.exp(-s * lam[None, :] * trg[0][:, None] + 1j * lam[None, :] * trg[1][:, None])
    fc = f.astype(complex)
    ca = np.einsum("rcj,mj->rcm", fc, R - 1.0)
    cb = np.einsum("rcj,mj->rcm", fc * src[0][None, None, :], R)
    wa = np.einsum("mij,rjm->rim", Da, ca) + s * np.einsum("mij,rjm->rim", Db, cb)
    wb = np.einsum("mij,rjm->rim", Db, ca)
    vel = np.einsum("lm,rim->ril", L - 1.0, wa).real - s * trg[0][None, None, :] * np.einsum("lm,rim->ril", L, wb).real
    return _from_frame(fr, vel)


def _mstokes_sn(beta, cell, trg, src, f, eps, part):
    d, xi, eta = cell["d"], cell["xi"], cell["eta"]
    M = mpk0s(d, eta, eps)
    m = np.arange(-M, M + 1)
    al = 2 * np.pi * m / d
    chi = np.sqrt(al * al + beta * beta)
    a = np.abs(al)
    north = part == "north"
    sy = -1.0 if north else 1.0
    fc = f.astype(complex)
    vel = np.zeros((f.shape[0], 2, trg.shape[1]))
    fams = []
    # beta family, every m
    Qb = chi * eta - 1j * al * xi
    Mb = np.empty((m.size, 2, 2), complex)
    Mb[:, 0, 0] = chi
    Mb[:, 0, 1] = Mb[:, 1, 0] = 1j * al
    Mb[:, 1, 1] = -al * al / chi
    fams.append((chi, al, np.exp(-2 * Qb) / (1 - np.exp(-Qb)), Mb))
    # Laplace family, m != 0
    nz = m != 0
    Q0 = a[nz] * eta - 1j * al[nz] * xi
    M0 = np.empty((nz.sum(), 2, 2), complex)
    M0[:, 0, 0] = -a[nz]
    M0[:, 0, 1] = M0[:, 1, 0] = -1j * al[nz]
    M0[:, 1, 1] = a[nz]
    fams.append((a[nz], al[nz], np.exp(-2 * Q0) / (1 - np.exp(-Q0)), M0))
    for dec, alp, lat, Mat in fams:
        D = (lat / (2 * beta * beta * d))[:, None, None] * Mat
        if north:
            D = np.conj(D)
        R = np.exp(sy * dec[:, None] * src[1][None, :] - 1j * alp[:, None] * src[0][None, :])
        L = np.exp(-sy * dec[None, :] * trg[1][:, None] + 1j * alp[None, :] * trg[0][:, None])
        c = np.einsum("rcj,mj->rcm", fc, R)
        w = np.einsum("mij,rjm->rim", D, c)
        vel += np.einsum("lm,rim->ril", L, w).real
    return vel


def _mstokes_we(beta, cell, trg, src, f, eps, part):
    m0 = cell["m0"]
    fr = we_frame(cell)
    trg, src = _to_frame(fr, trg), _to_frame(fr, src)
    f = _to_frame(fr, f.transpose(1, 0, 2)).transpose(1, 0, 2)
    P = m0 + 1
    east = part == "east"
    s = -1.0 if east else 1.0
    fc = f.astype(complex)
    vel = np.zeros((f.shape[0], 2, trg.shape[1]))
    for fam_beta in (beta, 0.0):
        lam, w = we_quadrature(cell, fam_beta, eps)
        if lam.size == 0:
            continue
        kap = np.sqrt(lam * lam + fam_beta * fam_beta)
        B = sum(np.exp(n * (kap * fr["xr"] - 1j * lam * fr["yr"])) for n in (-1, 0, 1))
        g = kap * fr["dx"] - 1j * lam * fr["dy"]
        F = np.exp(-P * g) / (1 - np.exp(-g))
        Mat = np.empty((lam.size, 2, 2), complex)
        if fam_beta > 0:
            Mat[:, 0, 0] = -lam * lam / kap
            Mat[:, 0, 1] = Mat[:, 1, 0] = 1j * lam
            Mat[:, 1, 1] = kap
        else:
            Mat[:, 0, 0] = lam
            Mat[:, 0, 1] = Mat[:, 1, 0] = -1j * lam
            Mat[:, 1, 1] = -lam
        D = (w / (2 * np.pi * beta * beta) * F * B)[:, None, None] * Mat
        if east:
            D = np.conj(D)
        R = np.exp(s * kap[:, None] * src[0][None, :] - 1j * lam[:, None] * src[1][None, :])
        L = np.exp(-s * kap[None, :] * trg[0][:, None] + 1j * lam[None, :] * trg[1][:, None])
        c = np.einsum("rcj,mj->rcm", fc, R)
        wv = np.einsum("mij,rjm->rim", D, c)
        vel += np.einsum("lm,rim->ril", L, wv).real
    return _from_frame(fr, vel)


def far_field(kernel, beta, cell, trg, src, q, eps=1e-14, parts=PARTS, want_grad=True, chunk=4096,
              rows=(-1, 0, 1)):
    """Sum of the requested far-field parts at the targets.
    Returns (pot, grad) for scalar kernels, (vel, None) for stokes.
    rows: the image rows n of the west/east parts (all three for the doubly
    periodic sum; (0,) for the singly periodic one)."""
    trg = np.asarray(trg, np.float64)
    src = np.asarray(src, np.float64)
    q = np.asarray(q, np.float64)
    nt = trg.shape[1]
    nrhs = q.shape[0]
    if kernel == "stokes":
        out = np.zeros((nrhs, 2, nt))
        for l0 in range(0, nt, chunk):
            t = trg[:, l0:l0 + chunk]
            for p in parts:
                if p in ("south", "north"):
                    out[:, :, l0:l0 + chunk] += _stokes_sn(cell, t, src, q, eps, p)
                else:
                    out[:, :, l0:l0 + chunk] += _stokes_we(cell, t, src, q, eps, p, rows)
        return out, None
    if kernel == "mstokes":
        if tuple(rows) != (-1, 0, 1):
            raise ValueError("mstokes: doubly periodic only")
        out = np.zeros((nrhs, 2, nt))
        for l0 in range(0, nt, chunk):
            t = trg[:, l0:l0 + chunk]
            for p in parts:
                if p in ("south", "north"):
                    out[:, :, l0:l0 + chunk] += _mstokes_sn(beta, cell, t, src, q, eps, p)
                else:
                    out[:, :, l0:l0 + chunk] += _mstokes_we(beta, cell, t, src, q, eps, p)
        return out, None
    pot = np.zeros((nrhs, nt))
    grad = np.zeros((nrhs, 2, nt)) if want_grad else None
    for l0 in range(0, nt, chunk):
        t = trg[:, l0:l0 + chunk]
        for p in parts:
            if p in ("south", "north"):
                pp, gg = _scalar_sn(kernel, beta, cell, t, src, q, eps, p, want_grad)
            else:
                pp, gg = _scalar_we(kernel, beta, cell, t, src, q, eps, p, want_grad, rows)
            pot[:, l0:l0 + chunk] += pp
            if want_grad:
                grad[:, :, l0:l0 + chunk] += gg
    return pot, grad
