"""Full-size parity: each workload at its full size and in the configuration
the benchmark times, compared on sampled targets with the oracle evaluated
one target at a time (direct near-image sum + the plain L D R method with the
oracle's own quadrature, eps 1e-11).  Potentials/velocities are compared
modulo a constant (the sample mean), gradients directly.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import api as oapi
from oracle import ewald, lattice, method

pytestmark = pytest.mark.gpu
NSAMP = 160


def _oracle_at(kernel, beta, e1, e2, src, q, trg_sample, eps=1e-11):
    cell, s, t = lattice.to_canonical(e1, e2, src, trg_sample)
    rot = cell["rot"]
    vec = kernel in ("stokes", "mstokes")
    qq = np.einsum("ij,rjn->rin", rot, q) if vec else q
    g = not vec
    p0, g0 = ewald.near_sum(kernel, beta, cell, t, s, qq, want_grad=g)
    p1, g1 = method.far_field(kernel, beta, cell, t, s, qq, eps=eps, want_grad=g)
    pot, grad = p0 + p1, (g0 + g1 if g else None)
    if vec:
        return np.einsum("ij,rjn->rin", rot.T, pot), None
    return pot, np.einsum("ij,rjn->rin", rot.T, grad)


def _cmp(got, ref, mc):
    return oapi.rel_err(got, ref, modconst=mc)


def _run(w, precision, tol, path, idx=None, singly=False):
    import torch
    from paper_2111_01083_gb300 import PeriodicOp
    dev = torch.device("cuda", 0)
    S = torch.tensor(w["src"], device=dev)
    Q = torch.tensor(w["q"], device=dev)
    self_t = w["trg"] is w["src"]
    T = None if self_t else torch.tensor(w["trg"], device=dev)
    ns = S.shape[1]
    nt = ns if self_t else T.shape[1]
    op = PeriodicOp(w["kernel"], w["e1"], w["e2"], beta=w.get("beta", 0.0), tol=tol, precision=precision, path=path,
                    nufft_w=w.get("nufft_w", 0), n_gl=w.get("n_gl", 0), ns_max=ns, nt_max=nt, singly=singly)
    pot, grad = op(S, Q, T, grad=w["kernel"] not in ("stokes", "mstokes"))
    torch.cuda.synchronize()
    op.status()
    return pot.cpu().numpy(), (None if grad is None else grad.cpu().numpy())


@pytest.mark.parametrize("precision,tol,path", [("mixed", 1e-6, "nufft"), ("fp64", 1e-10, "direct")])
def test_laplace_aspect16_gmm_full(precision, tol, path):
    """1e5 Gaussian-mixture sources in the 16 x 1 cell: the mixed path through the
    NUFFT (w = 8, 8 lines, the timed configuration) and the plain FP64 path."""
    w = workloads.make("laplace_aspect16_gmm_n1e5")
    if precision == "fp64":
        w = dict(w, nufft_w=0, n_gl=0)
    pot, grad = _run(w, precision, tol, path)
    idx = np.random.default_rng(0).choice(w["src"].shape[1], NSAMP, replace=False)
    ref_p, ref_g = _oracle_at("laplace", 0.0, w["e1"], w["e2"], w["src"], w["q"], w["src"][:, idx])
    assert _cmp(pot[:, idx], ref_p, True) < tol
    assert _cmp(grad[:, :, idx], ref_g, False) < tol


def test_stokes_skew_full():
    """2e5 Stokeslets, 2e5 separate targets, skew cell, mixed precision."""
    w = workloads.make("stokes_skew_n2e5")
    vel, _ = _run(w, "mixed", 1e-6, "direct")
    idx = np.random.default_rng(1).choice(w["trg"].shape[1], NSAMP, replace=False)
    ref, _ = _oracle_at("stokes", 0.0, w["e1"], w["e2"], w["src"], w["q"], w["trg"][:, idx])
    assert _cmp(vel[:, :, idx], ref, True) < 1e-6


def test_stokes_hex_full():
    """2e5 Stokeslets, 2e5 separate targets, hexagonal cell: the default
    rotated west/east direction (3 x 3 near block), mixed precision."""
    w = workloads.make("stokes_hex_n2e5")
    vel, _ = _run(w, "mixed", 1e-6, "direct")
    idx = np.random.default_rng(5).choice(w["trg"].shape[1], NSAMP, replace=False)
    ref, _ = _oracle_at("stokes", 0.0, w["e1"], w["e2"], w["src"], w["q"], w["trg"][:, idx])
    assert _cmp(vel[:, :, idx], ref, True) < 1e-6


def test_mstokes_skew_full():
    """1e5 modified Stokeslets (beta = 1, forces with nonzero net force), 1e5
    separate targets, skew cell, mixed precision: the timed configuration."""
    w = workloads.make("mstokes_skew_beta1_n1e5")
    vel, _ = _run(w, "mixed", 1e-6, "direct")
    # 64 sampled targets, far field at eps 1e-9 (the oracle's cost is the
    # formation over all 1e5 sources for both plane-wave families)
    idx = np.random.default_rng(6).choice(w["trg"].shape[1], 64, replace=False)
    ref, _ = _oracle_at("mstokes", 1.0, w["e1"], w["e2"], w["src"], w["q"], w["trg"][:, idx], eps=1e-9)
    assert _cmp(vel[:, :, idx], ref, False) < 1e-6


def test_laplace_adjoint_full():
    """5e4 charges in the 4 x 1 cell: dE/dq = phi, dE/dx = q grad phi at sampled points."""
    import torch
    from paper_2111_01083_gb300 import PeriodicOp, periodic
    w = workloads.make("laplace_adjoint_4x1_n5e4")
    dev = torch.device("cuda", 0)
    n = w["src"].shape[1]
    S = torch.tensor(w["src"], device=dev, requires_grad=True)
    Q = torch.tensor(w["q"], device=dev, requires_grad=True)
    op = PeriodicOp("laplace", w["e1"], w["e2"], tol=1e-6, precision="mixed", ns_max=n, nt_max=n)
    pot, _ = periodic(op, S, Q)
    (0.5 * (Q * pot).sum()).backward()
    idx = np.random.default_rng(2).choice(n, NSAMP, replace=False)
    ref_p, ref_g = _oracle_at("laplace", 0.0, w["e1"], w["e2"], w["src"], w["q"], w["src"][:, idx])
    assert _cmp(Q.grad.detach().cpu().numpy()[:, idx], ref_p, True) < 1e-6
    force = w["q"][0][idx][None, :] * ref_g[0]
    assert _cmp(S.grad.detach().cpu().numpy()[:, idx], force, False) < 1e-6


def test_laplace_adjoint_fd_full():
    """Central finite differences (h = 1e-6, FP64 oracle) of E = 1/2 sum q_i phi(x_i)
    at the full differentiation workload (5e4 charges, 4 x 1 cell), 64 seeded
    position directions and 64 paired charge directions, against the adjoint.

    Only the terms of E that change are evaluated.  Moving x_i by +-h d changes
    the pair terms of i with every other charge and image; by the symmetry of
    the periodic kernel, E(x_i + h d) - E(x_i - h d) = q_i (phi(x_i + h d) -
    phi(x_i - h d)), phi the potential of all charges evaluated at the two
    displaced points (the i-i image terms do not depend on x_i, and the
    singular q_i G(+-h d) terms are equal and cancel).  E is quadratic in q, so
    for the neutral direction v = e_i - e_j, E(q + h v) - E(q - h v) = 2 h v.K q
    = 2 h (phi(x_i) - phi(x_j)) exactly."""
    import torch
    from paper_2111_01083_gb300 import PeriodicOp, periodic
    w = workloads.make("laplace_adjoint_4x1_n5e4")
    dev = torch.device("cuda", 0)
    n = w["src"].shape[1]
    S = torch.tensor(w["src"], device=dev, requires_grad=True)
    Q = torch.tensor(w["q"], device=dev, requires_grad=True)
    op = PeriodicOp("laplace", w["e1"], w["e2"], tol=1e-6, precision="mixed", ns_max=n, nt_max=n)
    pot, _ = periodic(op, S, Q)
    (0.5 * (Q * pot).sum()).backward()
    dq = Q.grad.detach().cpu().numpy()[0]
    dx = S.grad.detach().cpu().numpy()
    h = 1e-6
    rng = np.random.default_rng(64)
    # positions: 64 seeded indices and unit directions
    idx = rng.choice(n, 64, replace=False)
    ang = rng.uniform(0.0, 2.0 * math.pi, 64)
    d = np.stack([np.cos(ang), np.sin(ang)])
    x = w["src"][:, idx]
    pts = np.concatenate([x + h * d, x - h * d], axis=1)
    phi, _ = _oracle_at("laplace", 0.0, w["e1"], w["e2"], w["src"], w["q"], pts)
    fd_x = w["q"][0, idx] * (phi[0, :64] - phi[0, 64:]) / (2 * h)
    ad_x = np.einsum("kn,kn->n", dx[:, idx], d)
    assert _cmp(ad_x, fd_x, False) < 1e-5
    # charges: 64 seeded pairs (i, j), direction e_i - e_j
    pi = rng.choice(n, 64, replace=False)
    pj = rng.choice(n, 64, replace=False)
    keep = pi != pj
    pi, pj = pi[keep], pj[keep]
    phi_q, _ = _oracle_at("laplace", 0.0, w["e1"], w["e2"], w["src"], w["q"],
                          np.concatenate([w["src"][:, pi], w["src"][:, pj]], axis=1))
    m = len(pi)
    fd_q = (2 * h * (phi_q[0, :m] - phi_q[0, m:])) / (2 * h)
    assert _cmp(dq[pi] - dq[pj], fd_q, False) < 1e-5


@pytest.mark.parametrize("beta", [1.0, 10.0, 100.0])
def test_batch_modhelm_full(beta):
    """256 cells, N log-uniform in [500, 5e4], aspect in [1, 64], 8 rhs, one
    graph replay, for each beta of the batched workload; the largest cell and
    3 seeded cells, 48 sampled targets each, against the oracle.  At beta =
    100 the south/north far field is pruned (below eps) and the P2P skips
    (target block, source tile, image) triples beyond the K0 cutoff, so this is
    the configuration that checks those two shortcuts at full size."""
    import torch
    from paper_2111_01083_gb300 import BatchOp
    cells = workloads.batch_cells(ncell=256, seed=3, nrhs=8)
    counts = [c["src"].shape[1] for c in cells]
    dev = torch.device("cuda", 0)
    S = torch.tensor(np.concatenate([c["src"] for c in cells], axis=1), device=dev)
    Q = torch.tensor(np.concatenate([c["q"] for c in cells], axis=1), device=dev)
    op = BatchOp("modhelm", [dict(e1=c["e1"], e2=c["e2"], beta=beta) for c in cells], counts, precision="mixed",
                 nrhs=8, tol=1e-6)
    graph, out = op.capture(S, Q, grad=False)
    graph.replay()
    torch.cuda.synchronize()
    op.status(dev)
    pot = out[0].cpu().numpy()
    edges = np.concatenate([[0], np.cumsum(counts)])
    rng = np.random.default_rng(4)
    big = int(np.argmax(counts))
    for c in [big] + list(rng.choice(256, 3, replace=False)):
        cell = cells[c]
        n = counts[c]
        idx = rng.choice(n, min(48, n), replace=False)
        ref, _ = _oracle_at("modhelm", beta, cell["e1"], cell["e2"], cell["src"], cell["q"], cell["src"][:, idx])
        got = pot[:, edges[c]:edges[c + 1]][:, idx]
        assert _cmp(got, ref, False) < 1e-6, (beta, c, n)


def test_laplace_p1_strip_full():
    """Singly periodic: 1e5 uniform sources in the 1 x 4 strip segment, mixed,
    against the P1 oracle on sampled targets (modulo the constant)."""
    from oracle import p1
    w = workloads.make("laplace_p1_strip4_n1e5")
    pot, grad = _run(dict(w, nufft_w=0, n_gl=0), "mixed", 1e-6, "auto", singly=True)
    idx = np.random.default_rng(5).choice(w["src"].shape[1], NSAMP, replace=False)
    ref_p, ref_g = p1.evaluate("laplace", 0.0, w["e1"], w["e2"], w["src"], w["q"], w["src"][:, idx], eps=1e-11)
    assert _cmp(pot[:, idx], ref_p, True) < 1e-6
    assert _cmp(grad[:, :, idx], ref_g, False) < 1e-6
