"""Adjoint / autograd (pfmm_execute_adjoint behind torch.autograd.Function).

* Energy E = 1/2 sum_i q_i phi(x_i) (targets = sources, self pairs excluded):
  dE/dq = phi and dE/dx_i = q_i grad phi(x_i), checked against the oracle's
  potential and gradient, and against central finite differences of the FP64
  oracle energy (h = 1e-6; q perturbed along e_i - e_j to keep zero net charge).
* Weighted loss L = sum_l w_l u(t_l) with separate targets: dL/dq, dL/ds,
  dL/dt against the oracle (adjoint field of charges w at the targets).
Laplace gradients w.r.t. q are compared after removing the mean (gauge).
"""
import numpy as np
import pytest

import workloads
from gpu_util import oracle
from oracle import api as oapi

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-10, "mixed": 1e-6}


def _tensors(*arrs, grad=True):
    import torch
    dev = torch.device("cuda", 0)
    return [torch.tensor(a, device=dev, requires_grad=grad) for a in arrs]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 2.0)])
def test_energy_gradients_vs_oracle(precision, kernel, beta):
    import torch
    from paper_2111_01083_gb300 import PeriodicOp, periodic
    e1, e2 = (4.0, 0.0), (0.0, 1.0)
    rng = np.random.default_rng(41)
    n = 700
    src = workloads.points(rng, e1, e2, n)
    q = workloads.strengths(rng, 1, n, neutral=kernel != "modhelm")
    S, Q = _tensors(src, q)
    op = PeriodicOp(kernel, e1, e2, beta=beta, tol=TOL[precision], precision=precision, ns_max=n, nt_max=n)
    pot, _ = periodic(op, S, Q)
    E = 0.5 * (Q * pot).sum()
    E.backward()
    phi, gphi = oracle(kernel, e1, e2, src, q, None, beta=beta)
    mc = kernel == "laplace"
    dq = Q.grad.detach().cpu().numpy()
    assert oapi.rel_err(dq, phi, modconst=mc) < TOL[precision]
    force = q[0][None, :] * gphi[0]
    assert oapi.rel_err(S.grad.detach().cpu().numpy(), force) < TOL[precision]


def test_energy_gradients_vs_finite_differences():
    """Central differences of the FP64 oracle energy, h = 1e-6, at 6 seeded
    indices and directions; the adjoint (mixed precision) to 1e-5 relative."""
    import torch
    from paper_2111_01083_gb300 import PeriodicOp, periodic
    e1, e2 = (4.0, 0.0), (0.0, 1.0)
    rng = np.random.default_rng(42)
    n = 160
    src = workloads.points(rng, e1, e2, n)
    q = workloads.strengths(rng, 1, n)
    S, Q = _tensors(src, q)
    op = PeriodicOp("laplace", e1, e2, tol=1e-6, precision="mixed", ns_max=n, nt_max=n)
    pot, _ = periodic(op, S, Q)
    (0.5 * (Q * pot).sum()).backward()
    dq = Q.grad.detach().cpu().numpy()[0]
    dx = S.grad.detach().cpu().numpy()

    def energy(s, qq):
        p, _ = oapi.evaluate("laplace", 0.0, e1, e2, s, qq, s, want_grad=False)
        return 0.5 * float(np.sum(qq * p))

    h = 1e-6
    pick = np.random.default_rng(7)
    for _ in range(3):
        i, j = pick.choice(n, 2, replace=False)
        d = np.zeros_like(q)
        d[0, i], d[0, j] = h, -h
        fd = (energy(src, q + d) - energy(src, q - d)) / (2 * h)
        ad = dq[i] - dq[j]
        assert abs(fd - ad) <= 1e-5 * max(abs(fd), np.abs(dq).max())
    for _ in range(3):
        i = int(pick.integers(n))
        k = int(pick.integers(2))
        d = np.zeros_like(src)
        d[k, i] = h
        fd = (energy(src + d, q) - energy(src - d, q)) / (2 * h)
        assert abs(fd - dx[k, i]) <= 1e-5 * max(abs(fd), np.abs(dx).max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kernel,beta", [("laplace", 0.0), ("modhelm", 1.5)])
def test_weighted_loss_separate_targets(precision, kernel, beta):
    import torch
    from paper_2111_01083_gb300 import PeriodicOp, periodic
    e1, e2 = (2.0, 0.0), (0.4, 1.0)
    rng = np.random.default_rng(43)
    ns, nt = 500, 300
    src = workloads.points(rng, e1, e2, ns)
    trg = workloads.points(rng, e1, e2, nt)
    neutral = kernel != "modhelm"
    q = workloads.strengths(rng, 2, ns, neutral=neutral)
    w = workloads.strengths(rng, 2, nt, neutral=neutral)
    S, Q, T = _tensors(src, q, trg)
    op = PeriodicOp(kernel, e1, e2, beta=beta, tol=TOL[precision], precision=precision, nrhs=2,
                    ns_max=max(ns, nt), nt_max=max(ns, nt))
    pot, _ = periodic(op, S, Q, T)
    W = torch.tensor(w, device=pot.device)
    (W * pot).sum().backward()
    tol = TOL[precision]
    # dL/dq_j = sum_l w_l K(t_l, s_j): the field of charges w at the targets, evaluated at the sources
    psi, gpsi = oracle(kernel, e1, e2, trg, w, src, beta=beta)
    assert oapi.rel_err(Q.grad.detach().cpu().numpy(), psi, modconst=neutral) < tol
    ds = (q[:, None, :] * gpsi).sum(0)
    assert oapi.rel_err(S.grad.detach().cpu().numpy(), ds) < tol
    u, gu = oracle(kernel, e1, e2, src, q, trg, beta=beta)
    dt = (w[:, None, :] * gu).sum(0)
    assert oapi.rel_err(T.grad.detach().cpu().numpy(), dt) < tol


def test_stokes_adjoint_strengths():
    import torch
    from paper_2111_01083_gb300 import PeriodicOp, periodic
    e1, e2 = (1.0, 0.0), (0.3, 0.8)
    rng = np.random.default_rng(44)
    ns, nt = 400, 250
    src = workloads.points(rng, e1, e2, ns)
    trg = workloads.points(rng, e1, e2, nt)
    f = workloads.strengths(rng, 1, ns, stokes=True)
    w = workloads.strengths(rng, 1, nt, stokes=True)
    S, T = _tensors(src, trg, grad=False)
    (F,) = _tensors(f)
    op = PeriodicOp("stokes", e1, e2, tol=1e-10, precision="fp64", ns_max=max(ns, nt), nt_max=max(ns, nt))
    vel = periodic(op, S, F, T)
    (torch.tensor(w, device=vel.device) * vel).sum().backward()
    ref, _ = oracle("stokes", e1, e2, trg, w, src, grad=False)
    assert oapi.rel_err(F.grad.detach().cpu().numpy(), ref, modconst=True) < 1e-10
