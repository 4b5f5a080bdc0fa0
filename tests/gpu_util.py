"""Helpers for the GPU parity tests: run the CUDA library through the C ABI
(the Python binding) and compare with the oracle."""
import numpy as np

from oracle import api as oapi


def run_lib(kernel, e1, e2, src, q, trg=None, beta=0.0, tol=1e-6, precision="mixed", part="total",
            path="direct", grad=True, **kw):
    import torch
    from paper_2111_01083_gb300 import PeriodicOp
    dev = torch.device("cuda", 0)
    S = torch.tensor(np.ascontiguousarray(src), dtype=torch.float64, device=dev)
    Q = torch.tensor(np.ascontiguousarray(q), dtype=torch.float64, device=dev)
    T = None if trg is None else torch.tensor(np.ascontiguousarray(trg), dtype=torch.float64, device=dev)
    nt = S.shape[1] if T is None else T.shape[1]
    op = PeriodicOp(kernel, e1, e2, beta=beta, tol=tol, precision=precision, part=part, path=path,
                    nrhs=q.shape[0], ns_max=S.shape[1], nt_max=nt, **kw)
    pot, g = op(S, Q, T, grad=grad)
    op.status()
    torch.cuda.synchronize()
    return pot.cpu().numpy(), (None if g is None else g.cpu().numpy()), op


def oracle(kernel, e1, e2, src, q, trg=None, beta=0.0, part="total", how="ewald", grad=True, we="auto"):
    t = src if trg is None else trg
    return oapi.evaluate(kernel, beta, e1, e2, src, q, t, part=part, how=how, want_grad=grad, we=we)


def errs(kernel, got, ref):
    """(potential/velocity error, gradient error); Laplace/Stokes modulo constant."""
    mc = kernel != "modhelm"
    ep = oapi.rel_err(got[0], ref[0], modconst=mc)
    eg = None
    if got[1] is not None and ref[1] is not None:
        eg = oapi.rel_err(got[1], ref[1])
    return ep, eg
