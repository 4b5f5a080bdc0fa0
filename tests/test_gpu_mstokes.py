"""GPU parity of the modified Stokes kernel (Eq. msgreen; Theorems
south_thm_ms, west_thm_ms): the CUDA library (through the C ABI) against the
FP64 oracle's plain method (near images + the paper's factorized far parts,
pinned in tests/test_oracle_mstokes_pins.py against exact image-row sums).

Tolerances: FP64 path 1e-10, mixed path 1e-6 (relative l2 over all targets,
rhs and components; no constant is removed: the modified Stokes velocity is
unique).  Sizes span several 128-source tiles and 256-target blocks with
ragged tails; forces need no zero net force.
"""
import math

import numpy as np
import pytest

import workloads
from gpu_util import oracle, run_lib
from oracle import api as oapi

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}
LAT = {
    "square": ((1.0, 0.0), (0.0, 1.0)),
    "skew": ((1.0, 0.0), (0.3, 0.8)),
    "hex": ((1.0, 0.0), (0.5, math.sqrt(3) / 2)),
    "rotated": ((1.2, 0.4), (-0.5, 0.9)),
    "rect8": ((8.0, 0.0), (0.0, 1.0)),
}


def _case(lat, ns, nt=None, seed=0, nrhs=1, dist="uniform"):
    e1, e2 = LAT[lat]
    rng = np.random.default_rng(seed)
    src = workloads.points(rng, e1, e2, ns, dist)
    f = rng.standard_normal((nrhs, 2, ns))  # net force not zero
    trg = None if nt is None else workloads.points(rng, e1, e2, nt)
    return e1, e2, src, f, trg


def _err(got, ref):
    return oapi.rel_err(got, ref)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("beta", [0.5, 3.0])
@pytest.mark.parametrize("lat", ["square", "skew", "hex", "rotated", "rect8"])
def test_total(precision, beta, lat):
    e1, e2, src, f, trg = _case(lat, 700, nt=333, seed=70)
    got = run_lib("mstokes", e1, e2, src, f, trg, beta=beta, tol=TOL[precision], precision=precision, grad=False)
    ref = oracle("mstokes", e1, e2, src, f, trg, beta=beta, how="plain", grad=False)
    assert _err(got[0], ref[0]) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nrhs", [3, 5])
def test_self_targets_multi_rhs(precision, nrhs):
    """targets = sources (self pairs skipped), clustered points, rhs groups of 4/2/1."""
    e1, e2, src, f, _ = _case("skew", 1100, seed=71, nrhs=nrhs, dist="gmm")
    got = run_lib("mstokes", e1, e2, src, f, None, beta=2.0, tol=TOL[precision], precision=precision, grad=False)
    ref = oracle("mstokes", e1, e2, src, f, None, beta=2.0, how="plain", grad=False)
    assert _err(got[0], ref[0]) < TOL[precision]


@pytest.mark.parametrize("part", ["far", "near"])
@pytest.mark.parametrize("we", ["rotated", "axis"])
def test_parts_fp64(part, we):
    e1, e2, src, f, trg = _case("hex", 400, nt=257, seed=72)
    got = run_lib("mstokes", e1, e2, src, f, trg, beta=1.5, tol=1e-10, precision="fp64", part=part, grad=False, we=we)
    assert got[2].describe()["m0"] == (1 if we == "rotated" else 2)
    ref = oracle("mstokes", e1, e2, src, f, trg, beta=1.5, part=part, how="plain", grad=False, we=we)
    assert _err(got[0], ref[0]) < 1e-10


@pytest.mark.parametrize("ns,nt", [(1, 5), (2, 1), (129, 1), (300, 0)])
def test_tiny_and_empty(ns, nt):
    e1, e2 = LAT["skew"]
    rng = np.random.default_rng(73)
    src = workloads.points(rng, e1, e2, ns)
    f = rng.standard_normal((1, 2, ns))
    trg = workloads.points(rng, e1, e2, nt)
    for precision in ("fp64", "mixed"):
        got = run_lib("mstokes", e1, e2, src, f, trg, beta=1.0, tol=TOL[precision], precision=precision, grad=False)
        if nt == 0:
            assert got[0].size == 0
            continue
        ref = oracle("mstokes", e1, e2, src, f, trg, beta=1.0, how="plain", grad=False)
        assert _err(got[0], ref[0]) < TOL[precision]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_periodicity(precision, tol):
    """The field just inside one edge equals the field just inside the
    opposite edge (Sec. 7), on a 4 x 1 skewed cell."""
    e1, e2 = (4.0, 0.0), (0.7, 1.0)
    rng = np.random.default_rng(74)
    src = workloads.points(rng, e1, e2, 1500, "gmm")
    f = rng.standard_normal((1, 2, 1500))
    E = np.array([e1, e2]).T
    s = rng.uniform(-0.45, 0.45, 200)
    pairs = []
    for w in (0, 1):
        a = np.zeros((2, 200))
        b = np.zeros((2, 200))
        a[w], b[w] = -0.5 + 1e-13, 0.5 - 1e-13
        a[1 - w] = b[1 - w] = s
        pairs.append((E @ a, E @ b))
    trg = np.concatenate([x for pr in pairs for x in pr], axis=1)
    u, _, _ = run_lib("mstokes", e1, e2, src, f, trg, beta=1.0, tol=tol, precision=precision, grad=False)
    u = u[0]
    for k in range(2):
        ua, ub = u[:, 400 * k:400 * k + 200], u[:, 400 * k + 200:400 * k + 400]
        assert np.linalg.norm(ua - ub) / np.linalg.norm(u) < 2 * tol


@pytest.mark.parametrize("precision,self_t", [("mixed", False), ("fp64", False), ("mixed", True)])
def test_batch(precision, self_t):
    """Four cells of different shape and beta in one batch (mixed: the
    persistent batched P2P; separate targets or targets = sources) against
    the oracle cell by cell."""
    import torch
    from paper_2111_01083_gb300 import BatchOp
    rng = np.random.default_rng(75)
    specs = [(LAT["square"], 0.7), (LAT["hex"], 2.0), (LAT["rect8"], 1.0), (LAT["rotated"], 4.0)]
    cells, srcs, fs, trgs = [], [], [], []
    for (e1, e2), beta in specs:
        n = int(rng.integers(200, 700))
        srcs.append(workloads.points(rng, e1, e2, n))
        fs.append(rng.standard_normal((2, 2, n)))
        trgs.append(srcs[-1] if self_t else workloads.points(rng, e1, e2, int(rng.integers(100, 400))))
        cells.append(dict(e1=e1, e2=e2, beta=beta))
    dev = torch.device("cuda", 0)
    S = torch.tensor(np.concatenate(srcs, axis=1), device=dev)
    Q = torch.tensor(np.concatenate(fs, axis=-1), device=dev)
    T = None if self_t else torch.tensor(np.concatenate(trgs, axis=1), device=dev)
    tol = TOL[precision]
    op = BatchOp("mstokes", cells, [s.shape[1] for s in srcs], None if self_t else [t.shape[1] for t in trgs],
                 precision=precision, nrhs=2, tol=tol)
    vel, _ = op(S, Q, T, grad=False)
    torch.cuda.synchronize()
    op.status(dev)
    vel = vel.cpu().numpy()
    o = 0
    for ((e1, e2), beta), s_, f_, t_ in zip(specs, srcs, fs, trgs):
        n = t_.shape[1]
        ref = oracle("mstokes", e1, e2, s_, f_, None if self_t else t_, beta=beta, how="plain", grad=False)
        assert _err(vel[:, :, o:o + n], ref[0]) < tol
        o += n


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("beta", [0.5, 3.0])
@pytest.mark.parametrize("e1,e2", [((40.0, 0.0), (0.0, 1.0)), ((48.0, 0.0), (0.5, 1.0))])
def test_nufft_path(precision, beta, e1, e2):
    """Long cells on the NUFFT south/north path (both plane-wave families from
    one spread), west/east on the direct kernels."""
    rng = np.random.default_rng(76)
    src = workloads.points(rng, e1, e2, 900)
    f = rng.standard_normal((2, 2, 900))
    trg = workloads.points(rng, e1, e2, 400)
    got = run_lib("mstokes", e1, e2, src, f, trg, beta=beta, tol=TOL[precision], precision=precision, grad=False,
                  path="nufft")
    assert got[2].describe()["path"] == 2
    ref = oracle("mstokes", e1, e2, src, f, trg, beta=beta, how="plain", grad=False)
    assert _err(got[0], ref[0]) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nufft_matches_direct(precision):
    e1, e2 = (24.0, 0.0), (0.2, 1.0)
    rng = np.random.default_rng(77)
    src = workloads.points(rng, e1, e2, 3000, "gmm")
    f = rng.standard_normal((1, 2, 3000))
    a = run_lib("mstokes", e1, e2, src, f, None, beta=1.0, tol=TOL[precision], precision=precision, grad=False,
                path="nufft")
    b = run_lib("mstokes", e1, e2, src, f, None, beta=1.0, tol=TOL[precision], precision=precision, grad=False,
                path="direct")
    assert _err(a[0], b[0]) < TOL[precision]


@pytest.mark.parametrize("self_t", [False, True])
def test_adjoint_strengths(self_t):
    """dL/df for L = sum w . u through periodic() (pfmm_execute_adjoint): the
    operator is symmetric, so dL/df_j = (P w)(s_j), the velocity at the
    sources of forces w at the targets, checked against the oracle."""
    import torch
    from paper_2111_01083_gb300 import PeriodicOp, periodic
    e1, e2 = LAT["hex"]
    rng = np.random.default_rng(78)
    ns, nt = 400, 250
    src = workloads.points(rng, e1, e2, ns)
    trg = src if self_t else workloads.points(rng, e1, e2, nt)
    nt = trg.shape[1]
    f = rng.standard_normal((1, 2, ns))
    w = rng.standard_normal((1, 2, nt))
    dev = torch.device("cuda", 0)
    S = torch.tensor(src, device=dev)
    T = None if self_t else torch.tensor(trg, device=dev)
    F = torch.tensor(f, device=dev, requires_grad=True)
    n = max(ns, nt)
    op = PeriodicOp("mstokes", e1, e2, beta=1.3, tol=1e-10, precision="fp64", ns_max=n, nt_max=n)
    vel = periodic(op, S, F, T)
    (torch.tensor(w, device=dev) * vel).sum().backward()
    ref, _ = oracle("mstokes", e1, e2, trg, w, None if self_t else src, beta=1.3, how="plain", grad=False)
    assert _err(F.grad.detach().cpu().numpy(), ref) < 1e-10
