"""GPU parity of the rotated west/east plane-wave direction (App. A, Eq.
k0west2): plane waves decaying along e2-perp, so the near block is 3 x 3
images on every parallelogram.  The CUDA library (through the C ABI) against
the FP64 oracle on the hexagonal cell (where the axis direction needs a
5 x 3 block), a tilted hexagonal cell, a skewed cell and a long sheared cell
on the NUFFT path; both directions, both precisions, the parts (far / near)
and the batch.

Tolerances as in test_gpu_parity: FP64 1e-10, mixed 1e-6 (relative l2;
Laplace potentials and Stokes velocities modulo the best-fit constant).
"""
import math

import numpy as np
import pytest

import workloads
from gpu_util import errs, oracle, run_lib

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}
_A = 0.4
LAT = {
    "hex": ((1.0, 0.0), (0.5, math.sqrt(3) / 2)),
    "hex_tilted": ((math.cos(_A), math.sin(_A)), (math.cos(_A + math.pi / 3), math.sin(_A + math.pi / 3))),
    "skew": ((1.0, 0.0), (0.3, 0.8)),
    "long_sheared": ((16.0, 0.0), (0.03, 1.0)),
}
KERNELS = [("laplace", 0.0), ("modhelm", 2.0), ("stokes", 0.0)]


def _case(kernel, lat, ns, nt=None, seed=0, dist="uniform", nrhs=1):
    e1, e2 = LAT[lat]
    rng = np.random.default_rng(seed)
    src = workloads.points(rng, e1, e2, ns, dist)
    q = workloads.strengths(rng, nrhs, ns, stokes=kernel == "stokes", neutral=kernel != "modhelm")
    trg = None if nt is None else workloads.points(rng, e1, e2, nt)
    return e1, e2, src, q, trg


def _check(kernel, got, ref, tol):
    ep, eg = errs(kernel, got, ref)
    assert ep < tol, ep
    if eg is not None:
        assert eg < tol, eg


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("we", ["rotated", "axis"])
@pytest.mark.parametrize("kernel,beta", KERNELS)
def test_hex_total(precision, we, kernel, beta):
    st = kernel == "stokes"
    e1, e2, src, q, trg = _case(kernel, "hex", 800, nt=331 if st else None, seed=50, nrhs=2)
    got = run_lib(kernel, e1, e2, src, q, trg, beta=beta, tol=TOL[precision], precision=precision, grad=not st,
                  we=we)
    desc = got[2].describe()
    assert (desc["m0"], desc["we_rotated"]) == ((1, 1) if we == "rotated" else (2, 0))
    ref = oracle(kernel, e1, e2, src, q, trg, beta=beta, grad=not st, we=we)
    _check(kernel, got, ref, TOL[precision])


@pytest.mark.parametrize("lat", ["hex", "skew"])
@pytest.mark.parametrize("part", ["far", "near"])
@pytest.mark.parametrize("kernel,beta", KERNELS)
def test_rotated_parts_fp64(lat, part, kernel, beta):
    """The near/far split follows the rotated frame's 3 x 3 block."""
    st = kernel == "stokes"
    e1, e2, src, q, trg = _case(kernel, lat, 400, nt=257, seed=51)
    got = run_lib(kernel, e1, e2, src, q, trg, beta=beta, tol=1e-10, precision="fp64", part=part, grad=not st,
                  we="rotated")
    ref = oracle(kernel, e1, e2, src, q, trg, beta=beta, part=part, grad=not st, we="rotated")
    _check(kernel, got, ref, 1e-10 if part == "near" else 1e-9)


@pytest.mark.parametrize("kernel,beta", KERNELS)
def test_tilted_hex_mixed_clustered(kernel, beta):
    """Default direction (rotated on a hexagonal lattice in any orientation),
    clustered points spanning several P2P tiles with a ragged tail."""
    st = kernel == "stokes"
    e1, e2, src, q, trg = _case(kernel, "hex_tilted", 1500, nt=701, seed=52, dist="gmm")
    got = run_lib(kernel, e1, e2, src, q, trg, beta=beta, tol=1e-6, precision="mixed", grad=not st)
    assert got[2].describe()["we_rotated"] == 1
    ref = oracle(kernel, e1, e2, src, q, trg, beta=beta, grad=not st)
    _check(kernel, got, ref, 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kernel,beta", KERNELS)
def test_long_sheared_nufft_rotated(precision, kernel, beta):
    """A sheared 16 x 1 cell with the rotated direction forced (the image
    columns shift y~ by d xi/|e2| = 0.48 per step: complex column ratio) and
    the NUFFT south/north path.  (A reduced cell with |xi| > 3d/8 has
    eta > 0.7 d, so the default never rotates a long cell.)"""
    st = kernel == "stokes"
    e1, e2, src, q, trg = _case(kernel, "long_sheared", 900, nt=400, seed=53)
    got = run_lib(kernel, e1, e2, src, q, trg, beta=beta, tol=TOL[precision], precision=precision, grad=not st,
                  path="nufft", we="rotated")
    desc = got[2].describe()
    assert desc["path"] == 2 and desc["we_rotated"] == 1 and desc["m0"] == 1
    assert abs(desc["we_dir"][1]) > 0.02
    ref = oracle(kernel, e1, e2, src, q, trg, beta=beta, grad=not st, we="rotated")
    _check(kernel, got, ref, TOL[precision])


def test_batch_mixes_directions():
    """A batch with rotated (hexagonal, default and forced) and axis cells."""
    import torch
    from paper_2111_01083_gb300 import BatchOp
    rng = np.random.default_rng(54)
    kernel, beta = "modhelm", 3.0
    specs = [(LAT["hex"], "auto"), (LAT["skew"], "rotated"), (LAT["hex_tilted"], "axis"), (LAT["skew"], "auto")]
    cells, srcs, qs = [], [], []
    for (e1, e2), we in specs:
        n = int(rng.integers(300, 900))
        srcs.append(workloads.points(rng, e1, e2, n))
        qs.append(workloads.strengths(rng, 1, n))
        cells.append(dict(e1=e1, e2=e2, beta=beta, we=we))
    dev = torch.device("cuda", 0)
    S = torch.tensor(np.concatenate(srcs, axis=1), device=dev)
    Q = torch.tensor(np.concatenate(qs, axis=-1), device=dev)
    op = BatchOp(kernel, cells, [s.shape[1] for s in srcs], precision="mixed", nrhs=1, tol=1e-6)
    pot, grad = op(S, Q, None, grad=True)
    torch.cuda.synchronize()
    op.status(dev)
    pot, grad = pot.cpu().numpy(), grad.cpu().numpy()
    o = 0
    for ((e1, e2), we), src, q in zip(specs, srcs, qs):
        n = src.shape[1]
        ref = oracle(kernel, e1, e2, src, q, None, beta=beta, we=we)
        _check(kernel, (pot[:, o:o + n], grad[:, :, o:o + n]), ref, 1e-6)
        o += n
