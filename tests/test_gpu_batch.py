"""Batched execution (many cells in one call): parity with the single-cell path
(itself checked against the oracle) and, for two cells, with the oracle
directly; CUDA-graph capture and replay; the chunk-size autotuner."""
import math

import numpy as np
import pytest

import workloads
from gpu_util import errs, oracle, run_lib
from oracle import api as oapi

pytestmark = pytest.mark.gpu


def _cells(ncell, seed, kernel, nmin, nmax, amax, betas=(1.0,), skew=False, nrhs=1):
    rng = np.random.default_rng(seed)
    cells, srcs, qs = [], [], []
    for i in range(ncell):
        A = math.exp(rng.uniform(0, math.log(amax)))
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        e1, e2 = (A, 0.0), ((0.3 * A if skew and i % 2 else 0.0), 1.0)
        src = workloads.points(rng, e1, e2, n)
        q = workloads.strengths(rng, nrhs, n, stokes=kernel == "stokes", neutral=kernel != "modhelm")
        cells.append(dict(e1=e1, e2=e2, beta=betas[i % len(betas)]))
        srcs.append(src)
        qs.append(q)
    return cells, srcs, qs


def _run_batch(kernel, cells, srcs, qs, precision, tol, nrhs, trgs=None, p2p_chunk=0, graph=False):
    import torch
    from paper_2111_01083_gb300 import BatchOp
    dev = torch.device("cuda", 0)
    S = torch.tensor(np.concatenate(srcs, axis=1), device=dev)
    Q = torch.tensor(np.concatenate(qs, axis=-1), device=dev)
    T = None if trgs is None else torch.tensor(np.concatenate(trgs, axis=1), device=dev)
    op = BatchOp(kernel, cells, [s.shape[1] for s in srcs], None if trgs is None else [t.shape[1] for t in trgs],
                 precision=precision, nrhs=nrhs, tol=tol, p2p_chunk=p2p_chunk)
    grad = kernel != "stokes"
    if graph:
        g, out = op.capture(S, Q, T, grad=grad)
        for o in out:
            if o is not None:
                o.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
    else:
        out = op(S, Q, T, grad=grad)
        torch.cuda.synchronize()
    op.status(dev)
    pot = out[0].cpu().numpy()
    gr = None if out[1] is None else out[1].cpu().numpy()
    return pot, gr


def _split(arr, counts):
    edges = np.concatenate([[0], np.cumsum(counts)])
    return [arr[..., edges[i]:edges[i + 1]] for i in range(len(counts))]


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-6), ("fp64", 1e-10)])
def test_batch_modhelm_matches_single(precision, tol):
    cells, srcs, qs = _cells(10, 3, "modhelm", 150, 900, 8.0, betas=(1.0, 10.0, 3.0), skew=True, nrhs=4)
    pot, gr = _run_batch("modhelm", cells, srcs, qs, precision, tol, 4, p2p_chunk=256)
    counts = [s.shape[1] for s in srcs]
    for c, (p, g) in enumerate(zip(_split(pot, counts), _split(gr, counts))):
        ref = run_lib("modhelm", cells[c]["e1"], cells[c]["e2"], srcs[c], qs[c], None, beta=cells[c]["beta"],
                      tol=tol, precision=precision)
        ep, eg = errs("modhelm", (p, g), ref)
        assert ep < tol and eg < tol, (c, ep, eg)
    # two cells against the oracle itself
    for c in (0, 1):
        ref = oracle("modhelm", cells[c]["e1"], cells[c]["e2"], srcs[c], qs[c], None, beta=cells[c]["beta"])
        ep, eg = errs("modhelm", (_split(pot, counts)[c], _split(gr, counts)[c]), ref)
        assert ep < tol and eg < tol, (c, ep, eg)


@pytest.mark.parametrize("kernel", ["laplace", "stokes"])
def test_batch_separate_targets_mixed(kernel):
    cells, srcs, qs = _cells(7, 5, kernel, 200, 700, 6.0, skew=True, nrhs=2)
    rng = np.random.default_rng(9)
    trgs = [workloads.points(rng, c["e1"], c["e2"], int(rng.integers(50, 400))) for c in cells]
    pot, gr = _run_batch(kernel, cells, srcs, qs, "mixed", 1e-6, 2, trgs=trgs)
    counts = [t.shape[1] for t in trgs]
    pots = _split(pot, counts)
    grs = _split(gr, counts) if gr is not None else [None] * len(counts)
    for c in range(len(cells)):
        ref = oracle(kernel, cells[c]["e1"], cells[c]["e2"], srcs[c], qs[c], trgs[c], grad=kernel != "stokes")
        ep, eg = errs(kernel, (pots[c], grs[c]), ref)
        assert ep < 1e-6, (c, ep)
        if eg is not None:
            assert eg < 1e-6, (c, eg)


@pytest.mark.parametrize("kernel", ["modhelm", "stokes"])
def test_batch_mixes_nufft_and_direct_cells(kernel):
    """Wide cells (M >= 64) take the NUFFT south/north path inside a batch next
    to square ones on the direct path; graph replay against the oracle."""
    import torch
    from paper_2111_01083_gb300 import PeriodicOp
    rng = np.random.default_rng(21)
    beta = 0.5 if kernel == "modhelm" else 0.0
    shapes = [((48.0, 0.0), (0.0, 1.0)), ((1.0, 0.0), (0.2, 1.0)), ((64.0, 0.0), (0.3, 1.0)), ((2.0, 0.0), (0.0, 1.0))]
    cells, srcs, qs = [], [], []
    for e1, e2 in shapes:
        n = int(rng.integers(300, 900))
        srcs.append(workloads.points(rng, e1, e2, n, "gmm"))
        qs.append(workloads.strengths(rng, 2, n, stokes=kernel == "stokes", neutral=kernel != "modhelm"))
        cells.append(dict(e1=e1, e2=e2, beta=beta))
    paths = [PeriodicOp(kernel, c["e1"], c["e2"], beta=beta, tol=1e-6, precision="mixed", nrhs=2, ns_max=10,
                        nt_max=10).describe()["path"] for c in cells]
    assert paths == [2, 1, 2, 1]
    pot, gr = _run_batch(kernel, cells, srcs, qs, "mixed", 1e-6, 2, graph=True)
    counts = [s.shape[1] for s in srcs]
    pots = _split(pot, counts)
    grs = _split(gr, counts) if gr is not None else [None] * len(counts)
    for c in range(len(cells)):
        ref = oracle(kernel, cells[c]["e1"], cells[c]["e2"], srcs[c], qs[c], None, beta=beta,
                     grad=kernel != "stokes")
        ep, eg = errs(kernel, (pots[c], grs[c]), ref)
        assert ep < 1e-6, (c, ep)
        if eg is not None:
            assert eg < 1e-6, (c, eg)


def test_batch_graph_replay_matches_eager():
    cells, srcs, qs = _cells(6, 7, "modhelm", 300, 1200, 16.0, betas=(1.0, 10.0), nrhs=8)
    a = _run_batch("modhelm", cells, srcs, qs, "mixed", 1e-6, 8, p2p_chunk=512)
    b = _run_batch("modhelm", cells, srcs, qs, "mixed", 1e-6, 8, p2p_chunk=512, graph=True)
    assert np.all(np.isfinite(b[0]))
    assert np.linalg.norm(a[0] - b[0]) / np.linalg.norm(a[0]) < 1e-12
    assert np.linalg.norm(a[1] - b[1]) / np.linalg.norm(a[1]) < 1e-12


def test_autotune_picks_a_candidate(tmp_path):
    import torch
    from paper_2111_01083_gb300 import BatchOp, autotune_batch
    cells, srcs, qs = _cells(5, 8, "modhelm", 400, 1500, 4.0, nrhs=1)
    dev = torch.device("cuda", 0)
    S = torch.tensor(np.concatenate(srcs, axis=1), device=dev)
    Q = torch.tensor(np.concatenate(qs, axis=-1), device=dev)
    counts = [s.shape[1] for s in srcs]
    mk = lambda c: BatchOp("modhelm", cells, counts, precision="mixed", nrhs=1, p2p_chunk=c)
    cache = str(tmp_path / "tune.json")
    best, times = autotune_batch(mk, S, Q, candidates=(256, 1024), cache=cache, key="k")
    assert best in (256, 1024) and len(times) == 2
    best2, _ = autotune_batch(mk, S, Q, candidates=(256, 1024), cache=cache, key="k")
    assert best2 == best


def test_tune_batch_crossover_width_chunk(tmp_path):
    """tune_batch picks the direct/NUFFT crossover, the ES width (only widths
    whose bound meets the tolerance) and the P2P chunk by graph-replay time;
    the tuned batch is the fastest configuration it timed, matches the oracle
    at 1e-6 on sampled cells, and the cached choice is returned unchanged."""
    import torch
    from paper_2111_01083_gb300 import tune_batch, tuned_batch
    rng = np.random.default_rng(12)
    cells, srcs, qs = [], [], []
    for A in (1.0, 3.0, 20.0, 40.0, 64.0, 64.0):
        n = int(rng.integers(800, 3000))
        e1, e2 = (A, 0.0), (0.0, 1.0)
        cells.append(dict(e1=e1, e2=e2, beta=1.0))
        srcs.append(workloads.points(rng, e1, e2, n))
        qs.append(rng.standard_normal((8, n)))
    counts = [s.shape[1] for s in srcs]
    dev = torch.device("cuda", 0)
    S = torch.tensor(np.concatenate(srcs, axis=1), device=dev)
    Q = torch.tensor(np.concatenate(qs, axis=-1), device=dev)
    cache = str(tmp_path / "tune.json")
    cfg, times = tune_batch("modhelm", cells, counts, S, Q, nrhs=8, tol=1e-6, chunks=(1024, 4096),
                            crossovers=(64, 128, None), reps=2, cache=cache, key="k")
    assert cfg["nufft_w"] in (7, 8) and cfg["p2p_chunk"] in (1024, 4096) and cfg["crossover"] in (64, 128, None)
    import json
    assert times[json.dumps(cfg, sort_keys=True)] == min(times.values())
    cfg2, _ = tune_batch("modhelm", cells, counts, S, Q, nrhs=8, tol=1e-6, cache=cache, key="k")
    assert cfg2 == cfg
    op = tuned_batch("modhelm", cells, counts, cfg, nrhs=8, tol=1e-6)
    pot, _ = op(S, Q, grad=False)
    torch.cuda.synchronize()
    op.status(dev)
    pot = pot.cpu().numpy()
    edges = np.concatenate([[0], np.cumsum(counts)])
    for c in (1, 4):
        idx = rng.choice(counts[c], 40, replace=False)
        ref, _ = oracle("modhelm", cells[c]["e1"], cells[c]["e2"], srcs[c], qs[c], srcs[c][:, idx], beta=1.0, grad=False)
        got = pot[:, edges[c]:edges[c + 1]][:, idx]
        assert oapi.rel_err(got, ref) < 1e-6
