"""The multi-rank path of bench.py on CPU (gloo, world size 2): each rank
times its own independent cell (no collective on the data path); the job time
is the max over ranks and the whole-job value counts every rank's units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    import bench
    dev = torch.device("cpu")
    d = bench.init_dist(world, dev)
    try:
        local_s = [0.25, 0.5][rank]  # rank 1 is the slow one
        t = bench.max_over_ranks(d, local_s, dev)
        d.barrier()
        out[rank] = (t, bench.job_value(world, 1000, t))
    finally:
        d.destroy_process_group()


def test_two_ranks_max_time_and_job_value():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    for r in range(2):
        t, v = res[r]
        assert t == 0.5  # the job ends when the slowest rank does
        assert v == pytest.approx(2 * 1000 / 0.5)


def test_single_rank_has_no_process_group():
    import bench
    assert bench.init_dist(1, torch.device("cpu")) is None
    assert bench.max_over_ranks(None, 0.3, torch.device("cpu")) == 0.3
