"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): each
rank generates its own batch from a rank-dependent seed (weak scaling, no
data-path collective), and the reported time is the maximum over ranks while
the cell count is the sum."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    probs, desc = bench.make_workload("batched", rank=rank, processes=1, grids=2)
    cells = sum(p.ncells for p in probs)
    ms, total = bench.reduce_over_ranks(10.0 + rank, cells, "cpu")
    out[rank] = (ms, total, cells, desc, probs[0].U0[0, 0, 0, 0, 0])
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_reduction():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (ms0, tot0, c0, d0, v0), (ms1, tot1, c1, d1, v1) = out[0], out[1]
    assert ms0 == ms1 == 11.0                      # max over ranks
    assert tot0 == tot1 == c0 + c1                 # cells of both ranks
    assert d0 != d1 and v0 != v1                   # different seeds per rank
