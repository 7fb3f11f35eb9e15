"""The bench's multi-rank path (replicas only: no collective on the data
path) on CPU with two gloo ranks: the whole-job aggregate takes the slowest
rank's time and sums the ranks' iteration counts."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = 10.0 + 5.0 * rank
    res = bench.reduce_over_ranks(t, [6 + rank, 100 * (rank + 1)], world)
    out.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        t_all, counts = got[r]
        assert t_all == 15.0
        assert counts == [13.0, 300.0]


def test_single_rank_passes_through():
    import bench
    assert bench.reduce_over_ranks(2.5, [3, 4], 1) == (2.5, [3.0, 4.0])
