"""The bench's multi-rank path (replicas only: no collective on the data
path) on CPU with two gloo ranks: the whole-job aggregate takes the slowest
rank's time and sums the ranks' iteration counts.  The oracle (reference)
arm prints its one line on rank 0 only."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

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


def _bench(env_extra, *args):
    import subprocess
    import sys
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True,
                          text=True, env=env, timeout=600)


def test_reference_arm_prints_one_line_on_rank_zero_only():
    """The oracle arm under a multi-rank launch: ranks other than 0 exit 0
    without work or output; rank 0 prints one JSON line with the contract's
    keys and a one-core CPU baseline of the same sample."""
    import json
    quiet = _bench({"RANK": "1", "WORLD_SIZE": "2"}, "--impl", "reference", "--gpus", "2", "--steps", "1",
                   "--warmup", "0")
    assert quiet.returncode == 0 and quiet.stdout.strip() == ""
    r = _bench({"RANK": "0", "WORLD_SIZE": "1"}, "--impl", "reference", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == 1 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert line["config"]["workload"] == "mcc3d_2M"
