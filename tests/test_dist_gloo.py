"""The N>1 path of bench.py on CPU: two gloo ranks combine their timings."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2406_18109_gb300 import dist as D  # noqa: E402


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank               # rank 1 is the slowest
        units = 1000.0 * (rank + 1)
        q.put((rank, D.combine(ms, units), D.rank_seed(1, rank)))
    finally:
        dist.destroy_process_group()


def test_two_rank_weak_scaling_combination():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 500)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, (value, ms, units), seed in out:
        assert ms == 15.0 and units == 3000.0
        assert abs(value - 3000.0 / 0.015) < 1e-6
    assert out[0][2] == 1 and out[1][2] != 1


def test_single_process_combination():
    v, ms, u = D.combine(20.0, 500.0)
    assert ms == 20.0 and u == 500.0 and abs(v - 25000.0) < 1e-9
