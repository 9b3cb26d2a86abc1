"""The N > 1 path of bench.py with two gloo ranks on CPU: every rank runs its
own replica, the job sums the verified directions and takes the max of the
device times (weak scaling, no data-path collective)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, ms = bench.reduce_over_ranks(1000 * (rank + 1), 10.0 * (rank + 1), world)
    bench.barrier(world)
    out.put((rank, units, ms))
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results == [(0, 3000.0, 20.0), (1, 3000.0, 20.0)]


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(5, 7.5, 1) == (5.0, 7.5)


def test_dist_env_defaults(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
