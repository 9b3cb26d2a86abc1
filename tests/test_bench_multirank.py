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


def _distinct_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(rank)
    D = rng.integers(-3, 4, size=(500, 40)).astype(np.int8)
    shared = np.arange(40, dtype=np.int8)[None, :].repeat(20, 0) + np.arange(20, dtype=np.int8)[:, None]
    D[:20] = shared                      # the same 20 rows on both ranks
    out.put((rank, bench.distinct_over_ranks(bench.row_hashes(D), world)))
    dist.destroy_process_group()


def test_distinct_directions_over_two_gloo_ranks():
    """The union of the replicas' direction sets counts rows found by both
    ranks once: 2 x 500 rows with 20 in common (and no other collisions)."""
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_distinct_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results[0][1] == (980, 1000) and results[1][1] == (980, 1000)


def test_row_hashes_are_content_hashes():
    import numpy as np

    import bench
    D = np.array([[1, 2, 3], [1, 2, 3], [3, 2, 1], [-1, 0, 0]], dtype=np.int8)
    h = bench.row_hashes(D)
    assert h[0] == h[1] and len(set(h.tolist())) == 3
