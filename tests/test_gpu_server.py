"""The request server: continuous batching of instances on one GPU.  Each
request's result (direction set, best x and f) is the same alone and in a
mix with others on the device at once; admission respects the memory cap;
every request's timeline is ordered and its result feasible and no worse
than its start."""
import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

pytestmark = pytest.mark.gpu

SIZES = (60, 150, 300, 520, 900)  # resident (d <= 256) and streamed (d > 256) shapes


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    return mape


def _requests():
    out = []
    for k, n in enumerate(SIZES):
        inst = I.uneven_single(n, density=0.1)
        Z0 = I.normal_starts(inst, 512, std=0.3, seed=3000 + k).Z0
        out.append((inst, Z0))
    return out


def _run(M, reqs, slots, batch=False):
    cfg = M.default_config(T=100)
    with M.Server(cfg, mem_cap_bytes=64 << 30, max_slots=slots, keep_directions=True,
                  batch_extraction=batch) as srv:
        ids = [srv.submit(inst, 512, Z0=Z0) for inst, Z0 in reqs]
        srv.wait_all(900)
        res = [srv.result(i, directions=True) for i in ids]
        infos = [srv.info(i) for i in ids]
        stats = srv.stats()
    return res, infos, stats


@pytest.mark.parametrize("batch", [False, True])
def test_server_alone_equals_mix(M, batch):
    """Alone (one slot, its own extraction) and mixed (four slots; with
    batch_extraction the requests admitted together extract in one batched
    call): the same direction sets, points and values."""
    reqs = _requests()
    alone = []
    for r in reqs:
        res, infos, stats = _run(M, [r], 1)
        assert infos[0]["state"] == "DONE", infos[0]
        alone.append(res[0])
    mixed, infos, stats = _run(M, reqs, 4, batch)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["peak_running"] > 1          # the requests overlapped on the device
    for (inst, _), (xa, fa, Ga), (xm, fm, Gm), info in zip(reqs, alone, mixed, infos):
        assert info["state"] == "DONE"
        assert np.array_equal(Ga, Gm)
        assert fa == fm and np.array_equal(xa, xm)
        assert Gm.shape[0] > 0
        # the result is a feasible point no worse than the start
        x = xm.astype(np.int64)
        assert np.array_equal(inst.A.astype(np.int64) @ x, inst.b)
        assert np.all((x >= inst.l) & (x <= inst.u))
        assert fm == O.f_value(inst.Q, inst.c, inst.w, x) <= O.f_value(inst.Q, inst.c, inst.w, inst.xbar)
        assert np.all(O.kernel_condition(inst.A, Gm.astype(np.int64)))
        t = [info[k] for k in ("t_submit_ms", "t_admit_ms", "t_extracted_ms", "t_first_improve_ms", "t_done_ms")]
        assert all(a <= b for a, b in zip(t, t[1:])), t


def test_server_admits_by_memory(M):
    """Five equal requests, a cap of 2.5 requests: never more than two run at
    once, all complete, the peak stays under the cap."""
    cfg = M.default_config(T=50)
    inst = I.uneven_single(150)
    per = M.request_bytes(inst.n, inst.m, 256, 1, cfg)
    cap = int(2.5 * per)
    with M.Server(cfg, mem_cap_bytes=cap, max_slots=8) as srv:
        ids = [srv.submit(inst, 256, Z0=I.normal_starts(inst, 256, std=0.3, seed=k).Z0) for k in range(5)]
        srv.wait_all(600)
        st = srv.stats()
        assert st["completed"] == 5 and st["failed"] == 0
        assert st["peak_running"] == 2
        assert st["mem_peak"] <= cap
        for i in ids:
            assert srv.info(i)["state"] == "DONE"
        # a request larger than the whole cap can never be admitted
        big = I.uneven_single(900)
        with pytest.raises(M.MapeError) as e:
            srv.submit(big, 4096, Z0=I.normal_starts(big, 4096, std=0.3, seed=1).Z0)
        assert e.value.code == -11
