"""a10 over many candidate sets at once (mape_dedup_batch): every set's
distinct rows, in order, are those of its own mape_dedup and of the oracle's
sorted np.unique; sets of different widths and sizes (empty, one row, sets
that need the global bitonic stages, sets with runs of equal sort keys and
one run longer than a block sorts), and a set whose distinct rows exceed its
output capacity (status CAPACITY, K still counted, the other sets unharmed).
Also the handle batch, whose chunk merges go through it (tests/test_gpu_batch.py
covers its results)."""
import numpy as np
import pytest

from oracle import mape_oracle as O

from .gpu_common import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    return mape


def _set(M, rng, count, n, distinct, prefix_groups=None):
    """count rows drawn from `distinct` random rows of width n (entries in
    [-4, 4]); prefix_groups: the first 8 bytes from that many patterns."""
    ldc = M.round16(n)
    base = rng.integers(-4, 5, size=(max(1, distinct), n))
    if prefix_groups:
        k = min(8, n)
        base[:, :k] = rng.integers(-3, 4, size=(prefix_groups, k))[rng.integers(0, prefix_groups, size=base.shape[0])]
    rows = base[rng.integers(0, base.shape[0], size=count)].astype(np.int8)
    buf = np.zeros((max(count, 1), ldc), np.int8)
    buf[:count, :n] = rows
    return rows, dev(buf)


def test_dedup_batch_equals_single_and_oracle(M):
    rng = np.random.default_rng(77)
    specs = [(0, 20, 1, None), (1, 20, 1, None), (37, 8, 10, None), (3000, 40, 900, None),
             (20000, 64, 9000, None), (6000, 40, 2000, 1), (20000, 64, 7000, 300), (3000, 208, 800, 5),
             (500, 2000, 200, None)]
    sets, rows_all = [], []
    for count, n, distinct, groups in specs:
        rows, buf = _set(M, rng, count, n, distinct, groups)
        sets.append((buf, count, n, None))
        rows_all.append(rows)
    out = M.dedup_batch(sets)
    for (buf, count, n, _), rows, (uniq, K, status) in zip(sets, rows_all, out):
        assert status == 0
        expect = O.sort_directions(np.unique(rows.astype(np.int64), axis=0)) if count else np.zeros((0, n), np.int64)
        got = uniq.cpu().numpy()
        assert K == expect.shape[0]
        assert np.array_equal(got[:, :n].astype(np.int64), expect)
        assert np.all(got[:, n:] == 0)
        if count:
            single = M.dedup(buf, count, n).cpu().numpy()
            assert np.array_equal(single, got)


def test_dedup_batch_capacity_per_set(M):
    rng = np.random.default_rng(78)
    rows_a, a = _set(M, rng, 1000, 24, 300)
    rows_b, b = _set(M, rng, 2000, 24, 700)
    distinct_b = np.unique(rows_b.astype(np.int64), axis=0).shape[0]
    out = M.dedup_batch([(a, 1000, 24, None), (b, 2000, 24, distinct_b - 1)])
    (ua, Ka, sa), (ub, Kb, sb) = out
    assert sa == 0 and sb == -7 and Kb == distinct_b and ub.shape[0] == 0
    expect = O.sort_directions(np.unique(rows_a.astype(np.int64), axis=0))
    assert np.array_equal(ua.cpu().numpy()[:, :24].astype(np.int64), expect)
