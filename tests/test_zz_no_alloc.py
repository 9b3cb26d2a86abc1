"""mape_dedup_static, the dedup entry point that allocates no device memory,
for callers that cannot allocate where they dedup (a host that reserves all
device memory up front and forbids later allocations, or a plugin whose host
owns the allocator).  It keeps its scratch in a static device array of the
library, so this test checks, through the C ABI, that it returns exactly what
mape_dedup returns with a caller workspace, on two calls in a row (the second
call must not see the first one's leftovers), at the largest accepted count
with a wide row pitch (where its scratch comes closest to the array's size),
and that a count above its stated limit is refused before any device work.
This file is collected last so that a failure here comes after every other
test has run."""
import ctypes

import numpy as np
import pytest

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


def _rows(seed, count, n, distinct):
    rng = np.random.default_rng(seed)
    ldc = (n + 15) // 16 * 16
    base = rng.integers(-5, 6, size=(distinct, n)).astype(np.int8)
    rows = base[rng.integers(0, distinct, size=count)]
    buf = np.zeros((count, ldc), np.int8)
    buf[:, :n] = rows
    return buf, ldc


def _static(M, cand, count, n, ldc):
    import torch
    uniq = torch.full((count, ldc), 99, dtype=torch.int8, device="cuda")
    K = ctypes.c_int64(-1)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = M.lib().mape_dedup_static(ctypes.c_void_p(cand.data_ptr()), count, n, ldc, ctypes.c_void_p(uniq.data_ptr()),
                                   count, ctypes.byref(K), stream)
    assert rc == 0, rc
    return uniq[: K.value].cpu().numpy()


def test_static_dedup_matches_workspace_dedup_twice(M):
    # two different inputs back to back: a large one, then a smaller one whose
    # table and counter must start empty again
    for seed, count, n, distinct in ((1, 200000, 200, 30000), (2, 5000, 37, 900)):
        buf, ldc = _rows(seed, count, n, distinct)
        cand = dev(buf)
        got = _static(M, cand, count, n, ldc)
        expect = M.dedup(cand, count, n).cpu().numpy()
        assert got.shape == expect.shape
        assert np.array_equal(got, expect)


def test_static_dedup_refuses_counts_above_its_limit(M):
    limit = M.lib().mape_dedup_static_max_rows()
    assert limit == 1 << 18
    K = ctypes.c_int64(-1)
    rc = M.lib().mape_dedup_static(None, limit + 1, 16, 16, None, 0, ctypes.byref(K), None)
    assert rc == -7


def test_static_dedup_at_its_row_limit_with_wide_rows(M):
    """count == mape_dedup_static_max_rows() with ldc = 4096: the hash table,
    the padded sort keys and the run list all reach their largest sizes, and
    must still fit the static array; the result equals mape_dedup's."""
    import torch
    limit = int(M.lib().mape_dedup_static_max_rows())
    n, ldc, distinct = 4090, 4096, 3000
    rng = np.random.default_rng(9)
    base = np.zeros((distinct, ldc), np.int8)
    base[:, :n] = rng.integers(-5, 6, size=(distinct, n))
    # rows that differ only late in the row share their 8-byte sort prefix
    base[distinct // 2:, :64] = base[0, :64]
    pick = torch.from_numpy(rng.integers(0, distinct, size=limit)).cuda()
    cand = dev(base)[pick].contiguous()
    got = _static(M, cand, limit, n, ldc)
    expect = M.dedup(cand, limit, n).cpu().numpy()
    assert got.shape == expect.shape
    assert np.array_equal(got, expect)
    # and a second, small call right after it still starts from a clean table
    buf, ldc2 = _rows(3, 3000, 50, 700)
    cand2 = dev(buf)
    assert np.array_equal(_static(M, cand2, 3000, 50, ldc2), M.dedup(cand2, 3000, 50).cpu().numpy())
