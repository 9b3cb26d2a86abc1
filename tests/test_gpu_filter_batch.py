"""The filter stages over many instances at once: mape_kernel_test_batch
(a9), mape_minimal_filter_batch (a11) and mape_direction_coeffs_batch (a12)
give every instance exactly what its own call gives, and that is the
oracle's (C1 by exact products, the brute-force ⊑-minimal set, g'Qg and
sum w g^4)."""
import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

from .gpu_common import dev
from .test_gpu_stages import _kernel_test_case, _planted_dense, _planted_set

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    return mape


def _kernel_rows(M, name, K, seed):
    """Kernel elements B w with small w and planted rows outside the kernel."""
    A, B = _kernel_test_case(name)
    n = A.shape[1]
    rng = np.random.default_rng(seed)
    W = np.zeros((K, B.shape[1]), np.int64)
    for r in range(K):
        idx = rng.choice(B.shape[1], size=2, replace=False)
        W[r, idx] = rng.integers(-1, 2, size=2)
    G = W @ B.T.astype(np.int64)
    G = G[np.all(np.abs(G) <= 127, axis=1)]
    G[::5, 7] += 1
    ldg = M.round16(n)
    buf = np.zeros((max(G.shape[0], 1), ldg), np.int8)
    buf[: G.shape[0], :n] = G
    buf[:, n:] = 5  # the row padding must not take part
    return A, G, dev(buf)[: G.shape[0]]


def test_kernel_test_batch(M):
    cases = [_kernel_rows(M, name, K, 3 + k)
             for k, (name, K) in enumerate([("medium", 3000), ("large", 2000), ("dense300", 1500), ("medium", 1)])]
    out = M.kernel_test_batch([(dev(A), buf, A.shape[1]) for A, G, buf in cases])
    for (A, G, buf), (ok, fails) in zip(cases, out):
        ok = ok.cpu().numpy().astype(bool)
        single, sf = M.kernel_test(dev(A), buf, A.shape[1])
        expect = O.kernel_condition(A, G)
        assert np.array_equal(ok, expect) and np.array_equal(single.cpu().numpy().astype(bool), expect)
        assert fails == sf == int((~expect).sum())


def test_minimal_filter_batch(M):
    rng = np.random.default_rng(5)
    sets = [_planted_set(rng, 300, 12), _planted_set(rng, 2500, 40), _planted_dense(rng, 1000, 200),
            _planted_dense(rng, 400, 5), _planted_set(rng, 1200, 200)]
    cases, valids = [], []
    for k, G in enumerate(sets):
        n = G.shape[1]
        buf = np.zeros((G.shape[0], M.round16(n)), np.int8)
        buf[:, :n] = G
        valid = np.ones(G.shape[0], np.uint8)
        if k % 2:
            valid[::13] = 0
        valids.append(valid)
        cases.append((dev(buf), n, dev(valid)))
    out = M.minimal_filter_batch(cases)
    for G, valid, (buf, n, vd), (keep, kept) in zip(sets, valids, cases, out):
        keep = keep.cpu().numpy().astype(bool)
        sk, sout = M.minimal_filter(buf, n, valid=vd)
        assert np.array_equal(keep, sk.cpu().numpy().astype(bool))
        assert np.array_equal(kept.cpu().numpy(), sout.cpu().numpy())
        expect = np.zeros(G.shape[0], bool)
        expect[np.nonzero(valid)[0]] = O.minimal_elements(G[valid.astype(bool)])
        assert np.array_equal(keep, expect)
        assert np.array_equal(kept.cpu().numpy()[:, :n].astype(np.int64), G[expect])


def test_direction_coeffs_batch(M):
    rng = np.random.default_rng(9)
    cases, host = [], []
    for inst, quartic in [(I.small_dense(), False), (I.medium_sparse(), True), (I.uneven_single(300), True)]:
        D = rng.integers(-3, 4, size=(500, inst.n)) * (rng.random((500, inst.n)) < 0.2)
        w = rng.integers(0, 4, size=inst.n).astype(np.int32) if quartic else None
        buf = np.zeros((D.shape[0], M.round16(inst.n)), np.int8)
        buf[:, : inst.n] = D
        qr, qc, qv = (dev(x) for x in M.coo_upper(inst.Q))
        cases.append((qr, qc, qv, None if w is None else dev(w), inst.n, dev(buf)))
        host.append((inst, D, w))
    out = M.direction_coeffs_batch(cases)
    for (qr, qc, qv, wd, n, G), (inst, D, w), (a, q4) in zip(cases, host, out):
        sa, sq = M.direction_coeffs(qr, qc, qv, wd, n, G)
        assert np.array_equal(a.cpu().numpy(), sa.cpu().numpy())
        assert np.array_equal(q4.cpu().numpy(), sq.cpu().numpy())
        assert np.array_equal(a.cpu().numpy(), np.einsum("ki,ij,kj->k", D, inst.Q.astype(np.int64), D))
        q4e = (D.astype(np.int64) ** 4) @ w.astype(np.int64) if w is not None else np.zeros(D.shape[0], np.int64)
        assert np.array_equal(q4.cpu().numpy(), q4e)
