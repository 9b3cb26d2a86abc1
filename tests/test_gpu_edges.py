"""Edge and degenerate cases of the path on the GPU: empty calls, a single
start (one ragged tile), a one-dimensional kernel (n = 2, m = 1), empty and
single-row stage inputs, all-equal candidates, an augmentation with no
directions, and the step-count limit."""
import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

from .gpu_common import dev, rows_set

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    return mape


def _bufs(inst, Z0, cap):
    import torch
    from paper_2412_13576_gb300 import mape
    Z = dev(Z0)
    ldc = mape.round16(inst.n)
    return dict(B=dev(inst.B), span=dev((inst.u - inst.l).astype(np.int32)), Z=Z, M=torch.zeros_like(Z),
                V=torch.zeros_like(Z), cand=torch.zeros((cap, ldc), dtype=torch.int8, device="cuda"),
                cand_count=torch.zeros(1, dtype=torch.int64, device="cuda"),
                flags=torch.zeros(1, dtype=torch.int32, device="cuda"), ldc=ldc)


@pytest.mark.parametrize("precision", [0, 1, 1 | 0x100, 3])
def test_empty_calls_change_nothing(M, precision):
    import torch
    inst = I.small_dense()
    Z0 = I.normal_starts(inst, 8, seed=1).Z0
    b = _bufs(inst, Z0, 16)
    M.extract(t0=0, T=0, cfg=M.default_config(precision=precision), **b)  # T = 0
    torch.cuda.synchronize()
    assert np.array_equal(b["Z"].cpu().numpy(), Z0) and int(b["cand_count"].item()) == 0
    e = _bufs(inst, Z0[:0], 16)  # P = 0
    M.extract(t0=0, T=5, cfg=M.default_config(precision=precision), **e)
    torch.cuda.synchronize()
    assert int(e["cand_count"].item()) == 0 and int(e["flags"].item()) == 0


@pytest.mark.parametrize("precision", [0, 1, 1 | 0x100, 3])
def test_single_start(M, precision):
    """P = 1: one start in a tile of 64 or 128; the collected set is the
    oracle's collection of that start's iterates."""
    import torch
    inst = I.small_dense()
    Z0 = I.normal_starts(inst, 1, seed=4).Z0
    b = _bufs(inst, Z0, 64)
    expect = set()
    cfg = M.default_config(precision=precision)
    for t in range(30):
        M.extract(t0=t, T=1, cfg=cfg, **b)
        torch.cuda.synchronize()
        expect |= O.collect(inst.A, inst.B, inst.l, inst.u, b["Z"].cpu().numpy())
    assert int(b["flags"].item()) == 0
    assert rows_set(b["cand"][: int(b["cand_count"].item())].cpu().numpy(), inst.n) == expect


def test_one_dimensional_kernel(M):
    """n = 2, m = 1: A = [c 1], the kernel is spanned by (1, -c); the handle
    returns exactly the Graver basis {(1, -c)} and augments to the oracle's
    optimum."""
    import dataclasses
    inst = I.make_instance("line_n2_m1", 2, 1, c_k=2, c_density=None, lo=-6, hi=6, q_k=3, q_density=1.0, lin_k=5,
                           seed=3)
    if inst.A[0, 0] == 0:
        inst = dataclasses.replace(inst, A=np.array([[2, 1]], np.int32), B=np.array([[1], [-2]], np.int32),
                                   b=np.array([2 * inst.xbar[0] + inst.xbar[1]], np.int64))
    cfg = M.default_config(T=300, precision=1)
    with M.Instance.from_generated(inst, cfg) as h:
        h.extract_directions(64, Z0=I.normal_starts(inst, 64, seed=2).Z0)
        h.wait(120)
        D = h.directions()
        g = O.canonical_sign(inst.B[:, 0].astype(np.int64))
        assert D.shape[0] == 1 and np.array_equal(D[0], g)
        h.augment(inst.xbar[None, :])
        h.wait(120)
        x, fx = h.solution()
    xo, fo, _ = O.augment(inst.A, inst.b, inst.l, inst.u, inst.Q, inst.c, None, D, inst.xbar)
    assert fx == fo and np.array_equal(x, xo)


def test_stages_on_empty_and_single_row_inputs(M):
    import torch
    inst = I.small_dense()
    ldg = M.round16(inst.n)
    empty = torch.zeros((0, ldg), dtype=torch.int8, device="cuda")
    ok, fails = M.kernel_test(dev(inst.A), empty, inst.n)
    assert ok.numel() == 0 and fails == 0
    keep, out = M.minimal_filter(empty, inst.n)
    assert out.shape[0] == 0
    assert M.dedup(empty, 0, inst.n).shape[0] == 0
    g = np.zeros((1, ldg), np.int8)
    g[0, : inst.n] = O.canonical_sign(inst.B[:, 0].astype(np.int64))
    ok, fails = M.kernel_test(dev(inst.A), dev(g), inst.n)
    assert fails == 0 and int(ok[0].item()) == 1
    keep, out = M.minimal_filter(dev(g), inst.n)
    assert out.shape[0] == 1 and np.array_equal(out.cpu().numpy(), g)
    # many copies of one row dedup to that row
    many = np.repeat(g, 5000, axis=0)
    u = M.dedup(dev(many), 5000, inst.n).cpu().numpy()
    assert u.shape[0] == 1 and np.array_equal(u, g)


def test_augmentation_without_directions(M):
    """K = 0: every start is already terminal; f(x0) is reported and x0 kept."""
    import torch
    inst = I.small_dense()
    ldg = M.round16(inst.n)
    G = torch.zeros((0, ldg), dtype=torch.int8, device="cuda")
    qr, qc, qv = (dev(x) for x in M.coo_upper(inst.Q))
    a, q4 = M.direction_coeffs(qr, qc, qv, None, inst.n, G)
    X0 = np.stack([inst.xbar, inst.xbar]).astype(np.int32)
    X = dev(X0)
    fval, iters, _, _ = M.augment_run(G, inst.n, a, q4, qr, qc, qv, dev(inst.c), None, dev(inst.l), dev(inst.u), X)
    assert np.array_equal(X.cpu().numpy(), X0)
    assert list(fval.cpu().numpy()) == [O.f_value(inst.Q, inst.c, None, inst.xbar)] * 2


def test_step_count_limit(M):
    import torch
    inst = I.small_dense()
    b = _bufs(inst, I.normal_starts(inst, 4, seed=1).Z0, 16)
    for prec in (1, 1 | 0x100, 3):
        with pytest.raises(M.MapeError) as e:
            M.extract(t0=0, T=(1 << 20) + 1, cfg=M.default_config(precision=prec), **b)
        assert e.value.code == -2
    torch.cuda.synchronize()


def test_mma_issue_probe_and_launch_timing(M):
    """The measurement entry points: the MMA cost probe returns positive cycle
    counts for both operand kinds and refuses shapes tcgen05 does not take;
    launch timing counts every streamed launch of a call and times it."""
    import torch
    for kind in (0, 1):
        issue, total = M.mma_issue_probe(kind, 128, 256, 1, 64)
        assert 0 < issue <= total < 1e6
    with pytest.raises(M.MapeError):
        M.mma_issue_probe(0, 96, 256)
    inst = I.uneven_single(1000, density=0.05)
    Z = dev(I.normal_starts(inst, 256, std=0.3, seed=3).Z0)
    ldc = M.round16(inst.n)
    cand = torch.zeros((256 * 5, ldc), dtype=torch.int8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    M.launch_timing(True)
    try:
        M.extract(dev(inst.B), dev((inst.u - inst.l).astype(np.int32)), Z, torch.zeros_like(Z), torch.zeros_like(Z),
                  t0=0, T=4, cfg=M.default_config(precision=M.PREC_BF16, period=2), cand=cand, cand_count=cnt,
                  flags=flags, ldc=ldc)
        got = M.launch_timing_read()
    finally:
        M.launch_timing(False)
    assert got["stream_grad"][1] == 4 and got["stream_fwd"][1] == 5 and got["stream_collect"][1] == 2
    assert all(ms > 0 for ms, n in got.values() if n > 0)
