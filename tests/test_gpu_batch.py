"""Batched extraction: uneven instances (resident and streamed shapes,
identity-topped and general bases, ragged start counts) in one graph-captured
call of mape_extract_batch give, per instance, bitwise the same Z, M, V and
the same collected set as its own mape_extract call, and that set is exactly
the oracle's collection applied to the batch's iterates."""
import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

from .gpu_common import dev, rows_set
from .test_gpu_bf16 import _general_basis

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    return mape


def _cases():
    out = []
    for k, (make, P, std) in enumerate([(I.small_dense, 300, 2.0), (I.medium_sparse, 1000, 0.3),
                                        (I.tiny_graver_case, 130, 2.0), (_general_basis(I.small_dense), 256, 2.0),
                                        (lambda: I.uneven_single(500), 200, 0.3),
                                        (_general_basis(lambda: I.uneven_single(400)), 150, 0.3),
                                        (lambda: I.uneven_single(150), 700, 0.3),
                                        (lambda: I.uneven_single(1000, density=0.05), 130, 0.3)]):
        inst = make()
        Z0 = I.normal_starts(inst, P, std=std, seed=500 + k).Z0
        out.append((inst, Z0))
    return out


def _buffers(M, inst, Z0, T):
    import torch
    Z = dev(Z0)
    ldc = M.round16(inst.n)
    return dict(B=dev(inst.B), span=dev((inst.u - inst.l).astype(np.int32)), Z=Z, M=torch.zeros_like(Z),
                V=torch.zeros_like(Z), cand=torch.zeros((Z0.shape[0] * (T + 1) + 8, ldc), dtype=torch.int8,
                                                         device="cuda"),
                cand_count=torch.zeros(1, dtype=torch.int64, device="cuda"),
                flags=torch.zeros(1, dtype=torch.int32, device="cuda"), ldc=ldc)


@pytest.mark.parametrize("precision", [1, 2])
def test_batch_equals_single_calls(M, precision):
    import torch
    T = 8
    cases = _cases()
    cfg = M.default_config(precision=precision, period=1)
    single, batch = [], []
    for inst, Z0 in cases:
        b = _buffers(M, inst, Z0, T)
        M.extract(t0=0, T=T, cfg=cfg, **b)
        single.append(b)
    calls = [_buffers(M, inst, Z0, T) for inst, Z0 in cases]
    M.extract_batch(calls, t0=0, T=T, cfg=cfg)
    torch.cuda.synchronize()
    total = 0
    for (inst, Z0), s, b in zip(cases, single, calls):
        assert int(s["flags"].item()) == 0 and int(b["flags"].item()) == 0
        for k in ("Z", "M", "V"):
            assert torch.equal(s[k], b[k]), (inst.name, k)
        cs = s["cand"][: int(s["cand_count"].item())].cpu().numpy()
        cb = b["cand"][: int(b["cand_count"].item())].cpu().numpy()
        assert rows_set(cs, inst.n) == rows_set(cb, inst.n)
        assert np.all(cb[:, inst.n:] == 0)
        total += len(rows_set(cb, inst.n))
    assert total > 0


def test_batch_matches_oracle_collection(M):
    """Per step, the batch's collected rows are the oracle's collection of the
    batch's own iterates (the steps run one batched call each)."""
    import torch
    T = 5
    cases = _cases()
    cfg = M.default_config(precision=1, period=1)
    calls = [_buffers(M, inst, Z0, T) for inst, Z0 in cases]
    expect = [set() for _ in cases]
    for t in range(T):
        M.extract_batch(calls, t0=t, T=1, cfg=cfg)
        torch.cuda.synchronize()
        for k, ((inst, _), b) in enumerate(zip(cases, calls)):
            expect[k] |= O.collect(inst.A, inst.B, inst.l, inst.u, b["Z"].cpu().numpy())
    for (inst, _), b, e in zip(cases, calls, expect):
        assert int(b["flags"].item()) == 0
        got = rows_set(b["cand"][: int(b["cand_count"].item())].cpu().numpy(), inst.n)
        assert got == e, inst.name


def _batched_vs_single(M, cases, cfg):
    single = []
    for inst, Z0 in cases:
        with M.Instance.from_generated(inst, cfg) as h:
            h.extract_directions(Z0.shape[0], Z0=Z0)
            h.wait(300)
            h.augment(inst.xbar[None, :])
            h.wait(300)
            single.append((h.directions(), h.solution()))
    handles = [M.Instance.from_generated(inst, cfg) for inst, _ in cases]
    try:
        M.extract_directions_batch(handles, [(Z0.shape[0], Z0, None) for _, Z0 in cases])
        for h in handles:
            h.wait(300)
        for (inst, _), h, (D, (x, f)) in zip(cases, handles, single):
            st = h.poll()
            assert st["phase"] == "DONE" and st["error"] == 0
            assert np.array_equal(h.directions(), D)
            h.augment(inst.xbar[None, :])
            h.wait(300)
            x2, f2 = h.solution()
            assert f2 == f and np.array_equal(x2, x)
        return [h.poll() for h in handles]
    finally:
        for h in handles:
            h.close()


def test_batched_handles_equal_single_handles(M):
    """mape_extract_directions_batch on eight handles (resident and streamed
    shapes, identity-topped and general bases): every handle's direction set
    equals the set of its own mape_extract_directions, and Algorithm 1 then
    reaches the same point."""
    sts = _batched_vs_single(M, _cases(), M.default_config(T=60, period=2))
    assert sum(st["directions"] for st in sts) > 0


def test_batched_handles_in_chunks(M):
    """A candidate buffer of 2000 rows makes the extraction run in chunks (the
    batch takes the shortest chunk any handle allows, and merges each
    handle's candidates after every chunk): the sets still equal the single
    handles'."""
    inst = I.tiny_graver_case()
    cases = [(inst, I.normal_starts(inst, 256, seed=700 + k).Z0) for k in range(3)]
    sts = _batched_vs_single(M, cases, M.default_config(T=200, cand_capacity=2000))
    assert all(st["candidates"] > 2000 for st in sts)


def test_batched_handles_refuse_mixed_configs(M):
    inst = I.small_dense()
    h1 = M.Instance.from_generated(inst, M.default_config(T=10))
    h2 = M.Instance.from_generated(inst, M.default_config(T=20))
    try:
        Z0 = I.normal_starts(inst, 64, seed=1).Z0
        with pytest.raises(M.MapeError) as e:
            M.extract_directions_batch([h1, h2], [(64, Z0, None), (64, Z0, None)])
        assert e.value.code == -1
    finally:
        h1.close()
        h2.close()
