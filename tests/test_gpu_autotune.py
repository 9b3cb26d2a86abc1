"""The autotuner (MAPE_PREC_AUTOTUNE): it times every candidate (the resident
kernel where it fits, the streamed kernels with forward/gradient N-block
widths in {64, 128, 256}) on scratch copies, keeps the fastest, and the call
then gives bitwise the result of the chosen implementation on the caller's
untouched state."""
import numpy as np
import pytest

from paper_2412_13576_gb300 import instances as I

from .gpu_common import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    mape.lib().mape_autotune_clear()
    return mape


def _run(M, inst, Z0, T, precision):
    import torch
    ldc = M.round16(inst.n)
    Z = dev(Z0)
    Mm, V = torch.zeros_like(Z), torch.zeros_like(Z)
    cand = torch.zeros((Z0.shape[0] * (T + 1), ldc), dtype=torch.int8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    cfg = M.default_config(precision=precision)
    M.extract(dev(inst.B), dev((inst.u - inst.l).astype(np.int32)), Z, Mm, V, t0=0, T=T, cfg=cfg, cand=cand,
              cand_count=cnt, flags=flags, ldc=ldc)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0
    k = int(cnt.item())
    return Z.cpu().numpy(), Mm.cpu().numpy(), V.cpu().numpy(), {tuple(r) for r in cand[:k, : inst.n].cpu().numpy()}


@pytest.mark.parametrize("make,P,std", [(lambda: I.uneven_single(500), 1024, 0.3), (I.medium_sparse, 2048, 0.3)])
def test_autotuned_call_equals_chosen_implementation(M, make, P, std):
    inst = make()
    Z0 = I.normal_starts(inst, P, std=std, seed=21).Z0
    T = 12
    tuned = _run(M, inst, Z0, T, M.PREC_BF16 | M.PREC_AUTOTUNE)
    info = M.autotune_info(inst.n, inst.d, P, M.PREC_BF16)
    assert info is not None and len(info["candidates"]) >= 9
    fastest = min(info["candidates"], key=lambda c: c["ms"])
    assert (fastest["path"], fastest["wF"], fastest["wG"]) == (info["path"], info["wF"], info["wG"])
    resident_fits = any(c["path"] == "resident" for c in info["candidates"])
    assert resident_fits == (inst.d <= 256)
    # streamed results do not depend on the widths: compare with the default widths
    ref_prec = M.PREC_BF16 if info["path"] == "resident" else (M.PREC_BF16 | M.PREC_STREAMED)
    ref = _run(M, inst, Z0, T, ref_prec)
    for a, b in zip(tuned[:3], ref[:3]):
        assert np.array_equal(a, b)
    assert tuned[3] == ref[3]
    # a second call reuses the choice
    again = _run(M, inst, Z0, T, M.PREC_BF16 | M.PREC_AUTOTUNE)
    assert np.array_equal(again[0], tuned[0])


def test_autotuned_fp8_widths(M):
    """MAPE_PREC_FP8 | MAPE_PREC_AUTOTUNE: only the streamed kernels' widths
    are candidates (nine), and the tuned call gives bitwise the result of the
    default widths (the K order of every accumulation does not depend on
    them)."""
    inst = I.uneven_single(1000, density=0.05)
    P, T = 1024, 12
    Z0 = I.normal_starts(inst, P, std=0.3, seed=23).Z0
    tuned = _run(M, inst, Z0, T, M.PREC_FP8 | M.PREC_AUTOTUNE)
    info = M.autotune_info(inst.n, inst.d, P, M.PREC_FP8)
    assert info is not None and len(info["candidates"]) == 9
    assert all(c["path"] == "streamed" for c in info["candidates"])
    ref = _run(M, inst, Z0, T, M.PREC_FP8)
    for a, b in zip(tuned[:3], ref[:3]):
        assert np.array_equal(a, b)
    assert tuned[3] == ref[3]
