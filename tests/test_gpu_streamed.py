"""The streamed tensor-core path of Algorithm 2 (three kernels per step, B and
z, m, v streamed through shared memory) against the FP64 oracle, on the shapes
only it takes (d or the MMA rows above 256: the uneven family up to n = 1000,
the large n = 2000 instance) and, forced with MAPE_PREC_STREAMED, on the
shapes the resident kernel also takes.  Same bar as the resident path, per
start and step (tests/gpu_common.py), candidates bit-exact."""
import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

from .gpu_common import check_steps, dev, report, rows_set
from .test_gpu_bf16 import FP32_TOL, PRECISIONS, _general_basis, _starts
from .test_gpu_stages import _extract_steps

pytestmark = pytest.mark.gpu

STREAMED = 0x100


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    return mape


def uneven500():
    return I.uneven_single(500)


def uneven1000():
    return I.uneven_single(1000, density=0.05)


def _z0(inst, P, seed, std):
    """std None: the paper's projected uniform starts; else Z0 ~ N(0, std),
    small enough that the rounded points meet the box within a few steps."""
    if std is None:
        return _starts(inst, P, seed)
    return I.normal_starts(inst, P, std=std, seed=seed).Z0


# (instance, P, T, force the streamed path, start scale)
CASES = [
    (I.small_dense, 256, 20, True, None),
    (I.medium_sparse, 300, 5, True, None),          # 3 tiles, the last one ragged
    (I.tiny_graver_case, 130, 30, True, None),
    (_general_basis(I.small_dense), 256, 20, True, None),
    (uneven500, 200, 4, False, None),               # d = 400: streamed by necessity
    (uneven500, 200, 6, False, 0.3),
    (uneven1000, 130, 2, False, None),              # d = 800, 160 rows of B'
    (uneven1000, 130, 3, False, 0.3),
    (I.large_quartic, 256, 2, False, None),         # n = 2000, d = 1600: 2 row blocks, 7 coordinate blocks
    (I.large_quartic, 256, 3, False, 0.3),
    (_general_basis(uneven500), 130, 4, False, 0.3),  # general B: all 500 rows through the MMA
]

# Largest share of start-steps with an ambiguous row of B z, per case (name,
# start scale) and precision, as observed on GB300 (rounded up); those
# start-steps are still checked against the per-row allowance.  Projected
# uniform starts (scale None) on n >= 500 reach |z| ~ 10-20, where sum_j
# |B_ij z_j| is large against |(Bz)_i|; with z as one BF16 term (8 bits) every
# start then has ambiguous rows (a few of hundreds per start).
AMBIGUOUS_CAP = {
    ("small_dense", None, 1): 0.005, ("small_dense", None, 2): 0.12,
    ("medium_sparse", None, 1): 0.05, ("medium_sparse", None, 2): 0.9,
    ("tiny_graver_case", None, 1): 0.005, ("tiny_graver_case", None, 2): 0.02,
    ("small_dense_general_basis", None, 1): 0.005, ("small_dense_general_basis", None, 2): 0.12,
    ("uneven500", None, 1): 0.4, ("uneven500", None, 2): 1.0,
    ("uneven500", 0.3, 1): 0.07, ("uneven500", 0.3, 2): 0.95,
    ("uneven1000", None, 1): 0.75, ("uneven1000", None, 2): 1.0,
    ("uneven1000", 0.3, 1): 0.16, ("uneven1000", 0.3, 2): 1.0,
    ("large_quartic", None, 1): 0.9, ("large_quartic", None, 2): 1.0,
    ("large_quartic", 0.3, 1): 0.35, ("large_quartic", 0.3, 2): 1.0,
    ("uneven500_general_basis", 0.3, 1): 0.16, ("uneven500_general_basis", 0.3, 2): 1.0,
}


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("make,P,T,force,std", CASES)
def test_streamed_per_step(M, make, P, T, force, std, precision):
    """Per start and step, the rules of tests/gpu_common.py: gradient within
    1e-5 off the ambiguous rows' reach and within 2 |B_ij| per ambiguous row,
    Phi within the forward error bound, Adam within 1e-5; candidates
    bit-exact."""
    inst = make()
    Z0 = _z0(inst, P, 2003, std)
    ldc = M.round16(inst.n)
    bits = PRECISIONS[precision]
    prec = precision | (STREAMED if force else 0)
    states, grads, phis, cand = _extract_steps(M, inst, Z0, T, prec, ldc, cap=P * (T + 1) + 16)
    expect, share, rows, worst = check_steps(inst, states, grads, phis, bits, FP32_TOL)
    key = (make.__name__, std, precision)
    report(f"streamed_per_step/{make.__name__}/{std}/{precision}", ambiguous_share=share, ambiguous_rows=rows,
           max_rel_grad_determined=worst)
    assert share <= AMBIGUOUS_CAP[key]
    assert rows_set(cand, inst.n) == expect


# the forward product of the streamed path: the tensor-core one (default) or
# the CUDA-core sparse one (MAPE_PREC_SPARSE_FWD), which takes the
# identity-topped bases of density <= 1/16 (large_quartic at 0.01, uneven1000
# at 0.05)
SPARSE_FWD = 0x400


@pytest.mark.parametrize("fwd", [0, SPARSE_FWD])
@pytest.mark.parametrize("make,P,T,std", [(I.large_quartic, 256, 3, 0.3), (uneven1000, 200, 4, 0.3),
                                          (uneven1000, 130, 2, None)])
def test_streamed_sparse_and_dense_forward_per_step(M, make, P, T, std, fwd):
    """Both forward products on the bases the sparse one takes, per start and
    step (tests/gpu_common.py); the sparse forward carries z in FP32 (24
    bits), so its bound is the FP32 one."""
    inst = make()
    Z0 = _z0(inst, P, 2013, std)
    ldc = M.round16(inst.n)
    bits = 24 if fwd else 16
    states, grads, phis, cand = _extract_steps(M, inst, Z0, T, M.PREC_BF16 | STREAMED | fwd, ldc,
                                               cap=P * (T + 1) + 16)
    expect, share, rows, worst = check_steps(inst, states, grads, phis, bits, FP32_TOL)
    report(f"streamed_forward/{make.__name__}/{std}/{'sparse' if fwd else 'tensor'}", ambiguous_share=share,
           ambiguous_rows=rows, max_rel_grad_determined=worst)
    # observed on GB300, rounded up
    assert share <= {(True, 0.3): 0.3, (False, 0.3): 0.3, (True, None): 0.65, (False, None): 0.7}[(bool(fwd), std)]
    assert rows_set(cand, inst.n) == expect


FP8 = 4


@pytest.mark.parametrize("make,P,T,std", [(I.large_quartic, 256, 3, 0.3), (I.large_quartic, 256, 2, None),
                                          (uneven1000, 200, 4, 0.3), (I.medium_sparse, 300, 5, None),
                                          (I.small_dense, 256, 20, None)])
def test_fp8_forward_per_step(M, make, P, T, std):
    """MAPE_PREC_FP8: the forward product with z in e4m3 (per-start power-of-two
    scale) against the FP64 oracle, per start and step: z carries 4
    significant bits (relative 2^-4, plus half the e4m3 subnormal step in
    units of the start's scale), so most starts have rows whose sign is not
    fixed; those are held to the allowance of 2 |B_ij| per row; the gradient
    product, Adam and the exact B round(z) map are those of the BF16 path
    (candidates bit-exact)."""
    inst = make()
    Z0 = _z0(inst, P, 2017, std)
    ldc = M.round16(inst.n)
    states, grads, phis, cand = _extract_steps(M, inst, Z0, T, FP8, ldc, cap=P * (T + 1) + 16)
    expect, share, rows, worst = check_steps(inst, states, grads, phis, 4, FP32_TOL, fp8=True)
    report(f"fp8_per_step/{make.__name__}/{std}", ambiguous_share=share, ambiguous_rows=rows,
           max_rel_grad_determined=worst)
    assert rows_set(cand, inst.n) == expect


def test_fp8_rejects_basis_not_exact_in_e4m3(M):
    """An entry of B that e4m3 cannot hold (17) raises flag 8; nothing runs."""
    import torch
    inst = uneven1000()
    Bb = inst.B.copy()
    Bb[-1, 5] = 17
    Z = dev(_z0(inst, 128, 1, 0.3))
    cand = torch.zeros((1024, M.round16(inst.n)), dtype=torch.int8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    Z1 = Z.clone()
    M.extract(dev(Bb), dev((inst.u - inst.l).astype(np.int32)), Z1, torch.zeros_like(Z), torch.zeros_like(Z),
              t0=0, T=3, cfg=M.default_config(precision=FP8), cand=cand, cand_count=cnt, flags=flags,
              ldc=M.round16(inst.n))
    torch.cuda.synchronize()
    assert int(flags.item()) & 8
    assert int(cnt.item()) == 0 and torch.equal(Z1, Z)


@pytest.mark.parametrize("make,P,T,period,force,std,fwd", [(uneven500, 300, 12, 1, False, 0.3, 0),
                                                           (I.medium_sparse, 1000, 10, 3, True, None, 0),
                                                           (_general_basis(I.small_dense), 300, 15, 1, True, None, 0),
                                                           (uneven1000, 300, 12, 2, False, 0.3, 0),
                                                           (uneven1000, 300, 12, 2, False, 0.3, SPARSE_FWD),
                                                           (uneven1000, 300, 12, 2, False, 0.3, "fp8"),
                                                           (I.large_quartic, 300, 8, 3, False, 0.3, "fp8")])
def test_streamed_one_call_equals_single_steps(M, make, P, T, period, force, std, fwd):
    """T steps in one call give bitwise the same Z, M, V as T calls of one
    step, and the same set of collected directions (uneven1000: with the
    tensor-core, the sparse and the FP8 forward; large_quartic in FP8, where
    the steps without collection multiply both row blocks of Bm in one CTA
    per tile and the collecting steps one CTA per row block)."""
    import torch
    inst = make()
    Z0 = _z0(inst, P, 7, std)
    ldc = M.round16(inst.n)
    B, span = dev(inst.B), dev((inst.u - inst.l).astype(np.int32))
    # fwd: 0 or SPARSE_FWD with MAPE_PREC_BF16, or "fp8" for MAPE_PREC_FP8
    prec = (FP8 if fwd == "fp8" else M.PREC_BF16 | fwd) | (STREAMED if force else 0)
    results = []
    for single in (False, True):
        cfg = M.default_config(precision=prec, period=period)
        Z = dev(Z0)
        Mm = torch.zeros_like(Z)
        V = torch.zeros_like(Z)
        cand = torch.zeros((P * T + 8, ldc), dtype=torch.int8, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        flags = torch.zeros(1, dtype=torch.int32, device="cuda")
        if single:
            for t in range(T):
                M.extract(B, span, Z, Mm, V, t0=t, T=1, cfg=cfg, cand=cand, cand_count=cnt, flags=flags, ldc=ldc)
        else:
            M.extract(B, span, Z, Mm, V, t0=0, T=T, cfg=cfg, cand=cand, cand_count=cnt, flags=flags, ldc=ldc)
        torch.cuda.synchronize()
        assert int(flags.item()) == 0
        c = cand[: int(cnt.item())].cpu().numpy()
        results.append((Z.cpu().numpy(), Mm.cpu().numpy(), V.cpu().numpy(), rows_set(c, inst.n), c))
    (z1, m1, v1, s1, c1), (z2, m2, v2, s2, _) = results
    assert np.array_equal(z1, z2) and np.array_equal(m1, m2) and np.array_equal(v1, v2)
    assert s1 == s2
    assert len(s1) > 0
    assert np.all(c1[:, inst.n:] == 0)
    G = np.array(sorted(s1), dtype=np.int64)
    assert np.all(O.kernel_condition(inst.A, G)) and np.all(O.bound_consistent(G, inst.l, inst.u))


def test_streamed_rejects_inexact_basis(M):
    """|B_ij| > 256 is not exact in BF16: flag 8, nothing collected, state untouched."""
    import torch
    inst = uneven500()
    Bbig = inst.B.copy()
    Bbig[-1, 3] = 300
    Z0 = _starts(inst, 64, 1)
    Z = dev(Z0)
    cand = torch.zeros((1024, M.round16(inst.n)), dtype=torch.int8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    cfg = M.default_config(precision=M.PREC_BF16)
    M.extract(dev(Bbig), dev((inst.u - inst.l).astype(np.int32)), Z, torch.zeros_like(Z), torch.zeros_like(Z),
              t0=0, T=3, cfg=cfg, cand=cand, cand_count=cnt, flags=flags, ldc=M.round16(inst.n))
    torch.cuda.synchronize()
    assert int(flags.item()) & 8
    assert int(cnt.item()) == 0
    assert np.array_equal(Z.cpu().numpy(), Z0)


def _no_improving_move(inst, D, x, fx):
    """Termination of Algorithm 1: no g in +-D and integer lambda >= 1 keeps
    x + lambda g in the box and lowers f (A g = 0 keeps A x = b).  f is
    quadratic here, so f(x + lambda g) - f(x) = lambda^2 g'Qg + lambda (2 g'Qx + c'g),
    evaluated in float64 (exact: every term is an integer below 2^53)."""
    Dg = D.astype(np.float64)
    QG = Dg @ inst.Q.astype(np.float64)
    a = np.sum(QG * Dg, axis=1)
    xf = x.astype(np.float64)
    lin = 2.0 * (QG @ xf) + Dg @ inst.c.astype(np.float64)
    span = int(np.max(inst.u - inst.l))
    for sgn in (1.0, -1.0):
        for lam in range(1, span + 1):
            Y = xf[None, :] + lam * sgn * Dg
            inside = np.all((Y >= inst.l) & (Y <= inst.u), axis=1)
            delta = lam * lam * a + lam * sgn * lin
            assert not np.any(inside & (delta < 0))


def test_streamed_handle_end_to_end(M):
    """The handle on an instance only the streamed path takes (n = 500,
    d = 400): the returned set passes C1, C4, nonzero, canonical sign, order
    and distinctness, minimality on a sample of rows (the oracle's pairwise
    test), and augmentation from xbar ends feasible, no worse than xbar, with
    no improving move left in the set."""
    from .test_gpu_handle import check_direction_set
    inst = uneven500()
    cfg = M.default_config(T=60, precision=M.PREC_BF16)
    Z0 = _z0(inst, 512, 2003, 0.3)
    with M.Instance.from_generated(inst, cfg) as h:
        h.extract_directions(512, Z0=Z0)
        h.wait(600)
        s = h.poll()
        assert s["phase"] == "DONE" and s["error"] == 0
        D = h.directions()
        check_direction_set(inst, D)
        assert s["kernel_failures"] == 0
        rng = np.random.default_rng(0)
        sample = rng.choice(D.shape[0], size=min(200, D.shape[0]), replace=False)
        absD = np.abs(D.astype(np.int64))
        for i in sample:
            g = D[i].astype(np.int64)
            pos = np.all((D * g >= 0) & (absD <= absD[i]), axis=1)
            neg = np.all((-D * g >= 0) & (absD <= absD[i]), axis=1)
            hit = pos | neg
            hit[i] = False
            assert not hit.any()
        h.augment(inst.xbar[None, :])
        h.wait(600)
        x, fx = h.solution()
    assert np.array_equal(inst.A.astype(np.int64) @ x, inst.b)
    assert np.all((x >= inst.l) & (x <= inst.u))
    assert fx == O.f_value(inst.Q, inst.c, None, x)
    assert fx <= O.f_value(inst.Q, inst.c, None, inst.xbar)
    _no_improving_move(inst, D, x, fx)
