"""Initial feasible solutions (Eq. (4)) on the GPU against the FP64 oracle:
per step the objective, the gradient and the projected Adam update within
1e-5, the collected rows exactly the oracle's feasible roundings of the GPU's
own iterates; T steps in one launch bitwise equal to T launches of one step;
every collected point exactly feasible."""
import itertools

import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

from .gpu_common import dev, per_start_rel

pytestmark = pytest.mark.gpu

TOL = 1e-5
LAM3 = 0.1


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    return mape


def _starts(inst, P, seed):
    """Half uniform in the box, half within 0.45 of the feasible point xbar
    (so that feasible roundings occur and are collected)."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(inst.l, inst.u, size=(P, inst.n))
    h = P // 2
    X[:h] = inst.xbar + rng.uniform(-0.45, 0.45, size=(h, inst.n))
    return X.astype(np.float32)


def _buffers(M, inst, X0, cap):
    import torch
    X = dev(X0)
    return dict(A=dev(inst.A), b=dev(inst.b.astype(np.int64)), l=dev(inst.l), u=dev(inst.u), X=X,
                M=torch.zeros_like(X), V=torch.zeros_like(X),
                sol=torch.zeros((cap, M.round16(inst.n)), dtype=torch.uint8, device="cuda"),
                sol_count=torch.zeros(1, dtype=torch.int64, device="cuda"),
                flags=torch.zeros(1, dtype=torch.int32, device="cuda"), lds=M.round16(inst.n))


def _rows(inst, buf):
    k = int(buf["sol_count"].item())
    R = buf["sol"][:k, : inst.n].cpu().numpy().astype(np.int64) + inst.l.astype(np.int64)
    return {tuple(r) for r in R}


@pytest.mark.parametrize("make,P,T", [(I.small_dense, 256, 20), (I.medium_sparse, 300, 8), (I.tiny_graver_case, 130, 30),
                                      (I.large_quartic, 64, 3)])
def test_init_per_step(M, make, P, T):
    import torch
    inst = make()
    buf = _buffers(M, inst, _starts(inst, P, 11), P * (T + 1))
    f = torch.empty(P, dtype=torch.float32, device="cuda")
    g = torch.empty((P, inst.n), dtype=torch.float32, device="cuda")
    expect = set()
    lo, hi = inst.l.astype(np.float64), inst.u.astype(np.float64)
    for t in range(T):
        x0 = np.clip(buf["X"].cpu().numpy().astype(np.float64), lo, hi)
        m0, v0 = buf["M"].cpu().numpy(), buf["V"].cpu().numpy()
        keep = M.initial_solutions(t0=t, T=1, lambda3=LAM3, dbg_f=f, dbg_grad=g, **buf)
        torch.cuda.synchronize()
        del keep
        go = O.init_gradient(inst.A, inst.b, x0, LAM3)
        fo = O.init_objective(inst.A, inst.b, x0, LAM3)
        # per start: the residual A x - b in FP32 is off by at most
        # n 2^-23 (sum_k |A_ik x_k| + |b_i|) per row; the gradient 2 A^T r and
        # the objective |r|^2 carry that on
        Af = np.abs(inst.A.astype(np.float64))
        r = x0 @ inst.A.T.astype(np.float64) - inst.b
        e = inst.n * 2.0 ** -23 * (np.abs(x0) @ Af.T + np.abs(inst.b)) * 1.01
        gk = g.cpu().numpy().astype(np.float64)
        scale = np.maximum(np.abs(go).max(axis=1), 1.0)[:, None]
        assert np.all(np.abs(gk - go) <= 2.0 * e @ Af + TOL * scale)
        fk = f.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(fk - fo) <= (2.0 * np.abs(r) * e + e * e).sum(1) + TOL * np.abs(fo) + 1e-6)
        xo, mo, vo = O.projected_adam_update(x0, m0, v0, gk, t + 1, 0.003, inst.l, inst.u)
        x1 = buf["X"].cpu().numpy()
        for got, want in ((x1, xo), (buf["M"].cpu().numpy(), mo), (buf["V"].cpu().numpy(), vo)):
            nz = np.linalg.norm(want, axis=1) > 0
            assert np.all(per_start_rel(got, want)[nz] <= TOL)
        assert np.all((x1 >= inst.l) & (x1 <= inst.u))
        expect |= O.feasible_roundings(inst.A, inst.b, inst.l, inst.u, x1)
    assert int(buf["flags"].item()) == 0
    got = _rows(inst, buf)
    assert got == expect
    assert len(got) > 0


def test_init_one_launch_equals_single_steps(M):
    import torch
    inst = I.medium_sparse()
    X0 = _starts(inst, 500, 3)
    T = 25
    a = _buffers(M, inst, X0, 500 * (T + 1))
    b = _buffers(M, inst, X0, 500 * (T + 1))
    M.initial_solutions(t0=0, T=T, period=2, **a)
    for t in range(T):
        M.initial_solutions(t0=t, T=1, period=2, **b)
    torch.cuda.synchronize()
    for k in ("X", "M", "V"):
        assert torch.equal(a[k], b[k])
    assert _rows(inst, a) == _rows(inst, b)


def test_init_collects_only_feasible_points(M):
    """From uniform starts on the 6-variable instance, after 1500 steps (lr
    0.01) the collected points are a nonempty subset of the feasible points of
    the box found by enumeration."""
    import torch
    inst = I.tiny_graver_case()
    X0 = np.random.default_rng(5).uniform(inst.l, inst.u, size=(512, inst.n)).astype(np.float32)
    buf = _buffers(M, inst, X0, 512 * 10)
    M.initial_solutions(t0=0, T=1500, lr=0.01, period=50, **buf)
    torch.cuda.synchronize()
    pts = np.array(list(itertools.product(*[range(lo, hi + 1) for lo, hi in zip(inst.l, inst.u)])), dtype=np.int64)
    feas = {tuple(x) for x in pts[np.all(pts @ inst.A.T.astype(np.int64) == inst.b, axis=1)]}
    got = _rows(inst, buf)
    assert got and got <= feas
