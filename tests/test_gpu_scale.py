"""Parity at the sizes the benchmark runs, against the CPU oracle (run in a
pool of spawned processes, tests/oracle_pool.py):

* the minimality filter on 20 000 distinct candidate rows that the GPU
  extracted on the medium workload (n = 200, 8192 starts, 1000 steps);
* Algorithm 1 with 2500 GPU-extracted directions of the medium instance from
  8 starts: the same moves, final points and values;
* Algorithm 1 with the quartic objective of the large workload (n = 2000)
  with directions the GPU extracted there;
* the brute-force check of the definition of G(A): on the 6-variable, 2-row
  instance every direction the handle returns is a true Graver element."""
import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

from .gpu_common import dev, report

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    return mape


@pytest.fixture(scope="module")
def pool():
    from .oracle_pool import OraclePool
    p = OraclePool()
    yield p
    p.close()


def _extract_unique(M, inst, Z0, T, period=1, precision=1):
    """Algorithm 2 on the GPU (stage entry points): the distinct candidate
    rows that pass C1, as an int8 device tensor [K x ldg]."""
    import torch
    P = Z0.shape[0]
    ldc = M.round16(inst.n)
    B, span = dev(inst.B), dev((inst.u - inst.l).astype(np.int32))
    Z = dev(Z0.astype(np.float32))
    Mm, V = torch.zeros_like(Z), torch.zeros_like(Z)
    cand = torch.empty((P * (T // period + 1) + 16, ldc), dtype=torch.int8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    cfg = M.default_config(T=T, precision=precision, period=period)
    M.extract(B, span, Z, Mm, V, t0=0, T=T, cfg=cfg, cand=cand, cand_count=cnt, flags=flags, ldc=ldc)
    torch.cuda.synchronize()
    assert int(flags.item()) == 0
    U = M.dedup(cand, int(cnt.item()), inst.n)
    ok, fails = M.kernel_test(dev(inst.A), U, inst.n)
    assert fails == 0
    return U


@pytest.fixture(scope="module")
def medium_set(M):
    inst = I.medium_sparse()
    Z0 = O.project_to_coordinates(inst.B, I.uniform_samples(inst, 8192, seed=2002).G0).astype(np.float32)
    return inst, _extract_unique(M, inst, Z0, 1000)


def test_minimal_filter_on_extracted_set(M, pool, medium_set):
    """20 000 of the GPU's distinct candidates (every 5th of the sorted set,
    so that rows sharing long prefixes stay together less often): the kept
    mask equals the oracle's all-pairs minimality on exactly those rows."""
    inst, U = medium_set
    K_all = U.shape[0]
    assert K_all >= 100000
    sel = U[::5][:20000].contiguous()
    keep, out = M.minimal_filter(sel, inst.n)
    G = sel[:, : inst.n].cpu().numpy().astype(np.int64)
    expect = pool.minimal_elements(G)
    got = keep.cpu().numpy().astype(bool)
    report("minimal_filter_extracted", rows=int(G.shape[0]), kept=int(got.sum()), removed=int((~got).sum()))
    assert np.array_equal(got, expect)
    assert np.array_equal(out[:, : inst.n].cpu().numpy(), G[expect])


def _augment_case(M, pool, inst, w, D, X0, max_iters):
    import torch
    ldg = M.round16(inst.n)
    buf = np.zeros((D.shape[0], ldg), np.int8)
    buf[:, : inst.n] = D
    Gd = dev(buf)
    qr, qc, qv = (dev(x) for x in M.coo_upper(inst.Q))
    wd = None if w is None else dev(w)
    a, q4 = M.direction_coeffs(qr, qc, qv, wd, inst.n, Gd)
    X = dev(np.asarray(X0, np.int32))
    fval, iters, moves, nmoves = M.augment_run(Gd, inst.n, a, q4, qr, qc, qv, dev(inst.c), wd, dev(inst.l),
                                               dev(inst.u), X, max_iters=max_iters, moves_cap=4096)
    torch.cuda.synchronize()
    X, fval = X.cpu().numpy(), fval.cpu().numpy()
    moves, nmoves = moves.cpu().numpy(), nmoves.cpu().numpy()
    expect = pool.augment(inst, w, D, X0, max_iters=max_iters)
    total = 0
    for s, (xo, fo, mo) in enumerate(expect):
        got = [tuple(int(v) for v in moves[s, i]) for i in range(nmoves[s])]
        assert got == [(k, e, lam, f) for k, e, lam, f in mo], f"start {s}"
        assert fval[s] == fo and np.array_equal(X[s], xo)
        total += len(mo)
    return total


def _feasible_starts(inst, S, seed):
    """xbar and S - 1 other points of the feasible region: xbar + B w for
    random w with three entries +-1 (A B = 0 keeps A x = b), kept when they
    lie in the box (checked by the oracle)."""
    rng = np.random.default_rng(seed)
    B = inst.B.astype(np.int64)
    X0 = [inst.xbar.astype(np.int64)]
    for _ in range(100000):
        if len(X0) == S:
            break
        w = np.zeros(inst.d, np.int64)
        w[rng.choice(inst.d, size=3, replace=False)] = rng.choice([-1, 1], size=3)
        x = X0[0] + B @ w
        if O.in_feasible_region(inst.A, inst.b, inst.l, inst.u, x):
            X0.append(x)
    assert len(X0) == S
    return np.array(X0, np.int64)


def test_augment_with_extracted_directions(M, pool):
    """Algorithm 1 from 8 starts with 2500 directions of the GPU's extracted
    and minimality-filtered set on the medium instance: moves, points and
    values equal to the oracle's.  The starts are N(0, 0.3) (2048 starts, 300
    steps), whose roundings are short vectors; the projected uniform starts
    of the benchmark give long directions that leave the box from every
    feasible point, so Algorithm 1 would stop at once."""
    inst = I.medium_sparse()
    Z0 = I.normal_starts(inst, 2048, std=0.3, seed=2002).Z0
    U = _extract_unique(M, inst, Z0, 300)
    keep, out = M.minimal_filter(U, inst.n)
    D = out[:, : inst.n].cpu().numpy().astype(np.int64)
    assert D.shape[0] >= 2500
    rng = np.random.default_rng(17)
    D = D[np.sort(rng.choice(D.shape[0], size=2500, replace=False))]
    X0 = _feasible_starts(inst, 8, seed=23)
    moves = _augment_case(M, pool, inst, None, D, X0, max_iters=100000)
    report("augment_extracted_medium", directions=int(D.shape[0]), starts=int(X0.shape[0]), moves=moves)
    assert moves >= 8 * 5


def test_augment_large_quartic(M, pool):
    """The large workload's quartic f (n = 2000, w in [0,3]) with the 60
    shortest directions the GPU extracted there (512 starts N(0, 0.3), 600
    steps, collection every 50th; streamed kernels), from 4 starts, three
    iterations of Algorithm 1: the same moves.  The
    starts lie near a point x0 with entries in [-3, 3] (b = A x0, the same A,
    box and f), so that short directions stay in the box; from the generated
    xbar, whose entries fill the whole box, none of them does."""
    import dataclasses
    inst = I.large_quartic()
    Z0 = I.normal_starts(inst, 512, std=0.3, seed=2004).Z0
    U = _extract_unique(M, inst, Z0, 600, period=50)
    keep, out = M.minimal_filter(U, inst.n)
    D = out[:, : inst.n].cpu().numpy().astype(np.int64)
    assert D.shape[0] >= 60
    D = D[np.argsort(np.abs(D).sum(axis=1), kind="stable")[:60]]
    x0 = np.random.default_rng(31).integers(-3, 4, size=inst.n)
    inst = dataclasses.replace(inst, xbar=x0.astype(np.int32), b=inst.A.astype(np.int64) @ x0)
    X0 = _feasible_starts(inst, 4, seed=29)
    moves = _augment_case(M, pool, inst, inst.w, D, X0, max_iters=3)
    report("augment_large_quartic", directions=int(D.shape[0]), starts=int(X0.shape[0]), moves=moves)
    assert moves >= 4


def test_handle_returns_true_graver_elements(M):
    """The definition of G(A) (§1) by brute force: on the 6-variable, 2-row
    instance (entries in {-1, 0, 1}, box spans 3), every direction the handle
    returns from 4096 starts and 200 steps is a ⊑-minimal element of
    Ker_Z(A) \\ {0}, i.e. in the enumerated Graver basis; the share of the
    basis found is reported (the method is a heuristic and may miss some)."""
    inst = I.tiny_graver_case()
    graver = {tuple(int(v) for v in g) for g in O.graver_basis_box(inst.A, 3)}
    cfg = M.default_config(T=200)
    with M.Instance.from_generated(inst, cfg) as h:
        h.extract_directions(4096, Z0=I.normal_starts(inst, 4096, seed=2001).Z0)
        h.wait(300)
        D = h.directions()
    got = {tuple(int(v) for v in g) for g in D}
    report("tiny_graver_handle", returned=len(got), graver=len(graver), found=len(got & graver))
    assert got and got <= graver
    for g in D:
        assert O.is_graver_element(inst.A, g)
