"""Parity of every stage of the CUDA path against the CPU oracle, called
through the C ABI (device buffers).  Integer stages are compared bit-exactly;
the FP32 continuous stages per start within relative 1e-5, with the allowance
for rows of B z whose sign FP32 does not fix (tests/gpu_common.py)."""
import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

from .gpu_common import check_phi_grad, check_steps, dev, per_start_rel, report, rows_set

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    return mape


def _inst(name):
    return {"small": I.small_dense, "medium": I.medium_sparse, "tiny": I.tiny_graver_case,
            "large": I.large_quartic}[name]()


# --- a2 ----------------------------------------------------------------------

@pytest.mark.parametrize("name,P", [("small", 300), ("medium", 1000), ("large", 256)])
def test_project_starts(M, name, P):
    inst = _inst(name)
    G0 = I.uniform_samples(inst, P, seed=7).G0
    Z = M.project_starts(dev(inst.B), dev(G0)).cpu().numpy()
    Zo = O.project_to_coordinates(inst.B, G0)
    # FP32 Cholesky solve: relative error per start below d * cond(B^T B) * 2^-24 * 8
    H = inst.B.astype(np.float64).T @ inst.B
    bound = 8 * inst.d * np.linalg.cond(H) * 2.0 ** -24
    err = per_start_rel(Z, Zo)
    assert err.max() < bound, (err.max(), bound)


# --- a3-a5 -----------------------------------------------------------------------

@pytest.mark.parametrize("name,P,scale", [("small", 512, 3.0), ("small", 512, 0.45), ("medium", 700, 4.0)])
def test_phi_grad_fp32(M, name, P, scale):
    """Eq. (3) and its gradient in FP32, per start (tests/gpu_common.py):
    within 1e-5 where FP32 fixes every sign(Bz)_i, within 2 |B_ij| per row it
    does not fix; z = 0 gives +inf and a zero gradient."""
    inst = _inst(name)
    rng = np.random.default_rng(11)
    Z = rng.uniform(-scale, scale, size=(P, inst.d)).astype(np.float32)
    Z[0] = 0.0                                  # z = 0: Phi = inf, gradient 0
    Z[1] = np.rint(Z[1]) + (Z[1] == 0)          # an integer point
    phi, grad = M.phi_grad(dev(inst.B), dev(Z))
    phi, grad = phi.cpu().numpy(), grad.cpu().numpy()
    assert np.isinf(phi[0]) and np.all(grad[0] == 0)
    st = check_phi_grad(inst.B, Z, phi, grad, 24, FP32_TOL)
    report(f"phi_grad_fp32/{name}/{scale}", **st)
    assert st["ambiguous_share"] <= 0.02


# --- a3-a8 (FP32 path), step by step against the oracle ------------------------

def _extract_steps(M, inst, Z0, T, precision, ldc, cap=1 << 16):
    """Runs T single steps through mape_extract, returning per-step states,
    gradients at the input point, and the collected candidate rows."""
    import torch
    cfg = M.default_config(precision=precision, T=1)
    P = Z0.shape[0]
    B, span = dev(inst.B), dev((inst.u - inst.l).astype(np.int32))
    Z = dev(Z0.astype(np.float32))
    Mm = torch.zeros_like(Z)
    V = torch.zeros_like(Z)
    cand = torch.zeros((cap, ldc), dtype=torch.int8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    flags = torch.zeros(1, dtype=torch.int32, device="cuda")
    gbuf = torch.empty_like(Z)
    pbuf = torch.empty(P, dtype=torch.float32, device="cuda")
    states, grads, phis = [], [], []
    for t in range(T):
        before = (Z.cpu().numpy(), Mm.cpu().numpy(), V.cpu().numpy())
        M.extract(B, span, Z, Mm, V, t0=t, T=1, cfg=cfg, cand=cand, cand_count=cnt, flags=flags, ldc=ldc,
                  dbg_phi=pbuf, dbg_grad=gbuf)
        torch.cuda.synchronize()
        states.append((before, (Z.cpu().numpy(), Mm.cpu().numpy(), V.cpu().numpy())))
        grads.append(gbuf.cpu().numpy())
        phis.append(pbuf.cpu().numpy())
    assert int(flags.item()) == 0
    return states, grads, phis, cand[: int(cnt.item())].cpu().numpy()


@pytest.mark.parametrize("name,P,T", [("small", 256, 30), ("medium", 256, 6)])
def test_extract_fp32_per_step(M, name, P, T):
    """Each GPU step from the GPU's own state matches one oracle step per start
    (Phi, gradient, Adam update; tests/gpu_common.py) within 1e-5, and the
    candidate rows collected over the run are exactly the oracle's collection
    applied to the GPU's iterates."""
    inst = _inst(name)
    if name == "small":
        Z0 = I.normal_starts(inst, P, seed=2001).Z0
    else:
        Z0 = O.project_to_coordinates(inst.B, I.uniform_samples(inst, P, seed=2002).G0).astype(np.float32)
    ldc = M.round16(inst.n)
    states, grads, phis, cand = _extract_steps(M, inst, Z0, T, M.PREC_FP32, ldc)
    expect, share, rows, worst = check_steps(inst, states, grads, phis, 24, FP32_TOL)
    report(f"extract_fp32_per_step/{name}", ambiguous_share=share, ambiguous_rows=rows, max_rel_grad_determined=worst)
    assert share <= {"small": 0.005, "medium": 0.03}[name]      # observed on GB300, rounded up
    assert rows_set(cand, inst.n) == expect


# --- a10 -----------------------------------------------------------------------

@pytest.mark.parametrize("count,n", [(1, 5), (5000, 20), (40000, 200), (3, 300)])
def test_dedup_exact(M, count, n):
    rng = np.random.default_rng(count)
    ldc = M.round16(n)
    base = rng.integers(-4, 5, size=(max(1, count // 7), n)).astype(np.int8)
    rows = base[rng.integers(0, base.shape[0], size=count)]
    buf = np.zeros((count, ldc), np.int8)
    buf[:, :n] = rows
    uniq = M.dedup(dev(buf), count, n).cpu().numpy()
    expect = O.sort_directions(np.unique(rows.astype(np.int64), axis=0))
    assert np.array_equal(uniq[:, :n].astype(np.int64), expect)
    assert np.all(uniq[:, n:] == 0)


@pytest.mark.parametrize("count,n,groups", [(6000, 40, 1), (20000, 64, 300), (3000, 8, 5)])
def test_dedup_shared_prefixes(M, count, n, groups):
    """Rows sharing their first 8 bytes: many short runs of equal sort keys
    (sorted per run by the remaining bytes), one run longer than a block
    sorts (the whole array sorted again by the rows), rows of 8 bytes."""
    rng = np.random.default_rng(count + n)
    ldc = M.round16(n)
    base = rng.integers(-2, 3, size=(max(1, count // 3), n))
    base[:, : min(8, n)] = rng.integers(-3, 4, size=(groups, min(8, n)))[rng.integers(0, groups, size=base.shape[0])]
    rows = base[rng.integers(0, base.shape[0], size=count)].astype(np.int8)
    buf = np.zeros((count, ldc), np.int8)
    buf[:, :n] = rows
    uniq = M.dedup(dev(buf), count, n).cpu().numpy()
    expect = O.sort_directions(np.unique(rows.astype(np.int64), axis=0))
    assert np.array_equal(uniq[:, :n].astype(np.int64), expect)
    assert np.all(uniq[:, n:] == 0)


# --- a9 ------------------------------------------------------------------------

def _kernel_test_case(name):
    """(A, B) pairs for C1: the medium instance (int8 A, 208-byte rows: the
    dp4a path), the large one (n = 2000: compressed rows of A), a dense A with
    entries beyond int8 on short rows, and a dense int8 A on 304-byte rows
    (both compressed, the latter with every entry nonzero)."""
    if name == "medium":
        inst = I.medium_sparse()
        return inst.A, inst.B
    if name == "large":
        inst = I.large_quartic()
        return inst.A, inst.B
    rng = np.random.default_rng(21)
    if name == "wide_entries":
        m, n, k = 6, 40, 1 << 20
    else:
        m, n, k = 30, 300, 3
    C = rng.integers(-k, k + 1, size=(m, n - m))
    C[C == 0] = 1
    if name == "wide_entries":
        # equal column pairs: e_2k - e_2k+1 (and sums of them) are short
        # kernel elements although the entries of A are far beyond int8
        C[:, 1::2] = C[:, 0::2]
    A = np.concatenate([C, np.eye(m, dtype=np.int64)], axis=1)
    B = np.concatenate([np.eye(n - m, dtype=np.int64), -C], axis=0)
    return A.astype(np.int32), B


@pytest.mark.parametrize("name,K", [("medium", 3000), ("large", 5000), ("wide_entries", 3000), ("dense300", 3000)])
def test_kernel_test_exact(M, name, K):
    A, B = _kernel_test_case(name)
    m, n = A.shape
    rng = np.random.default_rng(3)
    # kernel elements B w with small w, rows outside the kernel planted among them
    W = np.zeros((K, B.shape[1]), np.int64)
    for r in range(K):
        if name == "wide_entries":
            for p in rng.choice(B.shape[1] // 2, size=2, replace=False):
                s = rng.choice([-1, 1])
                W[r, 2 * p], W[r, 2 * p + 1] = s, -s
        else:
            idx = rng.choice(B.shape[1], size=2, replace=False)
            W[r, idx] = rng.integers(-1, 2, size=2)
    G = W @ B.T.astype(np.int64)
    keep = np.all(np.abs(G) <= 127, axis=1)
    G = G[keep]
    G[::5, 7] += 1                      # planted rows outside the kernel
    G[1::7, n - 1] -= 1
    ldg = M.round16(n)
    buf = np.zeros((G.shape[0], ldg), np.int8)
    buf[:, :n] = G
    buf[:, n:] = 5                      # the row padding must not take part
    ok, fails = M.kernel_test(dev(A), dev(buf), n)
    expect = O.kernel_condition(A, G)
    assert np.array_equal(ok.cpu().numpy().astype(bool), expect)
    assert fails == int((~expect).sum()) > 0
    assert expect.sum() > 0.5 * len(G)


# --- a11 -----------------------------------------------------------------------

def _planted_set(rng, K, n):
    """Random canonical distinct rows plus conformal sums that must be removed."""
    base = rng.integers(-3, 4, size=(K, n)) * (rng.random((K, n)) < 0.3)
    base = base[np.any(base != 0, axis=1)]
    extra = []
    for _ in range(K // 4):
        a, b = base[rng.integers(0, base.shape[0], size=2)]
        s = np.where(a * b >= 0, a + b, a)          # a ⊑ s by construction
        if np.all(np.abs(s) <= 120):
            extra.append(s)
    G = np.concatenate([base, np.array(extra)]) if extra else base
    G = np.array([O.canonical_sign(g) for g in G])
    G = O.sort_directions(np.unique(G[np.any(G != 0, axis=1)], axis=0))
    return G


@pytest.mark.parametrize("K,n", [(300, 12), (2500, 40), (1200, 200)])
def test_minimal_filter_exact(M, K, n):
    rng = np.random.default_rng(K + n)
    G = _planted_set(rng, K, n)
    ldg = M.round16(n)
    buf = np.zeros((G.shape[0], ldg), np.int8)
    buf[:, :n] = G
    valid = np.ones(G.shape[0], np.uint8)
    valid[::17] = 0
    keep, out = M.minimal_filter(dev(buf), n, valid=dev(valid))
    keep = keep.cpu().numpy().astype(bool)
    sub = G[valid.astype(bool)]
    expect_sub = O.minimal_elements(sub)
    expect = np.zeros(G.shape[0], bool)
    expect[np.nonzero(valid)[0]] = expect_sub
    assert np.array_equal(keep, expect)
    assert np.array_equal(out.cpu().numpy()[:, :n].astype(np.int64), G[expect])
    assert 0 < expect.sum() < valid.sum()


def _planted_dense(rng, K, n):
    """Dense rows (about 5% zeros; half the rows zero on coordinates 0-1),
    plus rows s with a ⊑ s and, for about half of them, -a ⊑ s with s
    canonical through an extra leading entry where a is zero: pairs meet in
    the pattern lists of the key coordinates in both orientations, with and
    without zeros there."""
    base = rng.integers(1, 4, size=(K, n)) * rng.choice([-1, 1], size=(K, n))
    base = base * (rng.random((K, n)) > 0.05)
    base[:, :2] *= (rng.random((K, 1)) < 0.5)
    base = base[np.any(base != 0, axis=1)]
    base = np.array([O.canonical_sign(g) for g in base])
    extra = []
    for _ in range(K // 3):
        a = base[rng.integers(0, base.shape[0])]
        s = a + np.sign(a) * rng.integers(0, 3, size=n)  # a ⊑ s
        if rng.random() < 0.5 and a[0] == 0:
            s = -s
            s[0] = rng.integers(1, 3)  # canonical; -a ⊑ s
        extra.append(s)
    G = np.concatenate([base, np.array(extra)])
    G = np.array([O.canonical_sign(g) for g in G])
    return O.sort_directions(np.unique(G[np.any(G != 0, axis=1)], axis=0))


@pytest.mark.parametrize("K,n", [(2000, 64), (1000, 200), (400, 5)])
def test_minimal_filter_dense_buckets(M, K, n):
    """Dense rows spread the set over the sign-pattern lists of the key
    coordinates; the kept set equals the brute-force ⊑-minimal set."""
    rng = np.random.default_rng(7 * K + n)
    G = _planted_dense(rng, K, n)
    ldg = M.round16(n)
    buf = np.zeros((G.shape[0], ldg), np.int8)
    buf[:, :n] = G
    keep, out = M.minimal_filter(dev(buf), n)
    expect = O.minimal_elements(G)
    assert np.array_equal(keep.cpu().numpy().astype(bool), expect)
    assert np.array_equal(out.cpu().numpy()[:, :n].astype(np.int64), G[expect])
    assert 0 < expect.sum() < G.shape[0]


# --- a12-a14 ---------------------------------------------------------------------

def _directions_for(inst, P=256, T=60, seed=2001):
    Z0 = I.normal_starts(inst, P, seed=seed).Z0
    return O.parallel_extraction(inst.A, inst.B, inst.l, inst.u, Z0, T=T)["directions"]


@pytest.mark.parametrize("quartic", [False, True])
def test_direction_coeffs_exact(M, quartic):
    inst = I.small_dense()
    D = _directions_for(inst)
    w = np.random.default_rng(1).integers(0, 4, size=inst.n).astype(np.int32) if quartic else None
    ldg = M.round16(inst.n)
    buf = np.zeros((D.shape[0], ldg), np.int8)
    buf[:, : inst.n] = D
    qr, qc, qv = M.coo_upper(inst.Q)
    a, q4 = M.direction_coeffs(dev(qr), dev(qc), dev(qv), None if w is None else dev(w), inst.n, dev(buf))
    a_exp = np.einsum("ki,ij,kj->k", D, inst.Q.astype(np.int64), D)
    assert np.array_equal(a.cpu().numpy(), a_exp)
    q4_exp = (D ** 4) @ w.astype(np.int64) if quartic else np.zeros(D.shape[0], np.int64)
    assert np.array_equal(q4.cpu().numpy(), q4_exp)


@pytest.mark.parametrize("quartic", [False, True])
def test_augment_matches_algorithm1(M, quartic):
    """Same moves, final point and value as the oracle's Algorithm 1 (which
    evaluates f directly at every candidate point)."""
    import torch
    inst = I.small_dense()
    D = _directions_for(inst)
    w = np.random.default_rng(2).integers(0, 4, size=inst.n).astype(np.int32) if quartic else None
    ldg = M.round16(inst.n)
    buf = np.zeros((D.shape[0], ldg), np.int8)
    buf[:, : inst.n] = D
    Gd = dev(buf)
    qr, qc, qv = (dev(x) for x in M.coo_upper(inst.Q))
    wd = None if w is None else dev(w)
    a, q4 = M.direction_coeffs(qr, qc, qv, wd, inst.n, Gd)
    # several starts: xbar and feasible points reached by a few oracle moves
    starts = [inst.xbar.astype(np.int64)]
    x = starts[0]
    for k in range(3):
        for lam in O.feasible_step_lengths(inst.l, inst.u, x, D[k])[:1]:
            x = x + lam * D[k]
            starts.append(x.copy())
    X0 = np.array(starts, np.int32)
    X = dev(X0)
    fval, iters, moves, nmoves = M.augment_run(Gd, inst.n, a, q4, qr, qc, qv, dev(inst.c), wd, dev(inst.l),
                                               dev(inst.u), X, moves_cap=256)
    X, fval = X.cpu().numpy(), fval.cpu().numpy()
    moves, nmoves = moves.cpu().numpy(), nmoves.cpu().numpy()
    for s in range(X0.shape[0]):
        xo, fo, mo = O.augment(inst.A, inst.b, inst.l, inst.u, inst.Q, inst.c, w, D, X0[s])
        assert fval[s] == fo
        assert np.array_equal(X[s], xo)
        got = [tuple(int(v) for v in moves[s, i]) for i in range(nmoves[s])]
        assert got == [(k, e, lam, f) for k, e, lam, f in mo]
    assert iters == max(nmoves) + 1
