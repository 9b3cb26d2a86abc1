"""Algorithm 1 (§2; a12-a14) in its tuned and batched forms: the scoring
pass with every lane count per direction (and the byte-wise form for rows
that are not 16-byte aligned) gives the oracle's moves; many instances in
one mape_augment_run_batch give each instance exactly what its own
mape_augment_run gives; the handles' mape_augment_batch gives each handle
what its own mape_augment gives."""
import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

from .gpu_common import dev

pytestmark = pytest.mark.gpu

LANES = [1, 2, 4, 8, 16, 32, 0]  # 0: autotuned


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    return mape


def _directions(inst, P=256, T=60, seed=2001, std=2.0):
    Z0 = I.normal_starts(inst, P, std=std, seed=seed).Z0
    return O.parallel_extraction(inst.A, inst.B, inst.l, inst.u, Z0, T=T)["directions"]


def _starts(inst, D, extra, seed):
    """xbar and up to `extra` feasible points a few oracle moves away."""
    rng = np.random.default_rng(seed)
    starts = [inst.xbar.astype(np.int64)]
    x = starts[0]
    for k in rng.permutation(D.shape[0]):
        if len(starts) > extra:
            break
        lams = O.feasible_step_lengths(inst.l, inst.u, x, D[k])
        if lams:
            x = x + lams[0] * D[k]
            starts.append(x.copy())
    return np.array(starts, np.int32)


def _case(M, inst, D, w, X0, ldg=None, max_iters=10 ** 6, lanes=0):
    """augment_run's arguments on the device (rows at pitch ldg, default the
    16-byte multiple; coefficients from mape_direction_coeffs)."""
    ldg = ldg or M.round16(inst.n)
    buf = np.zeros((max(D.shape[0], 1), ldg), np.int8)
    buf[: D.shape[0], : inst.n] = D
    G = dev(buf)[: D.shape[0]]
    qr, qc, qv = (dev(x) for x in M.coo_upper(inst.Q))
    wd = None if w is None else dev(np.asarray(w, np.int32))
    a, q4 = M.direction_coeffs(qr, qc, qv, wd, inst.n, G)
    return dict(G=G, n=inst.n, a=a, q4=q4, qr=qr, qc=qc, qv=qv, c=dev(inst.c), w=wd, l=dev(inst.l), u=dev(inst.u),
                X=dev(np.asarray(X0, np.int32)), max_iters=max_iters, moves_cap=512, lanes=lanes)


def _run(M, r):
    fval, iters, moves, nmoves = M.augment_run(r["G"], r["n"], r["a"], r["q4"], r["qr"], r["qc"], r["qv"], r["c"],
                                               r["w"], r["l"], r["u"], r["X"], max_iters=r["max_iters"],
                                               moves_cap=r["moves_cap"], lanes=r["lanes"])
    return _host(r["X"], fval, iters, moves, nmoves)


def _host(X, fval, iters, moves, nmoves):
    import torch
    torch.cuda.synchronize()
    return (X.cpu().numpy(), fval.cpu().numpy(), iters, None if moves is None else moves.cpu().numpy(),
            nmoves.cpu().numpy())


_ORACLE = {}


def _oracle_moves(inst, w, D, X0, got, key=None):
    """The oracle's Algorithm 1 from every start (cached under `key`) against
    the GPU's points, values and moves."""
    if key is None or key not in _ORACLE:
        res = [O.augment(inst.A, inst.b, inst.l, inst.u, inst.Q, inst.c, w, D, X0[s]) for s in range(X0.shape[0])]
        if key is not None:
            _ORACLE[key] = res
    else:
        res = _ORACLE[key]
    X, fval, _, moves, nmoves = got
    for s, (xo, fo, mo) in enumerate(res):
        assert fval[s] == fo and np.array_equal(X[s], xo)
        assert [tuple(int(v) for v in moves[s, i]) for i in range(nmoves[s])] == [tuple(m) for m in mo]


_MEDIUM = {}


def _medium_case(quartic):
    if quartic not in _MEDIUM:
        inst = I.medium_sparse()
        D = _directions(inst, P=128, T=40, std=0.3)
        w = np.random.default_rng(3).integers(0, 4, size=inst.n) if quartic else None
        X0 = _starts(inst, D, 3, seed=5)
        _MEDIUM[quartic] = (inst, D, w, X0)
    return _MEDIUM[quartic]


@pytest.mark.parametrize("lanes", LANES)
@pytest.mark.parametrize("quartic", [False, True])
def test_score_lanes_match_algorithm1(M, lanes, quartic):
    """Every lane count of the scoring pass gives the oracle's moves (medium
    instance, n = 200: a row is 13 pieces of 16 bytes)."""
    inst, D, w, X0 = _medium_case(quartic)
    assert D.shape[0] > 10
    got = _run(M, _case(M, inst, D, w, X0, lanes=lanes))
    assert got[4].sum() > 0
    _oracle_moves(inst, w, D, X0, got, key=("medium", quartic))


def test_score_bytewise_rows(M):
    """Rows at a pitch that is not a multiple of 16 (n = 20): the byte-wise
    form, the same moves as the oracle."""
    inst = I.small_dense()
    D = _directions(inst)
    X0 = _starts(inst, D, 3, seed=7)
    _oracle_moves(inst, None, D, X0, _run(M, _case(M, inst, D, None, X0, ldg=inst.n, lanes=8)))


_WIDE = {}


def _wide_case(quartic):
    """Box spans of 127 (the largest the handle accepts) and direction entries
    up to 120 in magnitude: the λ bounds floor((u - x) / |g_i|) take their
    widest operands.  The directions are kernel vectors B z with sparse z of
    entries up to 40, 12 and 3 in magnitude, kept while max |g| <= 120."""
    if quartic not in _WIDE:
        inst = I.make_instance("wide", 24, 4, c_k=1, c_density=None, lo=-63, hi=64, q_k=3, q_density=0.3,
                               lin_k=200, w_max=2 if quartic else None, seed=1017)
        rng = np.random.default_rng(23)
        Z = np.concatenate([rng.integers(-k, k + 1, size=(200, inst.d)) * (rng.random((200, inst.d)) < 0.3)
                            for k in (40, 12, 3)])
        G = Z @ inst.B.T.astype(np.int64)
        G = G[(np.abs(G).max(axis=1) <= 120) & np.any(G != 0, axis=1)]
        G = np.unique(np.array([O.canonical_sign(g) for g in G]), axis=0)
        G = G[rng.permutation(G.shape[0])[:200]]
        X0 = _starts(inst, G, 2, seed=29)
        _WIDE[quartic] = (inst, G, inst.w, X0)
    return _WIDE[quartic]


@pytest.mark.parametrize("lanes", [1, 2, 0])
@pytest.mark.parametrize("quartic", [False, True])
def test_score_wide_spans_match_algorithm1(M, lanes, quartic):
    inst, D, w, X0 = _wide_case(quartic)
    assert D.shape[0] > 20 and int(np.abs(D).max()) > 90
    got = _run(M, _case(M, inst, D, w, X0, lanes=lanes))
    assert got[4].sum() > 0
    _oracle_moves(inst, w, D, X0, got, key=("wide", quartic))


def test_autotuned_lanes_recorded(M):
    inst, D, _, X0 = _medium_case(False)
    M.lib().mape_autotune_clear()
    _run(M, _case(M, inst, D, None, X0, lanes=0))
    info = M.augment_tune_lookup(inst.n, D.shape[0], X0.shape[0], False)
    assert info is not None and info["lanes"] in (1, 2, 4, 8, 16, 32)
    assert sorted(info["cand_lanes"]) == [1, 2, 4, 8, 16, 32]
    assert all(t > 0 for t in info["probe_ms"])


_BATCH = []


def _batch_cases(M):
    """Uneven instances: different n, directions, starts, objectives and
    iteration limits, one without directions and one without starts."""
    if _BATCH:
        return _BATCH
    cases = _BATCH
    rng = np.random.default_rng(11)
    for k, (make, P, T, std, quartic, max_iters) in enumerate([
            (I.small_dense, 256, 60, 2.0, False, 10 ** 6),
            (I.small_dense, 256, 60, 2.0, True, 10 ** 6),
            (I.tiny_graver_case, 128, 40, 2.0, False, 10 ** 6),
            (I.medium_sparse, 128, 40, 0.3, False, 10 ** 6),
            (I.medium_sparse, 128, 40, 0.3, True, 3),
            (lambda: I.uneven_single(300), 128, 40, 0.3, False, 10 ** 6)]):
        inst = make()
        D = _directions(inst, P=P, T=T, std=std, seed=2001 + k)
        w = rng.integers(0, 4, size=inst.n) if quartic else None
        X0 = _starts(inst, D, 3, seed=13 + k)
        cases.append((inst, D, w, X0, max_iters))
    inst = I.small_dense()
    cases.append((inst, np.zeros((0, inst.n), np.int64), None, inst.xbar[None, :].astype(np.int32), 10 ** 6))
    cases.append((inst, _directions(inst), None, np.zeros((0, inst.n), np.int32), 10 ** 6))
    return cases


@pytest.mark.parametrize("lanes", [0, 4])
def test_run_batch_equals_single_runs(M, lanes):
    """mape_augment_run_batch over eight uneven instances: each instance's
    points, values, moves, move counts and iteration count are those of its
    own mape_augment_run, and those are the oracle's."""
    cases = _batch_cases(M)
    single = [_run(M, _case(M, inst, D, w, X0, max_iters=mi, lanes=lanes)) for inst, D, w, X0, mi in cases]
    runs = [_case(M, inst, D, w, X0, max_iters=mi, lanes=lanes) for inst, D, w, X0, mi in cases]
    reported = []
    batch = [_host(r["X"], *out) for r, out in zip(runs, M.augment_run_batch(
        runs, on_done=lambda i, it: reported.append((i, it))))]
    # every run is reported once, with its iteration count; the runs without
    # starts or directions first
    assert sorted(i for i, _ in reported) == list(range(len(runs)))
    assert all(it == batch[i][2] for i, it in reported)
    assert [i for i, _ in reported][:2] == sorted([len(runs) - 2, len(runs) - 1])
    for (inst, D, w, X0, mi), s, b in zip(cases, single, batch):
        assert np.array_equal(s[0], b[0]) and np.array_equal(s[1], b[1])
        assert s[2] == b[2]
        assert np.array_equal(s[4], b[4])
        if X0.shape[0] > 0:
            for k in range(X0.shape[0]):
                assert np.array_equal(s[3][k, : s[4][k]], b[3][k, : b[4][k]])
        if inst.n <= 20 and D.shape[0] > 0 and X0.shape[0] > 0:  # the oracle's own run is quick there
            _oracle_moves(inst, w, D, X0, b)
    assert sum(int(b[4].sum()) for b in batch) > 10


def test_handle_augment_batch_equals_single(M):
    """mape_augment_batch over three handles (different n): each handle's best
    value, solutions and iteration count equal its own mape_augment."""
    insts = [I.small_dense(), I.medium_sparse(), I.uneven_single(300)]
    cfg = M.default_config(T=200, precision=M.PREC_BF16)
    hs = [M.Instance.from_generated(inst, cfg) for inst in insts]
    try:
        for h, inst in zip(hs, insts):
            h.extract_directions(1024, Z0=I.normal_starts(inst, 1024, std=0.3, seed=41).Z0)
        for h in hs:
            h.wait(300)
        X0s = []
        for h, inst in zip(hs, insts):
            D = h.directions()
            X0s.append(_starts(inst, D, 3, seed=43) if D.shape[0] else inst.xbar[None, :].astype(np.int32))
        single = []
        for h, X0 in zip(hs, X0s):
            h.augment(X0)
            h.wait(300)
            st = h.poll()
            single.append((st["best_f"], st["aug_iters"], h.solutions(X0.shape[0])))
        M.augment_batch(hs, X0s)
        for h, X0, (bf, it, (Xs, fs)) in zip(hs, X0s, single):
            h.wait(300)
            st = h.poll()
            Xb, fb = h.solutions(X0.shape[0])
            assert st["best_f"] == bf and st["aug_iters"] == it
            assert np.array_equal(Xb, Xs) and np.array_equal(fb, fs)
    finally:
        for h in hs:
            h.close()
