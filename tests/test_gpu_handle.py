"""The instance handle end to end (host arrays in, host arrays out): the
returned set satisfies C1, C4, nonzero, canonical sign, distinctness,
lexicographic order and ⊑-minimality; augmentation equals the oracle's
Algorithm 1 on the same set; status, errors and reuse behave."""
import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13576_gb300 import mape
    mape.lib(build_if_missing=True)
    return mape


def check_direction_set(inst, D):
    assert D.shape[0] > 0
    assert np.all(O.kernel_condition(inst.A, D))
    assert np.all(O.bound_consistent(D, inst.l, inst.u))
    assert np.all(np.any(D != 0, axis=1))
    assert all(np.array_equal(O.canonical_sign(g), g) for g in D)
    assert np.array_equal(O.sort_directions(D), D)
    assert np.unique(D, axis=0).shape[0] == D.shape[0]


def test_handles_reuse_pool_memory(M):
    """With the library's own pool (the binding's PyTorch allocator switched
    off): handles created one after another reuse the pool's memory; trimming
    hands it back and later handles still work."""
    import torch
    inst = I.small_dense()
    st = I.normal_starts(inst, 128, seed=3)
    cfg = M.default_config(T=50)
    sets = []
    M.use_torch_allocator(False)
    try:
        for k in range(3):
            with M.Instance.from_generated(inst, cfg) as h:
                h.extract_directions(128, Z0=st.Z0)
                h.wait(300)
                sets.append(h.directions())
            if k == 1:
                M.trim_memory()
    finally:
        M.use_torch_allocator(True)
    torch.cuda.synchronize()
    assert all(np.array_equal(sets[0], D) for D in sets[1:]) and sets[0].shape[0] > 0


def test_handle_memory_goes_through_torch(M):
    """By default the binding registers PyTorch's caching allocator with the
    library (mape_set_allocator): a handle's device buffers are counted by
    torch.cuda.memory_allocated() while it lives (at least Z, M, V and the
    two candidate buffers of the extraction) and given back when it closes;
    the results equal those of the library's own pool."""
    import torch
    inst = I.medium_sparse()
    P, T = 2048, 60
    st = I.normal_starts(inst, P, std=0.3, seed=5)
    cfg = M.default_config(T=T)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    with M.Instance.from_generated(inst, cfg) as h:
        h.extract_directions(P, Z0=st.Z0)
        h.wait(300)
        D_torch = h.directions()
        torch.cuda.synchronize()
        held = torch.cuda.memory_allocated() - base
    ldg = M.round16(inst.n)
    cap = P * (T + 1)
    assert held >= 3 * P * inst.d * 4 + 2 * cap * ldg
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    M.use_torch_allocator(False)
    try:
        with M.Instance.from_generated(inst, cfg) as h:
            h.extract_directions(P, Z0=st.Z0)
            h.wait(300)
            D_pool = h.directions()
    finally:
        M.use_torch_allocator(True)
    assert np.array_equal(D_torch, D_pool) and D_torch.shape[0] > 0


@pytest.mark.parametrize("precision", [0, 1])
def test_handle_small(M, precision):
    inst = I.small_dense()
    st = I.normal_starts(inst, 256, seed=2001)
    cfg = M.default_config(T=200, precision=precision)
    with M.Instance.from_generated(inst, cfg) as h:
        h.extract_directions(256, Z0=st.Z0)
        h.wait(300)
        s = h.poll()
        assert s["phase"] == "DONE" and s["error"] == 0
        D = h.directions()
        check_direction_set(inst, D)
        assert np.all(O.minimal_elements(D))
        assert s["directions"] == D.shape[0] <= s["unique"] <= s["candidates"]
        # the int8 copy: the same rows, into a wider caller buffer
        D8 = h.directions_i8()
        assert D8.dtype == np.int8 and np.array_equal(D8.astype(np.int32), D)
        wide = np.full((D.shape[0] + 3, inst.n + 5), 77, dtype=np.int8)
        D8w = h.directions_i8(out=wide)
        assert np.array_equal(D8w, D8) and np.all(wide[:, inst.n:] == 77) and np.all(wide[D.shape[0]:] == 77)
        with pytest.raises(ValueError):
            h.directions_i8(out=np.zeros((max(D.shape[0] - 1, 0), inst.n), dtype=np.int8))
        assert s["kernel_failures"] == 0
        h.augment(inst.xbar[None, :])
        h.wait(300)
        x, fx = h.solution()
        xo, fo, mo = O.augment(inst.A, inst.b, inst.l, inst.u, inst.Q, inst.c, None, D, inst.xbar)
        assert fx == fo and np.array_equal(x, xo)
        assert h.poll()["aug_iters"] == len(mo) + 1
        # reuse: a new objective on the same direction set (§1, reusability)
        rng = np.random.default_rng(5)
        c2 = rng.integers(-10, 11, size=inst.n).astype(np.int32)
        h.augment(inst.xbar[None, :], f=(inst.Q, c2, None))
        h.wait(300)
        x2, f2 = h.solution()
        xo2, fo2, _ = O.augment(inst.A, inst.b, inst.l, inst.u, inst.Q, c2, None, D, inst.xbar)
        assert f2 == fo2 and np.array_equal(x2, xo2)


def test_handle_errors(M):
    inst = I.small_dense()
    bad_B = inst.B.copy()
    bad_B[-1, 0] += 1
    with pytest.raises(M.MapeError) as e:
        M.Instance(inst.A, inst.b, inst.l, inst.u, inst.Q, inst.c, None, bad_B)
    assert e.value.code == -3
    with M.Instance.from_generated(inst, M.default_config(T=5, precision=0)) as h:
        with pytest.raises(M.MapeError) as e:
            h.augment(inst.xbar[None, :])           # no direction set yet
        assert e.value.code == -10
        h.extract_directions(64, Z0=I.normal_starts(inst, 64, seed=1).Z0)
        h.wait(60)
        x = inst.xbar.copy()
        x[0] += 1                                    # breaks A x = b
        with pytest.raises(M.MapeError) as e:
            h.augment(x[None, :])
        assert e.value.code == -5


def test_handle_projects_g0_starts(M):
    """Starts given as samples g (a2: z0 = (B^T B)^{-1} B^T g inside the
    handle, the projection formed at the first such call and kept): two calls
    with G0 on one handle and one call with the stage entry point's z0 on
    another return the same direction set (the projection's numerics are
    checked against the oracle in the stage tests)."""
    import torch
    inst = I.small_dense()
    P = 256
    G0 = I.uniform_samples(inst, P, seed=11).G0
    cfg = M.default_config(T=80)
    Z = M.project_starts(torch.from_numpy(inst.B.astype(np.int32)).cuda(),
                         torch.from_numpy(G0).cuda()).cpu().numpy()
    sets = []
    with M.Instance.from_generated(inst, cfg) as h:
        for _ in range(2):
            h.extract_directions(P, G0=G0)
            h.wait(300)
            sets.append(h.directions())
    with M.Instance.from_generated(inst, cfg) as h:
        h.extract_directions(P, Z0=Z)
        h.wait(300)
        sets.append(h.directions())
    check_direction_set(inst, sets[0])
    assert all(np.array_equal(sets[0], D) for D in sets[1:])


def test_handle_initial_solutions_and_multistart_augmentation(M):
    """Eq. (4) on the handle gives distinct, exactly feasible starts S0; the
    multi-start augmentation from all of them (§3.3) gives, per start, the
    oracle's Algorithm 1 result on the same direction set, and the best of
    them is reported."""
    inst = I.small_dense()
    rng = np.random.default_rng(9)
    X0 = rng.uniform(inst.l, inst.u, size=(256, inst.n)).astype(np.float32)
    X0[:64] = inst.xbar + rng.uniform(-0.45, 0.45, size=(64, inst.n))
    cfg = M.default_config(T=200, precision=1)
    with M.Instance.from_generated(inst, cfg) as h:
        S0 = h.initial_solutions(X0, T=400, period=10)
        assert S0.shape[0] >= 1
        S0i = S0.astype(np.int64)
        assert np.all(S0i @ inst.A.T.astype(np.int64) == inst.b)
        assert np.all((S0i >= inst.l) & (S0i <= inst.u))
        assert np.unique(S0i, axis=0).shape[0] == S0.shape[0]
        S0 = S0[:16]
        h.extract_directions(256, Z0=I.normal_starts(inst, 256, seed=2001).Z0)
        h.wait(300)
        D = h.directions()
        h.augment(S0)
        h.wait(300)
        X, F = h.solutions(S0.shape[0])
        for k in range(S0.shape[0]):
            xo, fo, _ = O.augment(inst.A, inst.b, inst.l, inst.u, inst.Q, inst.c, None, D, S0[k])
            assert F[k] == fo and np.array_equal(X[k], xo)
        x, fx = h.solution()
        assert fx == F.min()


def test_handle_with_linear_inequalities(M):
    """§3.4: the small instance with three inequalities G x >= h, run as its
    equality form with slacks: every direction lies in Ker([A 0; G -I]), the
    augmentation equals the oracle's Algorithm 1 on that set, and the final x
    satisfies G x >= h."""
    inst = I.small_dense()
    rng = np.random.default_rng(4)
    G = rng.choice([-1, 0, 1], p=[0.15, 0.7, 0.15], size=(3, inst.n))
    h = G @ inst.xbar.astype(np.int64) - rng.integers(0, 4, size=3)
    e = M.inequality_extension(inst, G, h)
    assert np.max(e.u - e.l) <= 127  # direction entries are stored as int8
    cfg = M.default_config(T=200, precision=1)
    with M.Instance.from_generated(e, cfg) as hd:
        hd.extract_directions(256, Z0=I.normal_starts(e, 256, seed=2001).Z0)
        hd.wait(300)
        D = hd.directions()
        check_direction_set(e, D)
        hd.augment(e.xbar[None, :])
        hd.wait(300)
        x, fx = hd.solution()
    xo, fo, _ = O.augment(e.A, e.b, e.l, e.u, e.Q, e.c, None, D, e.xbar)
    assert fx == fo and np.array_equal(x, xo)
    xs = x[: inst.n].astype(np.int64)
    assert np.all(G @ xs >= h)
    assert np.array_equal(inst.A.astype(np.int64) @ xs, inst.b)
    assert fx <= O.f_value(inst.Q, inst.c, None, inst.xbar)


def test_handle_on_general_A_with_computed_basis(M):
    """A general A (not [C | I]) with the LLL-reduced kernel basis from
    mape_kernel_basis (Lemma 3.1, Appendix A): the extracted directions pass
    C1, C4 and minimality, and augmentation equals the oracle's Algorithm 1."""
    import dataclasses
    inst = I.general_instance(n=16, m=5, seed=11)
    inst = dataclasses.replace(inst, B=M.kernel_basis(inst.A))
    assert np.abs(inst.B).max() <= 256  # exact in BF16
    cfg = M.default_config(T=300, precision=1)
    with M.Instance.from_generated(inst, cfg) as h:
        h.extract_directions(512, Z0=I.normal_starts(inst, 512, seed=3).Z0)
        h.wait(300)
        D = h.directions()
        check_direction_set(inst, D)
        assert np.all(O.minimal_elements(D))
        h.augment(inst.xbar[None, :])
        h.wait(300)
        x, fx = h.solution()
    xo, fo, _ = O.augment(inst.A, inst.b, inst.l, inst.u, inst.Q, inst.c, None, D, inst.xbar)
    assert fx == fo and np.array_equal(x, xo)
