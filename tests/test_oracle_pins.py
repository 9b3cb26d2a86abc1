"""Pins for the CPU oracle: each test checks it against something other than
itself -- a hand-evaluated example, a textbook Graver basis, a closed form, a
library routine (torch.optim.Adam), finite differences, an invariant or brute
force on tiny inputs.  CPU only."""
import itertools
import os

import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            rows.setdefault(key, []).append([float(v) for v in vals])
    return rows


# --- §3.1, Theorem 3.2 ------------------------------------------------------

@pytest.mark.parametrize("make", [I.small_dense, I.medium_sparse, I.tiny_graver_case])
def test_closed_form_basis_is_kernel(make):
    inst = make()
    assert O.kernel_basis_check(inst.A, inst.B)
    bad = inst.B.copy()
    bad[-1, 0] += 1
    assert not O.kernel_basis_check(inst.A, bad)
    assert np.all(inst.A @ inst.xbar.astype(np.int64) == inst.b)
    assert np.all(inst.xbar >= inst.l) and np.all(inst.xbar <= inst.u)


def test_projection_is_inverse_map():
    """z = (B^T B)^{-1} B^T g returns w exactly (to fp64 rounding) when g = B w."""
    inst = I.small_dense()
    rng = np.random.default_rng(0)
    W = rng.integers(-4, 5, size=(50, inst.d))
    G = W @ inst.B.T
    Z = O.project_to_coordinates(inst.B, G)
    np.testing.assert_allclose(Z, W, atol=1e-9)
    # for a generic g the residual is orthogonal to the range of B
    G0 = I.uniform_samples(inst, 40, seed=3).G0
    Z = O.project_to_coordinates(inst.B, G0)
    resid = G0.astype(np.float64) - Z @ inst.B.T
    np.testing.assert_allclose(resid @ inst.B, 0.0, atol=1e-9)


# --- §3.2, Eq. (3) ------------------------------------------------------------

def test_phi_and_grad_hand_example():
    gold = _read_golden("phi_hand_example.txt")
    B = np.array(gold["B"])
    z = np.array(gold["z"])
    assert O.phi(B, z, 0.85, 1.0)[0] == pytest.approx(gold["phi"][0][0], abs=1e-12)
    np.testing.assert_allclose(O.phi_grad(B, z, 0.85, 1.0)[0], gold["grad"][0], atol=1e-12)


def test_phi_at_integer_points_is_l1_norm():
    inst = I.small_dense()
    rng = np.random.default_rng(1)
    Z = rng.integers(-3, 4, size=(64, inst.d)).astype(np.float64)
    Z[np.abs(Z).max(axis=1) == 0, 0] = 1.0
    expect = np.abs(Z @ inst.B.T).sum(axis=1)
    np.testing.assert_allclose(O.phi(inst.B, Z, 0.85, 1.0), expect, rtol=0, atol=1e-12)
    # the integrality term has zero gradient at integers; with ||z||_inf >= 1
    # the gradient is B^T sign(Bz) alone
    g = O.phi_grad(inst.B, Z, 0.85, 1.0)
    np.testing.assert_allclose(g, np.sign(Z @ inst.B.T) @ inst.B, atol=1e-12)


def test_phi_at_origin_is_infinite():
    B = np.eye(3)
    assert np.isinf(O.phi(B, np.zeros((1, 3)), 0.85, 1.0)[0])
    assert np.all(O.phi_grad(B, np.zeros((1, 3)), 0.85, 1.0) == 0)


def _away_from_kinks(B, Z, tol):
    Y = Z @ np.asarray(B, np.float64).T
    fr = np.abs(Z - np.rint(Z))
    a = np.sort(np.abs(Z), axis=1)
    zinf = a[:, -1]
    return ((np.abs(Y).min(axis=1) > tol) & (fr.min(axis=1) > tol)
            & (np.abs(zinf - 1.0) > tol) & (a[:, -1] - a[:, -2] > tol))


@pytest.mark.parametrize("scale", [0.4, 3.0])
def test_grad_matches_central_differences(scale):
    """Central differences of Phi alone (no gradient formula) at points away
    from the kinks of |.|, floor/ceil and the max; scale 0.4 puts most points
    inside ||z||_inf < 1 so the inverse-norm term is active."""
    inst = I.small_dense()
    rng = np.random.default_rng(2)
    Z = rng.uniform(-scale, scale, size=(400, inst.d))
    Z = Z[_away_from_kinks(inst.B, Z, 1e-3)][:40]
    assert Z.shape[0] >= 10
    h = 1e-7
    fd = np.zeros_like(Z)
    for j in range(inst.d):
        e = np.zeros(inst.d)
        e[j] = h
        fd[:, j] = (O.phi(inst.B, Z + e, 0.85, 1.0) - O.phi(inst.B, Z - e, 0.85, 1.0)) / (2 * h)
    np.testing.assert_allclose(O.phi_grad(inst.B, Z, 0.85, 1.0), fd, rtol=1e-6, atol=1e-5)
    if scale < 1:
        assert (np.abs(Z).max(axis=1) < 1).any()


def test_adam_first_step_moves_by_lr_sign():
    rng = np.random.default_rng(3)
    z = rng.standard_normal((5, 7))
    grad = rng.standard_normal((5, 7))
    z1, m1, v1 = O.adam_update(z, np.zeros_like(z), np.zeros_like(z), grad, 1, 0.003)
    np.testing.assert_allclose(z1 - z, -0.003 * np.sign(grad), rtol=1e-6)


def test_adam_matches_torch_optimizer():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    z0 = rng.standard_normal((6, 5))
    p = torch.nn.Parameter(torch.tensor(z0, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=0.003, betas=(0.9, 0.999), eps=1e-8)
    z, m, v = z0.copy(), np.zeros_like(z0), np.zeros_like(z0)
    for t in range(1, 26):
        grad = rng.standard_normal(z0.shape)
        p.grad = torch.tensor(grad)
        opt.step()
        z, m, v = O.adam_update(z, m, v, grad, t, 0.003)
    np.testing.assert_allclose(z, p.detach().numpy(), rtol=1e-12, atol=1e-14)


# --- Algorithm 2: rounding, C1, C4, canonical sign ----------------------------

def test_rounding_breaks_ties_to_even():
    B = np.eye(4, dtype=np.int64)
    zhat, g = O.round_and_map(B, np.array([[0.5, 1.5, -2.5, 2.4999]]))
    assert zhat.tolist() == [[0, 2, -2, 2]]
    assert g.tolist() == [[0, 2, -2, 2]]


def test_bound_and_kernel_conditions():
    A = np.array([[1, 1, 1]])
    l = np.array([0, 0, 0])
    u = np.array([2, 1, 3])
    G = np.array([[2, -1, -1], [3, 0, -3], [1, 1, 0], [0, 1, -1]])
    assert O.bound_consistent(G, l, u).tolist() == [True, False, True, True]
    assert O.kernel_condition(A, G).tolist() == [True, True, False, True]


def test_canonical_sign_and_conformal_order():
    assert O.canonical_sign([0, -2, 1]).tolist() == [0, 2, -1]
    assert O.canonical_sign([0, 3, -1]).tolist() == [0, 3, -1]
    assert O.conformal_leq([1, 0, -1], [2, 1, -1])
    assert not O.conformal_leq([1, 0, -1], [2, 1, 1])     # sign conflict
    assert not O.conformal_leq([1, 0, -2], [2, 1, -1])    # too long
    assert O.conformal_leq([0, 0, 0], [1, -1, 0])


# --- Graver basis: textbook cases and the definition ---------------------------

def test_graver_basis_textbook_cases():
    ones3 = O.graver_basis_box(np.array([[1, 1, 1]]), 3)
    assert sorted(map(tuple, ones3.tolist())) == [(0, 1, -1), (1, -1, 0), (1, 0, -1)]
    assert O.graver_basis_box(np.array([[1, 2]]), 4).tolist() == [[2, -1]]
    assert O.graver_basis_box(np.array([[2, -3]]), 4).tolist() == [[3, 2]]
    gold = _read_golden("twisted_cubic_graver.txt")
    A = np.array(gold["A"], dtype=np.int64)
    expect = sorted(tuple(int(v) for v in g) for g in gold["g"])
    got = sorted(map(tuple, O.graver_basis_box(A, 3).tolist()))
    assert got == expect
    for g in expect:
        assert O.is_graver_element(A, g)
    assert not O.is_graver_element(A, (2, -4, 2, 0))   # twice an element
    assert not O.is_graver_element(A, (1, -1, 0, 0))   # not in the kernel


def _conformal_decomposition_exists(v, basis):
    """Graver property: every kernel vector is a sum of basis elements (either
    sign) each conformal to it."""
    v = np.asarray(v, np.int64)
    while np.any(v):
        for g in basis:
            for s in (1, -1):
                if O.conformal_leq(s * g, v):
                    v = v - s * g
                    break
            else:
                continue
            break
        else:
            return False
    return True


def test_tiny_graver_basis_decomposes_the_kernel_box():
    inst = I.tiny_graver_case()
    basis = O.graver_basis_box(inst.A, 3)
    assert basis.shape[0] > 0
    kernel = O.kernel_box(inst.A, 3)
    for v in kernel:
        assert _conformal_decomposition_exists(v, basis)
    for g in basis:
        assert O.is_graver_element(inst.A, g)


def test_minimal_elements_agrees_with_enumeration():
    inst = I.tiny_graver_case()
    kernel = O.kernel_box(inst.A, 3)
    canon = np.unique(np.array([O.canonical_sign(g) for g in kernel]), axis=0)
    mins = canon[O.minimal_elements(canon)]
    assert sorted(map(tuple, mins.tolist())) == sorted(map(tuple, O.graver_basis_box(inst.A, 3).tolist()))
    # a selection of rows is judged against the whole set, as in the full mask
    full = O.minimal_elements(canon)
    for rows in ([0], [3, 1, 2], list(range(canon.shape[0] - 1, -1, -2))):
        assert np.array_equal(O.minimal_elements(canon, rows=rows), full[rows])


def test_extraction_on_tiny_instance_returns_graver_elements():
    """Algorithm 2 with many starts: every returned direction is a true Graver
    element (checked against the enumerated basis), lies in the kernel and in
    the bound box; most of the basis is found."""
    inst = I.tiny_graver_case()
    st = I.normal_starts(inst, 2048, seed=5)
    res = O.parallel_extraction(inst.A, inst.B, inst.l, inst.u, st.Z0, T=150)
    D = res["directions"]
    basis = set(map(tuple, O.graver_basis_box(inst.A, 3).tolist()))
    assert D.shape[0] > 0
    assert set(map(tuple, D.tolist())) <= basis
    assert np.all(O.kernel_condition(inst.A, D))
    assert np.all(O.bound_consistent(D, inst.l, inst.u))
    assert D.shape[0] >= 0.5 * len(basis)


# --- Algorithm 1 and Proposition 2.1 ------------------------------------------

def test_f_value_hand_example():
    Q = np.array([[2, -1], [-1, 0]])
    c = np.array([3, -4])
    w = np.array([1, 2])
    x = np.array([2, -1])
    # x^T Q x = 2*4 + 2*(-1)*2*(-1) + 0 = 8 + 4 = 12; c^T x = 6 + 4 = 10;
    # sum w x^4 = 16 + 2 = 18
    assert O.f_value(Q, c, w, x) == 40
    assert O.f_value(Q, c, None, x) == 22


def test_step_lengths_by_bounds():
    l = np.array([0, 0, -3])
    u = np.array([10, 4, 3])
    assert O.feasible_step_lengths(l, u, [1, 1, 0], [2, 1, -1]) == [1, 2, 3]
    assert O.feasible_step_lengths(l, u, [10, 1, 0], [1, 0, 0]) == []


def _box_points(inst):
    import itertools
    rng = [range(int(a), int(b) + 1) for a, b in zip(inst.l, inst.u)]
    pts = np.array(list(itertools.product(*rng)), dtype=np.int64)
    return pts[np.all(pts @ inst.A.T.astype(np.int64) == inst.b, axis=1)]


@pytest.mark.parametrize("seed", [11, 12, 13, 14])
def test_prop21_graver_augmentation_reaches_optimum(seed):
    """Proposition 2.1: for separable convex f the Graver basis is a test set,
    so Algorithm 1 from any feasible point reaches the global minimum (found
    here by enumerating S)."""
    inst = I.tiny_graver_case(seed=seed)
    rng = np.random.default_rng(seed)
    Q = np.diag(rng.integers(0, 4, size=inst.n))
    c = rng.integers(-6, 7, size=inst.n)
    w = rng.integers(0, 2, size=inst.n)
    basis = O.graver_basis_box(inst.A, 3)
    S = _box_points(inst)
    best = min(O.f_value(Q, c, w, x) for x in S)
    for x0 in S[rng.choice(S.shape[0], size=min(6, S.shape[0]), replace=False)]:
        x, fx, moves = O.augment(inst.A, inst.b, inst.l, inst.u, Q, c, w, basis, x0)
        assert fx == best
        assert O.in_feasible_region(inst.A, inst.b, inst.l, inst.u, x)


def test_augment_moves_keep_feasibility_and_strictly_decrease():
    inst = I.small_dense()
    st = I.normal_starts(inst, 256, seed=2001)
    res = O.parallel_extraction(inst.A, inst.B, inst.l, inst.u, st.Z0, T=60)
    D = res["directions"]
    x = inst.xbar.astype(np.int64)
    fx = O.f_value(inst.Q, inst.c, None, x)
    xf, ff, moves = O.augment(inst.A, inst.b, inst.l, inst.u, inst.Q, inst.c, None, D, x)
    assert len(moves) > 0
    prev = fx
    for k, s, lam, fval in moves:
        x = x + lam * s * D[k]
        assert O.in_feasible_region(inst.A, inst.b, inst.l, inst.u, x)
        assert O.f_value(inst.Q, inst.c, None, x) == fval < prev
        prev = fval
    assert np.array_equal(x, xf)


# --- Eq. (4): initial feasible solutions ----------------------------------------

def test_init_objective_hand_example():
    """A = [1 2], b = 3: at x = (0.5, 1.25) A x = b, so only the integrality
    term remains, lambda3 (0.5*0.5 + 0.25*0.75) = 0.1 * 0.4375; at the integer
    feasible point (1, 1) the objective is 0, its global minimum."""
    A, b = np.array([[1, 2]]), np.array([3])
    f = O.init_objective(A, b, np.array([[0.5, 1.25], [1.0, 1.0], [0.0, 0.0]]), 0.1)
    assert f[0] == pytest.approx(0.04375, abs=1e-15)
    assert f[1] == 0.0
    assert f[2] == pytest.approx(9.0)


def test_init_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    A = rng.integers(-3, 4, size=(4, 9))
    b = rng.integers(-5, 6, size=4)
    X = rng.uniform(-4, 4, size=(6, 9))
    X[np.abs(X - np.rint(X)) < 0.05] += 0.1  # stay off the kinks of the integrality term
    G = O.init_gradient(A, b, X, 0.1)
    h = 1e-6
    for j in range(9):
        E = np.zeros_like(X)
        E[:, j] = h
        fd = (O.init_objective(A, b, X + E, 0.1) - O.init_objective(A, b, X - E, 0.1)) / (2 * h)
        np.testing.assert_allclose(G[:, j], fd, rtol=1e-6, atol=1e-5)


def test_projected_adam_first_step_and_box():
    """First Adam step moves every coordinate by lr against the gradient sign;
    the projection keeps the iterate in [l, u]."""
    x = np.array([[0.0, 5.0, 2.5]])
    g = np.array([[1.0, -3.0, 0.5]])
    l, u = np.array([0, 0, 0]), np.array([5, 5, 5])
    z, m, v = O.projected_adam_update(x, np.zeros_like(x), np.zeros_like(x), g, 1, 0.003, l, u)
    np.testing.assert_allclose(z, [[0.0, 5.0, 2.497]], atol=1e-9)  # 0 - 0.003 clipped to 0, 5 + 0.003 to 5


def test_feasible_roundings_agree_with_enumeration():
    inst = I.tiny_graver_case()
    pts = np.array(list(itertools.product(*[range(lo, hi + 1) for lo, hi in zip(inst.l, inst.u)])), dtype=np.int64)
    feas = pts[np.all(pts @ inst.A.T.astype(np.int64) == inst.b, axis=1)]
    assert len(feas) > 0
    expect = {tuple(x) for x in feas}
    assert O.feasible_roundings(inst.A, inst.b, inst.l, inst.u, feas) == expect
    rng = np.random.default_rng(1)
    noisy = feas + rng.uniform(-0.49, 0.49, size=feas.shape)
    assert O.feasible_roundings(inst.A, inst.b, inst.l, inst.u, noisy) == expect
    # every infeasible box point is rejected
    other = pts[~np.all(pts @ inst.A.T.astype(np.int64) == inst.b, axis=1)]
    assert O.feasible_roundings(inst.A, inst.b, inst.l, inst.u, other) == set()


def test_initial_solutions_identity_system_reaches_b():
    """A = I, b integer in the box: Eq. (4) is ||x - b||^2 plus the integrality
    term, whose unique minimiser is b; projected Adam from the box reaches it
    and the only feasible rounding is b."""
    n = 5
    A = np.eye(n, dtype=np.int64)
    b = np.array([1, -2, 0, 3, -1])
    l, u = np.full(n, -4), np.full(n, 4)
    X0 = np.random.default_rng(2).uniform(-4, 4, size=(16, n))
    X, found = O.initial_solutions(A, b, l, u, X0, T=3000, lr=0.01)
    assert found == {tuple(b)}
    assert np.max(np.abs(X - b)) < 0.1
    assert np.all((X >= l) & (X <= u))


def test_initial_solutions_on_tiny_instance_are_feasible():
    inst = I.tiny_graver_case()
    X0 = np.random.default_rng(4).uniform(inst.l, inst.u, size=(64, inst.n))
    _, found = O.initial_solutions(inst.A, inst.b, inst.l, inst.u, X0, T=1500, lr=0.01)
    assert len(found) > 0
    for x in found:
        x = np.array(x)
        assert np.array_equal(inst.A.astype(np.int64) @ x, inst.b)
        assert np.all((x >= inst.l) & (x <= inst.u))


# --- §3.4: linear inequalities through slack variables ---------------------------

def _tiny_with_inequality():
    inst = I.tiny_graver_case()
    G = np.array([[1, 1, 0, 0, 0, 0], [0, 0, 1, -1, 0, 1]])
    h = G @ inst.xbar.astype(np.int64) - np.array([1, 2])  # xbar satisfies both with slack 1 and 2
    return inst, G, h


def test_inequality_extension_kernel_basis():
    """Corollary 3.3: A' [B; GB] = 0, and every kernel element of
    A' = [A 0; G -I] in a box is an integer combination of [B; GB]
    (enumeration on the 6-variable instance with two inequalities)."""
    inst, G, h = _tiny_with_inequality()
    A2, b2, l2, u2, B2 = O.inequality_extension(inst.A, inst.b, inst.l, inst.u, G, h, inst.B)
    assert A2.shape == (4, 8) and B2.shape == (8, 4)
    assert np.all(A2 @ B2 == 0)
    x2 = np.concatenate([inst.xbar, G @ inst.xbar - h])
    assert np.array_equal(A2 @ x2, b2) and np.all((x2 >= l2) & (x2 <= u2))
    K = O.kernel_box(A2, 2)
    assert len(K) > 0
    assert all(O.lattice_contains(B2, g) for g in K)
    # a vector outside the kernel is not in the lattice
    assert not O.lattice_contains(B2, np.eye(8, dtype=np.int64)[0])


def test_inequality_extension_slack_bounds():
    """u' of a slack is its largest value over the box; an inequality that no
    point of the box satisfies is refused."""
    A = np.array([[1, 1]])
    B = np.array([[1], [-1]])
    G = np.array([[2, -1]])
    l, u = np.array([0, 0]), np.array([3, 4])
    _, _, l2, u2, _ = O.inequality_extension(A, [2], l, u, G, [1], B)
    assert l2[-1] == 0 and u2[-1] == 2 * 3 - 0 - 1
    with pytest.raises(ValueError):
        O.inequality_extension(A, [2], l, u, G, [7], B)


# --- Lemma 3.1 / Theorem 3.2 (kernel basis of a general A) and Appendix A (LLL) ---

def _same_lattice(B1, B2):
    B1 = np.asarray(B1, np.int64)
    B2 = np.asarray(B2, np.int64)
    return all(O.lattice_contains(B1, B2[:, j]) for j in range(B2.shape[1])) and \
        all(O.lattice_contains(B2, B1[:, j]) for j in range(B1.shape[1]))


def _det_exact(M):
    """Determinant of an integer matrix by fraction-free (Bareiss) elimination."""
    M = [[int(v) for v in row] for row in M]
    n, sign, prev = len(M), 1, 1
    for k in range(n - 1):
        if M[k][k] == 0:
            sw = next((r for r in range(k + 1, n) if M[r][k] != 0), None)
            if sw is None:
                return 0
            M[k], M[sw] = M[sw], M[k]
            sign = -sign
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                M[i][j] = (M[i][j] * M[k][k] - M[i][k] * M[k][j]) // prev
        prev = M[k][k]
    return sign * M[n - 1][n - 1]


def test_hnf_kernel_basis_is_a_kernel_basis():
    """A K = (H | 0) with K unimodular (|det K| = 1); B = K's last d columns
    spans the same lattice as the closed-form basis [I; -C] of A = [C | I]."""
    assert _det_exact([[2, 1], [7, 4]]) == 1 and _det_exact([[1, 2, 3], [4, 5, 6], [7, 8, 10]]) == -3
    for inst in (I.tiny_graver_case(), I.small_dense()):
        A = inst.A.astype(np.int64)
        B, K = O.hnf_kernel_basis(A)
        AK = np.array(A.astype(object).dot(K), dtype=object)
        m = A.shape[0]
        assert all(v == 0 for v in AK[:, m:].ravel())
        assert all(AK[i, j] == 0 for i in range(m) for j in range(i + 1, m))  # H lower triangular
        assert abs(_det_exact(K.tolist())) == 1
        assert _same_lattice(np.array(B, dtype=np.int64), inst.B)


def test_hnf_kernel_basis_general_matrix_contains_every_kernel_element():
    """A general full-row-rank A (not of the form [C | I]): every kernel
    element in a box is an integer combination of the HNF basis."""
    A = np.array([[2, 3, -1, 4], [1, -2, 5, 0]])
    B, _ = O.hnf_kernel_basis(A)
    B = np.array(B, dtype=np.int64)
    assert B.shape == (4, 2) and np.all(A @ B == 0)
    for g in O.kernel_box(A, 6):
        assert O.lattice_contains(B, g)
    with pytest.raises(ValueError):
        O.hnf_kernel_basis(np.array([[1, 2, 3], [2, 4, 6]]))


def test_lll_hand_example_and_conditions():
    """(1,0), (7,1) size-reduces to (1,0), (0,1); every output satisfies
    Appendix A's conditions and spans the input's lattice."""
    out = np.array(O.lll_reduce(np.array([[1, 7], [0, 1]])), dtype=np.int64)
    assert np.array_equal(out, np.array([[1, 0], [0, 1]]))
    rng = np.random.default_rng(8)
    for _ in range(5):
        B = rng.integers(-20, 21, size=(6, 4))
        if np.linalg.matrix_rank(B) < 4:
            continue
        R = O.lll_reduce(B)
        assert O.lll_conditions(R) == (True, True)
        assert _same_lattice(np.array(R, dtype=np.int64), B)
    # the first reduced vector of a reduced basis is short: within
    # 2^((d-1)/2) of the shortest kernel element of the tiny instance
    inst = I.tiny_graver_case()
    Bh, _ = O.hnf_kernel_basis(inst.A)
    R = np.array(O.lll_reduce(Bh), dtype=np.int64)
    shortest = min(np.linalg.norm(g) for g in O.kernel_box(inst.A, 2))
    assert np.linalg.norm(R[:, 0]) <= 2 ** ((R.shape[1] - 1) / 2) * shortest + 1e-9


# --- Algorithm 2: the collection step, by hand -------------------------------

def test_collect_hand_example():
    """A = [1 1], B = [1; -1] (Ker_Z(A) is spanned by (1, -1)), box [0, 2] so
    that C4 admits |g_i| <= 2.  Worked by hand: z = 0.4 and 0.5 round to 0 (ties
    to even) and give g = 0 (dropped); z = 1.6, 2.5 and -2.5 round to 2, 2 and
    -2 and give (2, -2) up to sign; z = -0.7 gives (-1, 1), canonically (1, -1);
    z = 3.2 gives (3, -3), outside the box.  With B = [1; 0], which is not in
    the kernel, A g = 1 != 0 and C1 drops everything."""
    A = np.array([[1, 1]])
    l, u = np.array([0, 0]), np.array([2, 2])
    Z = np.array([[0.4], [0.5], [1.6], [2.5], [-2.5], [-0.7], [3.2]])
    assert O.collect(A, np.array([[1], [-1]]), l, u, Z) == {(2, -2), (1, -1)}
    assert O.collect(A, np.array([[1], [0]]), l, u, Z) == set()
    # the bound of C4 is inclusive: span 1 keeps (1, -1) and drops (2, -2)
    assert O.collect(A, np.array([[1], [-1]]), l, np.array([1, 1]), Z) == {(1, -1)}


def test_sort_directions_is_tuple_order():
    rng = np.random.default_rng(4)
    G = rng.integers(-3, 4, size=(200, 5))
    expect = sorted(tuple(int(v) for v in r) for r in G)
    assert [tuple(int(v) for v in r) for r in O.sort_directions(G)] == expect
    assert O.sort_directions(np.zeros((0, 5), np.int64)).shape == (0, 5)


def test_egcd_bezout_against_math_gcd():
    import math
    rng = np.random.default_rng(6)
    pairs = [(0, 0), (0, 7), (7, 0), (-12, 18), (18, -12), (1, 1)]
    pairs += [(int(a), int(b)) for a, b in rng.integers(-10 ** 6, 10 ** 6, size=(300, 2))]
    for a, b in pairs:
        g, x, y = O._egcd(a, b)
        assert g == math.gcd(a, b) and x * a + y * b == g


def test_lll_conditions_reject_unreduced_bases():
    """Appendix A's two conditions, each violated on its own, by hand.
    Columns (1,0), (7,1): mu_21 = 7 > 1/2, not size-reduced; the
    Gram-Schmidt norms are 1 and 1, so the exchange condition holds.
    Columns (3,0), (0,1): mu_21 = 0, but ||b1*||^2 = 9 > 2 ||b2*||^2 = 2.
    Columns (2,0), (1,2): mu_21 = 1/2 exactly (allowed) and norms 4 <= 2 * 4.
    Columns (2,0), (1,1): mu_21 = 1/2, but 4 > 2 * 1.  Columns (1,0), (1,1):
    mu_21 = 1 > 1/2, norms 1 and 1."""
    def cols(*vs):
        return np.array(vs, dtype=np.int64).T
    assert O.lll_conditions(cols((1, 0), (7, 1))) == (False, True)
    assert O.lll_conditions(cols((3, 0), (0, 1))) == (True, False)
    assert O.lll_conditions(cols((2, 0), (1, 2))) == (True, True)
    assert O.lll_conditions(cols((2, 0), (1, 1))) == (True, False)
    assert O.lll_conditions(cols((1, 0), (1, 1))) == (False, True)
    assert O.lll_conditions(cols((1, 0), (0, 1))) == (True, True)
    # a three-column case where only a non-adjacent coefficient (mu_31) is
    # too large: (1,0,0), (0,1,0), (5,0,1)
    assert O.lll_conditions(cols((1, 0, 0), (0, 1, 0), (5, 0, 1))) == (False, True)
    # and one where only the second pair fails the exchange test:
    # (1,0,0), (0,3,0), (0,0,1): norms 1, 9, 1 and 9 > 2
    assert O.lll_conditions(cols((1, 0, 0), (0, 3, 0), (0, 0, 1))) == (True, False)


def test_in_feasible_region_rejects_each_violation():
    """x in S needs A x = b and l <= x <= u; each part alone must fail.
    A = [1 1 0; 0 1 1], b = (2, 3), box [0, 3]: (1, 1, 2) is feasible;
    (1, 1, 1) is in the box with A x = (2, 2) != b; (-1, 3, 0) has
    A x = (2, 3) = b but leaves the box below, (4, -2, 5) above and below."""
    A = np.array([[1, 1, 0], [0, 1, 1]])
    b = np.array([2, 3])
    l, u = np.zeros(3, np.int64), np.full(3, 3)
    assert O.in_feasible_region(A, b, l, u, [1, 1, 2])
    assert not O.in_feasible_region(A, b, l, u, [1, 1, 1])
    assert not O.in_feasible_region(A, b, l, u, [-1, 3, 0])
    assert not O.in_feasible_region(A, b, l, u, [4, -2, 5])
    assert O.in_feasible_region(A, b, l, u, [2, 0, 3])
    # one row of A x = b wrong, the other right
    assert not O.in_feasible_region(A, b, l, u, [0, 2, 2])   # A x = (2, 4)
    assert not O.in_feasible_region(A, b, l, u, [0, 1, 2])   # A x = (1, 3)
