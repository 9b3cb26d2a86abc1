"""CPU oracle for MAPE's data-parallel hot path (test infrastructure only).

This file is test infrastructure.  Only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import it; the product path never
calls it.  It shares no code with the CUDA path: both sides receive the same
arrays from the seeded input generator and compute on their own.

Everything is plain numpy in float64 (continuous stages) and int64 (integer
stages), restating the paper's definitions and algorithm steps in the
paper's order.  A library matmul serves as a step where the paper writes a
matrix product; nothing is blocked, fused or reordered.

Notation follows the paper: B is the n x d kernel-lattice basis (Theorem 3.2,
§3.1), z in R^d a coordinate vector, g = B z a direction, l/u the bounds, and
starts are rows (one start per row of Z).

Readings of points the paper leaves open (each also listed in the design
notes of the repository):
  * gradient of the floor/ceil product: floor and ceil are treated as
    locally constant, so d/dz (z-floor z)(ceil z-z) = ceil z + floor z - 2z;
  * subgradient of |y| at 0 is 0 (sign(0) = 0);
  * gradient of max{1/||z||_inf - 1, 0}: zero when ||z||_inf >= 1, else
    -sign(z_k)/||z||_inf^2 at k = the FIRST index attaining max |z_j|; zero
    at z = 0 exactly (where Phi is +inf);
  * Adam: the textbook update with bias correction (Kingma & Ba), constants
    beta1 = 0.9, beta2 = 0.999, eps = 1e-8; the loss is summed over starts,
    so every start is an independent problem;
  * rounding to the nearest integer breaks ties to even;
  * the collected set excludes g = 0 and stores each direction once up to
    sign, with the first nonzero entry positive;
  * Algorithm 1 tries both +g and -g for every stored direction, with
    lambda >= 1; among optimal moves it takes the lowest direction index (in
    the sorted direction list), +g before -g, then the smallest lambda;
  * Eq. (4): x in [l, u] is kept by projecting (clipping) after every Adam
    step; the starts are clipped into the box first; the rounded iterate is
    collected when it is exactly feasible for model (1), after every
    `period`-th step like Algorithm 2's collection; lambda3 = 0.1 (§4).
"""
from __future__ import annotations

import itertools

import numpy as np

# ---------------------------------------------------------------------------
# §3.1: Theorem 3.2 and the inverse map z = (B^T B)^{-1} B^T g


def kernel_basis_check(A, B):
    """True iff A B = 0 exactly (condition for Theorem 3.2)."""
    return bool(np.all(np.asarray(A, np.int64) @ np.asarray(B, np.int64) == 0))


def project_to_coordinates(B, G0):
    """z = (B^T B)^{-1} B^T g for every sample row g (§3.2, Algorithm 2).

    Solved as the normal equations with a dense fp64 solve; B^T B is symmetric
    positive definite because B has full column rank.
    """
    Bf = np.asarray(B, np.float64)
    H = Bf.T @ Bf
    R = np.asarray(G0, np.float64) @ Bf            # rows: (B^T g)^T
    return np.linalg.solve(H, R.T).T               # (P, d)


# ---------------------------------------------------------------------------
# §3.2, Eq. (3): the surrogate Phi and its gradient


def phi(B, Z, lam1, lam2):
    """Phi(z) = ||B z||_1 + lam1 sum_i (z_i - floor z_i)(ceil z_i - z_i)
    + lam2 max{1/||z||_inf - 1, 0}, one value per start row (Eq. (3))."""
    Z = np.asarray(Z, np.float64)
    Y = Z @ np.asarray(B, np.float64).T                      # rows: (B z)^T
    l1 = np.abs(Y).sum(axis=1)
    frac = ((Z - np.floor(Z)) * (np.ceil(Z) - Z)).sum(axis=1)
    zinf = np.abs(Z).max(axis=1)
    with np.errstate(divide="ignore"):
        inv = np.where(zinf > 0, 1.0 / np.where(zinf > 0, zinf, 1.0), np.inf)
    return l1 + lam1 * frac + lam2 * np.maximum(inv - 1.0, 0.0)


def phi_grad(B, Z, lam1, lam2):
    """Gradient of Eq. (3) for every start row, under the readings above."""
    Z = np.asarray(Z, np.float64)
    Bf = np.asarray(B, np.float64)
    Y = Z @ Bf.T
    grad = np.sign(Y) @ Bf                                   # B^T sign(B z)
    grad += lam1 * (np.ceil(Z) + np.floor(Z) - 2.0 * Z)
    absZ = np.abs(Z)
    k = absZ.argmax(axis=1)                                   # first maximiser
    zinf = absZ[np.arange(Z.shape[0]), k]
    active = (zinf < 1.0) & (zinf > 0.0)
    rows = np.nonzero(active)[0]
    zk = Z[rows, k[rows]]
    grad[rows, k[rows]] += -lam2 * np.sign(zk) / (zinf[rows] ** 2)
    return grad


def adam_update(z, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step at step number t >= 1 (Kingma & Ba, Algorithm 1)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    z = z - lr * m_hat / (np.sqrt(v_hat) + eps)
    return z, m, v


# ---------------------------------------------------------------------------
# Algorithm 2: round, map, bound test; conditions C1-C4 (§3)


def round_and_map(B, Z):
    """zhat = nearest integer to z (ties to even); g = B zhat (int64)."""
    zhat = np.rint(np.asarray(Z, np.float64)).astype(np.int64)
    return zhat, zhat @ np.asarray(B, np.int64).T


def bound_consistent(G, l, u):
    """C4: l - u <= g <= u - l, per row."""
    span = np.asarray(u, np.int64) - np.asarray(l, np.int64)
    return np.all(np.abs(np.asarray(G, np.int64)) <= span, axis=1)


def kernel_condition(A, G):
    """C1: A g = 0 exactly, per row."""
    return np.all(np.asarray(G, np.int64) @ np.asarray(A, np.int64).T == 0, axis=1)


def canonical_sign(g):
    """The representative of {g, -g} whose first nonzero entry is positive."""
    g = np.asarray(g, np.int64)
    nz = np.nonzero(g)[0]
    if nz.size and g[nz[0]] < 0:
        return -g
    return g


def conformal_leq(x, y):
    """x ⊑ y  iff  x_i y_i >= 0 and |x_i| <= |y_i| for all i (§1)."""
    x = np.asarray(x, np.int64)
    y = np.asarray(y, np.int64)
    return bool(np.all(x * y >= 0) and np.all(np.abs(x) <= np.abs(y)))


def minimal_elements(G, rows=None):
    """Rows g of G (a set stored once up to sign) with no other row h such that
    h ⊑ g or -h ⊑ g: the ⊑-minimal elements of the symmetric set (C3).

    Returns a boolean mask over G, or over the selected `rows` (indices into
    G, each still compared with every row of G) when given.  Plain O(K^2 n)
    comparison of every pair.
    """
    G = np.asarray(G, np.int64)
    K = G.shape[0]
    sel = range(K) if rows is None else rows
    keep = np.ones(len(sel), dtype=bool)
    absG = np.abs(G)
    for q, i in enumerate(sel):
        g = G[i]
        dominated_pos = np.all((G * g >= 0) & (absG <= absG[i]), axis=1)
        dominated_neg = np.all((-G * g >= 0) & (absG <= absG[i]), axis=1)
        hit = dominated_pos | dominated_neg
        hit[i] = False
        keep[q] = not hit.any()
    return keep


def sort_directions(G):
    """Lexicographic row order (ascending, first column most significant)."""
    G = np.asarray(G, np.int64)
    if G.shape[0] == 0:
        return G
    order = np.lexsort(G.T[::-1])
    return G[order]


def collect(A, B, l, u, Z):
    """The collection step of Algorithm 2 for one snapshot of all starts:
    returns the set of canonical directions B round(z) that are nonzero,
    bound-consistent (C4) and satisfy A g = 0 (C1)."""
    _, G = round_and_map(B, Z)
    ok = bound_consistent(G, l, u) & np.any(G != 0, axis=1) & kernel_condition(A, G)
    return {tuple(canonical_sign(g)) for g in G[ok]}


def parallel_extraction(A, B, l, u, Z0, T, lam1=0.85, lam2=1.0, lr=0.003,
                        beta1=0.9, beta2=0.999, eps=1e-8, period=1,
                        keep_trace=False):
    """Algorithm 2 (§3.2) from given starting points Z0 (P x d).

    For t = 1..T every start takes one Adam step on Eq. (3); every ``period``
    steps the rounded point is mapped and, when it passes the tests, added to
    the set.  Afterwards the set is reduced to its ⊑-minimal elements and
    sorted.  Returns a dict with the final directions and counts.
    """
    z = np.asarray(Z0, np.float64).copy()
    m = np.zeros_like(z)
    v = np.zeros_like(z)
    found = set()
    trace = [] if keep_trace else None
    for t in range(1, T + 1):
        grad = phi_grad(B, z, lam1, lam2)
        z, m, v = adam_update(z, m, v, grad, t, lr, beta1, beta2, eps)
        if keep_trace:
            trace.append(z.copy())
        if t % period == 0:
            found |= collect(A, B, l, u, z)
    unique = sort_directions(np.array(sorted(found), dtype=np.int64).reshape(-1, len(l)))
    keep = minimal_elements(unique)
    return {"unique": unique, "directions": unique[keep], "Z": z, "M": m, "V": v,
            "trace": trace}


# ---------------------------------------------------------------------------
# Algorithm 1 (§2): augmentation with a direction set as the test set


def f_value(Q, c, w, x):
    """f(x) = x^T Q x + c^T x + sum_i w_i x_i^4 in exact integers."""
    x = np.asarray(x, np.int64)
    val = int(x @ np.asarray(Q, np.int64) @ x) + int(np.asarray(c, np.int64) @ x)
    if w is not None:
        val += int(np.asarray(w, np.int64) @ (x ** 4))
    return val


def in_feasible_region(A, b, l, u, x):
    """x in S: A x = b and l <= x <= u."""
    x = np.asarray(x, np.int64)
    return bool(np.all(np.asarray(A, np.int64) @ x == np.asarray(b, np.int64))
                and np.all(x >= l) and np.all(x <= u))


def feasible_step_lengths(l, u, x, g):
    """All lambda >= 1 with l <= x + lambda g <= u (by direct test)."""
    g = np.asarray(g, np.int64)
    x = np.asarray(x, np.int64)
    if not np.any(g):
        return []
    out = []
    lam = 1
    while True:
        y = x + lam * g
        if np.all(y >= l) and np.all(y <= u):
            out.append(lam)
            lam += 1
        else:
            return out


def augment(A, b, l, u, Q, c, w, directions, x0, max_iters=100000):
    """Algorithm 1: while some (g, lambda) with g in ±directions, lambda >= 1,
    x + lambda g in S and f(x + lambda g) < f(x) exists, move to the argmin of
    f(x + lambda g).  f is evaluated directly at every candidate point.

    Returns (x, f(x), list of moves (direction index, sign, lambda, f)).
    """
    x = np.asarray(x0, np.int64).copy()
    fx = f_value(Q, c, w, x)
    moves = []
    D = np.asarray(directions, np.int64)
    for _ in range(max_iters):
        best = None
        for k in range(D.shape[0]):
            for sgn in (1, -1):
                g = sgn * D[k]
                for lam in feasible_step_lengths(l, u, x, g):
                    y = x + lam * g
                    if not in_feasible_region(A, b, l, u, y):
                        continue
                    fy = f_value(Q, c, w, y)
                    if fy < fx and (best is None or fy < best[0]):
                        best = (fy, k, sgn, lam)
        if best is None:
            break
        fy, k, sgn, lam = best
        x = x + lam * sgn * D[k]
        fx = fy
        moves.append((k, sgn, lam, fy))
    return x, fx, moves


# ---------------------------------------------------------------------------
# Initial feasible solutions, Eq. (4) (§3.3)


def init_objective(A, b, X, lam3):
    """||A x - b||_2^2 + lam3 * sum_i (x_i - floor x_i)(ceil x_i - x_i), per
    row x of X."""
    X = np.asarray(X, np.float64)
    R = X @ np.asarray(A, np.float64).T - np.asarray(b, np.float64)
    frac = (X - np.floor(X)) * (np.ceil(X) - X)
    return np.sum(R * R, axis=1) + lam3 * np.sum(frac, axis=1)


def init_gradient(A, b, X, lam3):
    """Gradient of Eq. (4) in x: 2 A^T (A x - b) + lam3 (ceil x + floor x - 2 x)
    (the same reading of the floor/ceil product as for Eq. (3))."""
    X = np.asarray(X, np.float64)
    Af = np.asarray(A, np.float64)
    R = X @ Af.T - np.asarray(b, np.float64)
    return 2.0 * R @ Af + lam3 * (np.ceil(X) + np.floor(X) - 2.0 * X)


def projected_adam_update(x, m, v, grad, t, lr, l, u, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step on x followed by the projection onto the box [l, u]
    (Eq. (4) constrains x to [l, u]; Adam itself is unconstrained)."""
    z, m, v = adam_update(x, m, v, grad, t, lr, beta1, beta2, eps)
    return np.clip(z, np.asarray(l, np.float64), np.asarray(u, np.float64)), m, v


def feasible_roundings(A, b, l, u, X):
    """The set of rounded rows round(x) (ties to even) that are feasible for
    model (1): A round(x) = b exactly and l <= round(x) <= u."""
    Xr = np.rint(np.asarray(X, np.float64)).astype(np.int64)
    ok = np.all(Xr @ np.asarray(A, np.int64).T == np.asarray(b, np.int64), axis=1)
    ok &= np.all((Xr >= np.asarray(l, np.int64)) & (Xr <= np.asarray(u, np.int64)), axis=1)
    return {tuple(x) for x in Xr[ok]}


def initial_solutions(A, b, l, u, X0, T, lam3=0.1, lr=0.003, beta1=0.9, beta2=0.999, eps=1e-8, period=1):
    """Eq. (4) from every start row of X0 by projected Adam for T steps; after
    every `period`-th step the rounded points feasible for model (1) are
    collected.  Returns (final X, set of feasible integer points)."""
    X = np.clip(np.asarray(X0, np.float64), np.asarray(l, np.float64), np.asarray(u, np.float64))
    M = np.zeros_like(X)
    V = np.zeros_like(X)
    found = set()
    for t in range(1, T + 1):
        G = init_gradient(A, b, X, lam3)
        X, M, V = projected_adam_update(X, M, V, G, t, lr, l, u, beta1, beta2, eps)
        if t % period == 0:
            found |= feasible_roundings(A, b, l, u, X)
    return X, found


# ---------------------------------------------------------------------------
# Linear inequalities G x >= h (§3.4, Corollary 3.3)


def inequality_extension(A, b, l, u, G, h, B):
    """The equality form of model (1) with G x >= h: slack s = G x - h >= 0,
    constraint matrix [A 0; G -I], right-hand side (b, h), kernel basis
    [B; G B] (Corollary 3.3).  x is boxed, so each slack is bounded above by
    its largest value over the box, max_x (G x)_k - h_k.  Returns
    (A', b', l', u', B'); raises if some inequality cannot hold in the box."""
    A, G, B = (np.asarray(M, np.int64) for M in (A, G, B))
    b, h, l, u = (np.asarray(v, np.int64) for v in (b, h, l, u))
    m, n = A.shape
    m2 = G.shape[0]
    smax = np.sum(np.maximum(G * l, G * u), axis=1) - h
    if np.any(smax < 0):
        raise ValueError("an inequality cannot hold anywhere in the box")
    A2 = np.block([[A, np.zeros((m, m2), np.int64)], [G, -np.eye(m2, dtype=np.int64)]])
    b2 = np.concatenate([b, h])
    l2 = np.concatenate([l, np.zeros(m2, np.int64)])
    u2 = np.concatenate([u, smax])
    B2 = np.concatenate([B, G @ B], axis=0)
    return A2, b2, l2, u2, B2


def lattice_contains(B, g):
    """True if the integer vector g is an integer combination of the columns
    of B (full column rank): solve B z = g exactly in rationals via least
    squares and check that z is integral and reproduces g."""
    B = np.asarray(B, np.float64)
    z, *_ = np.linalg.lstsq(B, np.asarray(g, np.float64), rcond=None)
    zi = np.rint(z)
    return bool(np.allclose(z, zi, atol=1e-9) and np.array_equal(np.asarray(B, np.int64) @ zi.astype(np.int64),
                                                                   np.asarray(g, np.int64)))


# ---------------------------------------------------------------------------
# A kernel basis of a general A (Lemma 3.1, Theorem 3.2) and LLL (Appendix A)


def _egcd(a, b):
    """(g, x, y) with x a + y b = g = gcd(a, b) >= 0 (Python integers)."""
    x0, y0, x1, y1 = 1, 0, 0, 1
    while b != 0:
        q = a // b
        a, b = b, a - q * b
        x0, x1 = x1, x0 - q * x1
        y0, y1 = y1, y0 - q * y1
    if a < 0:
        a, x0, y0 = -a, -x0, -y0
    return a, x0, y0


def hnf_kernel_basis(A):
    """Lemma 3.1: unimodular integer column operations K bring A to (H | 0)
    with H lower triangular (row by row, each row's entries right of the pivot
    are cleared by extended-gcd combinations of two columns); the last
    d = n - m columns of K are a basis of Ker_Z(A) (Theorem 3.2).  Exact
    Python integers; A must have full row rank.  Returns (B [n x d], K)."""
    A = [[int(v) for v in row] for row in np.asarray(A, np.int64)]
    m, n = len(A), len(A[0])
    M = [row[:] for row in A]
    K = [[int(i == j) for j in range(n)] for i in range(n)]

    def combine(c, j, x, y, p, q):  # col_c <- x col_c + y col_j, col_j <- p col_c + q col_j
        for R in (M, K):
            for row in R:
                a, b = row[c], row[j]
                row[c], row[j] = x * a + y * b, p * a + q * b

    for i in range(m):
        c = i
        for j in range(c + 1, n):
            b = M[i][j]
            if b == 0:
                continue
            a = M[i][c]
            g, x, y = _egcd(a, b)
            combine(c, j, x, y, -b // g, a // g)
        if M[i][c] == 0:
            raise ValueError("A does not have full row rank")
        if M[i][c] < 0:
            for R in (M, K):
                for row in R:
                    row[c] = -row[c]
    B = np.array([[K[r][j] for j in range(m, n)] for r in range(n)], dtype=object)
    return B, np.array(K, dtype=object)


def lll_reduce(B, factor=2):
    """Appendix A's LLL in exact rationals: size-reduce column i against
    columns i-1, ..., 1 (mu_ij rounded to the nearest integer, halves away
    from zero), then exchange columns i-1 and i when
    ||B*_{i-1}||^2 > factor ||B*_i||^2 and step back, else step forward.  The
    Gram-Schmidt data are recomputed from scratch after every change (plain,
    slow, obviously the definition).  Returns the reduced basis (object ints)."""
    from fractions import Fraction
    Bc = [[int(B[r][j]) for r in range(len(B))] for j in range(len(B[0]))]  # columns
    d = len(Bc)

    def dot(u, v):
        return sum(Fraction(a) * b for a, b in zip(u, v))

    def gso():
        star, mu = [], [[Fraction(0)] * d for _ in range(d)]
        for i in range(d):
            v = [Fraction(a) for a in Bc[i]]
            for j in range(i):
                mu[i][j] = dot(Bc[i], star[j]) / dot(star[j], star[j])
                v = [a - mu[i][j] * b for a, b in zip(v, star[j])]
            star.append(v)
        return star, mu

    def nearest(q):
        f = q.numerator // q.denominator
        r = q - f
        return f + 1 if r > Fraction(1, 2) or (r == Fraction(1, 2) and q > 0) else f

    i = 1
    while i < d:
        for j in range(i - 1, -1, -1):
            _, mu = gso()
            k = nearest(mu[i][j])
            if k != 0:
                Bc[i] = [a - k * b for a, b in zip(Bc[i], Bc[j])]
        star, _ = gso()
        if dot(star[i - 1], star[i - 1]) > factor * dot(star[i], star[i]):
            Bc[i - 1], Bc[i] = Bc[i], Bc[i - 1]
            i = max(i - 1, 1)
        else:
            i += 1
    return np.array([[Bc[j][r] for j in range(d)] for r in range(len(Bc[0]))], dtype=object)


def lll_conditions(B, factor=2):
    """(size_reduced, exchange_condition) of Appendix A's definition, exact."""
    from fractions import Fraction
    Bc = [[Fraction(int(B[r][j])) for r in range(len(B))] for j in range(len(B[0]))]
    d = len(Bc)
    star, ok_size = [], True
    for i in range(d):
        v = Bc[i][:]
        for j in range(i):
            mu = sum(a * b for a, b in zip(Bc[i], star[j])) / sum(b * b for b in star[j])
            ok_size &= abs(mu) <= Fraction(1, 2)
            v = [a - mu * b for a, b in zip(v, star[j])]
        star.append(v)
    norms = [sum(a * a for a in v) for v in star]
    ok_ex = all(norms[j] <= factor * norms[j + 1] for j in range(d - 1))
    return ok_size, ok_ex


# ---------------------------------------------------------------------------
# Definition of the Graver basis (§1), by enumeration, for tiny instances


def kernel_box(A, bound):
    """All nonzero integer g with A g = 0 and |g_i| <= bound."""
    A = np.asarray(A, np.int64)
    n = A.shape[1]
    pts = np.array(list(itertools.product(range(-bound, bound + 1), repeat=n)),
                   dtype=np.int64)
    ok = np.all(pts @ A.T == 0, axis=1) & np.any(pts != 0, axis=1)
    return pts[ok]


def graver_basis_box(A, bound):
    """⊑-minimal elements of Ker_Z(A) \\ {0} among |g_i| <= bound, one per sign
    pair (canonical sign), sorted.  Inside a box, minimality among the box's
    kernel elements is the same as minimality in all of Ker_Z(A), because
    every h ⊑ g also lies in the box."""
    K = kernel_box(A, bound)
    absK = np.abs(K)
    out = set()
    for i in range(K.shape[0]):
        g = K[i]
        below = np.all((K * g >= 0) & (absK <= absK[i]), axis=1)
        below[i] = False
        if not below.any():
            out.add(tuple(canonical_sign(g)))
    return sort_directions(np.array(sorted(out), dtype=np.int64).reshape(-1, A.shape[1]))


def is_graver_element(A, g):
    """g is ⊑-minimal in Ker_Z(A) \\ {0}: no nonzero h ⊑ g, h != g, has A h = 0.
    Enumerates every h conformal to g directly."""
    g = np.asarray(g, np.int64)
    A = np.asarray(A, np.int64)
    if not np.any(g) or np.any(A @ g != 0):
        return False
    ranges = [range(0, abs(int(gi)) + 1) for gi in g]
    sgn = np.sign(g)
    for mags in itertools.product(*ranges):
        h = sgn * np.array(mags, np.int64)
        if np.any(h) and np.any(h != g) and np.all(A @ h == 0):
            return False
    return True
