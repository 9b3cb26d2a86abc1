"""Seeded synthetic instances of model (1) and the random draws of the method.

This module is the one piece shared by the CUDA path and the CPU oracle: it
draws numbers and lays them out, and holds none of the method's arithmetic.

An instance is min f(x) s.t. Ax = b, l <= x <= u, x integer (Eq. (1), §1),
generated with A = [C | I_m] so that the kernel-lattice basis is known in
closed form, B = [I_d ; -C] (n x d, d = n - m): A B = C - C = 0, and B has
full column rank because its top block is I_d.  This is the instance family
the workloads are defined on; Theorem 3.2 (§3.1) is what makes any such B a
basis of Ker_Z(A).

The objective is integer:  f(x) = x^T Q x + c^T x + sum_i w_i x_i^4 with Q
symmetric (no 1/2 factor) and w >= 0 optional.

Sparse integer draws: an entry is nonzero with probability ``density`` and
then uniform on [-k, k] \\ {0}.  "Dense" draws (density None) are uniform on
[-k, k] including 0.  Q is drawn on its upper triangle (diagonal included)
and mirrored.

Random numbers the method itself consumes are drawn here and passed to both
sides as inputs:
  * ``Z0`` (P x d, float32): starting points drawn directly, Z ~ N(0, 2)
    with standard deviation 2 (the small workload);
  * ``G0`` (P x n, float32): samples g ~ Uniform(l - u, u - l), one row per
    start, which the method projects to z0 = (B^T B)^{-1} B^T g
    (Algorithm 2, §3.2).  The projection is method arithmetic and is done by
    each side on its own.

Layouts (row-major, C order): A m x n, B n x d, Q n x n, Z0 P x d (one start
per row), G0 P x n.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Instance:
    name: str
    n: int
    m: int
    A: np.ndarray      # (m, n) int32
    B: np.ndarray      # (n, d) int32
    b: np.ndarray      # (m,)  int64
    l: np.ndarray      # (n,)  int32
    u: np.ndarray      # (n,)  int32
    Q: np.ndarray      # (n, n) int32, symmetric
    c: np.ndarray      # (n,)  int32
    w: np.ndarray | None  # (n,) int32 >= 0, or None (no quartic term)
    xbar: np.ndarray   # (n,)  int32, feasible: A xbar = b, l <= xbar <= u

    @property
    def d(self) -> int:
        return self.n - self.m


@dataclasses.dataclass
class Starts:
    P: int
    Z0: np.ndarray | None   # (P, d) float32, starts given directly
    G0: np.ndarray | None   # (P, n) float32, samples to be projected


def _int_matrix(rng, shape, k, density):
    if density is None:
        return rng.integers(-k, k + 1, size=shape).astype(np.int64)
    mask = rng.random(shape) < density
    mag = rng.integers(1, k + 1, size=shape)
    sgn = np.where(rng.random(shape) < 0.5, -1, 1)
    return np.where(mask, mag * sgn, 0).astype(np.int64)


def _sym_matrix(rng, n, k, density):
    full = _int_matrix(rng, (n, n), k, density)
    upper = np.triu(full)
    return upper + np.triu(upper, 1).T


def make_instance(name, n, m, *, c_k, c_density, lo, hi, q_k, q_density,
                  lin_k, w_max=None, seed=0) -> Instance:
    """Draw one instance with A = [C | I_m], B = [I_d ; -C]."""
    rng = np.random.default_rng(seed)
    d = n - m
    C = _int_matrix(rng, (m, d), c_k, c_density)
    A = np.concatenate([C, np.eye(m, dtype=np.int64)], axis=1)
    B = np.concatenate([np.eye(d, dtype=np.int64), -C], axis=0)
    l = np.full(n, lo, dtype=np.int64)
    u = np.full(n, hi, dtype=np.int64)
    xbar = rng.integers(l, u + 1)
    b = A @ xbar
    Q = _sym_matrix(rng, n, q_k, q_density)
    c = rng.integers(-lin_k, lin_k + 1, size=n)
    w = None if w_max is None else rng.integers(0, w_max + 1, size=n)
    return Instance(
        name=name, n=n, m=m,
        A=A.astype(np.int32), B=B.astype(np.int32), b=b.astype(np.int64),
        l=l.astype(np.int32), u=u.astype(np.int32), Q=Q.astype(np.int32),
        c=c.astype(np.int32), w=None if w is None else w.astype(np.int32),
        xbar=xbar.astype(np.int32))


def normal_starts(inst: Instance, P: int, std: float = 2.0, seed: int = 0) -> Starts:
    """Z0 ~ N(0, std) drawn directly in coordinate space."""
    rng = np.random.default_rng(seed)
    Z0 = (rng.standard_normal((P, inst.d)) * std).astype(np.float32)
    return Starts(P=P, Z0=Z0, G0=None)


def uniform_samples(inst: Instance, P: int, seed: int = 0) -> Starts:
    """g ~ Uniform(l - u, u - l) per coordinate, one row per start."""
    rng = np.random.default_rng(seed)
    lo = (inst.l - inst.u).astype(np.float64)
    hi = (inst.u - inst.l).astype(np.float64)
    G0 = (lo + (hi - lo) * rng.random((P, inst.n))).astype(np.float32)
    return Starts(P=P, Z0=None, G0=G0)


# ---------------------------------------------------------------------------
# The five workloads.  Seeds: instance 1000 + k, starts 2000 + k.

def small_dense(seed=1001) -> Instance:
    """n=20, m=5: C 5x15 uniform in [-2,2], box [-5,5], Q in [-3,3] at 0.3, c in [-10,10]."""
    return make_instance("small_dense_n20_m5", 20, 5, c_k=2, c_density=None,
                         lo=-5, hi=5, q_k=3, q_density=0.3, lin_k=10, seed=seed)


def medium_sparse(seed=1002) -> Instance:
    """n=200, m=40: C 40x160 in [-3,3] at 0.1, box [0,10], Q in [-5,5] at 0.05, c in [-20,20]."""
    return make_instance("medium_sparse_n200_m40", 200, 40, c_k=3, c_density=0.1,
                         lo=0, hi=10, q_k=5, q_density=0.05, lin_k=20, seed=seed)


def large_quartic(seed=1004) -> Instance:
    """n=2000, m=400: C in [-5,5] at 0.01, box [-20,20], Q in [-5,5] at 0.005, w in [0,3]."""
    return make_instance("large_quartic_n2000_m400", 2000, 400, c_k=5, c_density=0.01,
                         lo=-20, hi=20, q_k=5, q_density=0.005, lin_k=20, w_max=3,
                         seed=seed)


def uneven_batch(count=64, n_lo=50, n_hi=1000, seed=1003):
    """Instances with n log-uniform in [n_lo, n_hi], m = n/5, C in [-3,3] at a
    density uniform in [0.05, 0.2], box [-5,5], f as in the small workload."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        m = max(1, n // 5)
        dens = float(rng.uniform(0.05, 0.2))
        out.append(make_instance(f"uneven_{k}_n{n}", n, m, c_k=3, c_density=dens,
                                 lo=-5, hi=5, q_k=3, q_density=0.3, lin_k=10,
                                 seed=seed * 100 + k))
    return out


def uneven_single(n, density=0.1, seed=1003):
    """One instance of the uneven family at a chosen n (m = n/5, box [-5,5])."""
    return make_instance(f"uneven_n{n}", n, max(1, n // 5), c_k=3, c_density=density,
                         lo=-5, hi=5, q_k=3, q_density=0.3, lin_k=10, seed=seed * 100 + n)


def general_instance(n=12, m=4, seed=1005):
    """A general A (not of the form [C | I]): entries uniform in [-2, 2],
    drawn until it has full row rank; box [-3, 3]; Q sym [-3,3] at 0.3,
    c in [-10,10].  B is left empty: a kernel basis of A is the caller's to
    compute (Lemma 3.1)."""
    rng = np.random.default_rng(seed)
    while True:
        A = rng.integers(-2, 3, size=(m, n))
        if np.linalg.matrix_rank(A) == m:
            break
    l, u = np.full(n, -3, dtype=np.int64), np.full(n, 3, dtype=np.int64)
    xbar = rng.integers(l, u + 1)
    Q = _sym_matrix(rng, n, 3, 0.3)
    c = rng.integers(-10, 11, size=n)
    return Instance(name=f"general_n{n}_m{m}", n=n, m=m, A=A.astype(np.int32),
                    B=np.zeros((n, n - m), np.int32), b=(A @ xbar).astype(np.int64),
                    l=l.astype(np.int32), u=u.astype(np.int32), Q=Q.astype(np.int32),
                    c=c.astype(np.int32), w=None, xbar=xbar.astype(np.int32))


def tiny_graver_case(seed=7):
    """6 variables, 2 rows: A = [C | I_2] with C 2x4 in {-1,0,1}; box [-1,2],
    so that bound consistency (C4) admits exactly the entries |g_i| <= 3."""
    return make_instance("tiny_n6_m2", 6, 2, c_k=1, c_density=None,
                         lo=-1, hi=2, q_k=2, q_density=0.5, lin_k=5, seed=seed)
