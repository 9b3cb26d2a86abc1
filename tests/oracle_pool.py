"""A pool of spawned worker processes that run the CPU oracle for the
bench-scale GPU tests (test infrastructure).  Spawned, not forked: a process
forked after the parent has touched the GPU can hang.  Every function here
only calls oracle/ on the arrays it is given."""
import multiprocessing as mp
import os

import numpy as np


def _minimal_rows(args):
    from oracle import mape_oracle as O
    G, lo, hi = args
    return O.minimal_elements(G, rows=list(range(lo, hi)))


def _augment(args):
    from oracle import mape_oracle as O
    A, b, l, u, Q, c, w, D, x0, max_iters = args
    return O.augment(A, b, l, u, Q, c, w, D, x0, max_iters=max_iters)


class OraclePool:
    def __init__(self, procs=None):
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(k, "1")
        self.procs = procs or max(1, min(16, os.cpu_count() or 1))
        self.pool = mp.get_context("spawn").Pool(self.procs)

    def minimal_elements(self, G):
        """O.minimal_elements(G), rows split over the workers."""
        G = np.asarray(G, np.int64)
        K = G.shape[0]
        step = -(-K // (4 * self.procs))
        parts = self.pool.map(_minimal_rows, [(G, lo, min(lo + step, K)) for lo in range(0, K, step)])
        return np.concatenate(parts) if parts else np.zeros(0, bool)

    def augment(self, inst, w, D, X0, max_iters=100000):
        """O.augment from every row of X0, one start per task."""
        tasks = [(inst.A, inst.b, inst.l, inst.u, inst.Q, inst.c, w, np.asarray(D, np.int64),
                  np.asarray(x, np.int64), max_iters) for x in X0]
        return self.pool.map(_augment, tasks)

    def close(self):
        self.pool.close()
        self.pool.join()
