"""Helpers shared by the GPU tests: device copies of generated instances and
tolerance rules.  Imports torch/libmape lazily so CPU collection stays cheap."""
import numpy as np


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def rel_fro(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = max(np.linalg.norm(b), 1e-30)
    return float(np.linalg.norm(a - b) / den)


def sign_stable_rows(B, Z, factor=2.0):
    """Starts whose every (B z)_i is farther from 0 than the forward error
    bound of an FP32 dot product, factor * d * 2^-24 * sum_j |B_ij z_j|
    (sequential or blocked summation of d products): their sign(Bz), and so
    the whole gradient of Eq. (3), is the same in FP32 and FP64."""
    Bf = np.asarray(B, np.float64)
    Zf = np.asarray(Z, np.float64)
    Y = Zf @ Bf.T
    bound = factor * Bf.shape[1] * 2.0 ** -24 * (np.abs(Zf) @ np.abs(Bf).T)
    return np.all(np.abs(Y) > bound, axis=1)


def rows_set(G, n):
    G = np.asarray(G)
    return {tuple(int(v) for v in r[:n]) for r in G}
