"""The per-start parity rules of the GPU tests (tests/gpu_common.py), checked
on the CPU with outputs made from the oracle itself: exact outputs pass, and
one wrong start among many is caught (a single Frobenius norm over a whole
step would let it through)."""
import numpy as np
import pytest

from oracle import mape_oracle as O
from paper_2412_13576_gb300 import instances as I

from .gpu_common import check_adam, check_phi_grad, per_start_rel


def _case(P=512, seed=3):
    inst = I.medium_sparse()
    rng = np.random.default_rng(seed)
    Z = rng.uniform(-4, 4, size=(P, inst.d)).astype(np.float32)
    return inst, Z


def test_exact_outputs_pass():
    inst, Z = _case()
    phi = O.phi(inst.B, Z, 0.85, 1.0).astype(np.float32)
    grad = O.phi_grad(inst.B, Z, 0.85, 1.0).astype(np.float32)
    st = check_phi_grad(inst.B, Z, phi, grad, bits=16)
    assert st["worst_excess"] <= 0 and st["max_rel_grad"] < 1e-6


def test_one_wrong_start_is_caught():
    inst, Z = _case()
    phi = O.phi(inst.B, Z, 0.85, 1.0)
    grad = O.phi_grad(inst.B, Z, 0.85, 1.0)
    bad = grad.copy()
    bad[17] *= 1.0 + 1e-3          # one start of 512 off by 1e-3
    # the whole-step Frobenius error stays below 1e-4 ...
    assert np.linalg.norm(bad - grad) / np.linalg.norm(grad) < 1e-4
    # ... but the per-start rule rejects it
    with pytest.raises(AssertionError):
        check_phi_grad(inst.B, Z, phi, bad, bits=16)
    badphi = phi.copy()
    badphi[200] += 1e-2 * abs(badphi[200])
    with pytest.raises(AssertionError):
        check_phi_grad(inst.B, Z, badphi, grad, bits=16)


def test_sign_flip_on_an_ambiguous_row_is_allowed_and_bounded():
    """Put (B z)_i of one start exactly at 0: the kernel may take either sign
    there, so a gradient with B_i added (sign 0 -> +1) passes, while the same
    jump on a row far from 0 fails."""
    inst, Z = _case(P=64)
    B = inst.B.astype(np.float64)
    i = inst.d + 3                                   # a row of -C
    j = int(np.nonzero(B[i])[0][0])                  # one coordinate it touches
    z = Z[5].astype(np.float64)
    z[j] -= (B[i] @ z) / B[i, j]                     # (B z)_i = 0 up to rounding
    Z[5] = z.astype(np.float32)
    phi = O.phi(inst.B, Z, 0.85, 1.0)
    grad = O.phi_grad(inst.B, Z, 0.85, 1.0)
    flipped = grad.copy()
    flipped[5] += B[i]
    st = check_phi_grad(inst.B, Z, phi, flipped, bits=16)
    assert st["ambiguous_share"] > 0
    far = grad.copy()
    k = int(np.argmax(np.abs(Z[7].astype(np.float64) @ B.T)))
    far[7] += 2 * B[k]
    with pytest.raises(AssertionError):
        check_phi_grad(inst.B, Z, phi, far, bits=16)


def test_adam_rule_is_per_start():
    rng = np.random.default_rng(1)
    z, m, v, g = (rng.standard_normal((300, 40)) for _ in range(4))
    v = np.abs(v)
    z1, m1, v1 = O.adam_update(z, m, v, g, 3, 0.003)
    check_adam(z, m, v, g, 3, z1, m1, v1)
    z1b = z1.copy()
    z1b[123, 5] += 1e-3
    assert per_start_rel(z1b, z1).max() > 1e-5
    with pytest.raises(AssertionError):
        check_adam(z, m, v, g, 3, z1b, m1, v1)
