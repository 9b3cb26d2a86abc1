"""Helpers shared by the GPU tests: device copies of generated instances and
the per-start tolerance rules of the continuous stages.  Imports torch/libmape
lazily so CPU collection stays cheap.

Continuous parity is checked start by start (one row of Z is one start, an
independent problem of Eq. (3)), never through one norm over a whole step:

* the forward product B z is carried by the kernels with z to `bits`
  significant bits (24 on the FP32 paths, 16 for the hi + lo BF16 operands, 8
  for one BF16 term) and summed in FP32; its error per row i is at most
  (2^-bits + d 2^-23) sum_j |B_ij z_j|.  A row whose |(B z)_i| does not exceed
  that bound is *ambiguous*: its sign(B z)_i may legitimately differ from the
  FP64 oracle's;
* the gradient B^T sign(B z) then differs by at most 2 |B_ij| per ambiguous
  row i in coordinate j, so every start is checked coordinate-wise against
  2 sum_{i ambiguous} |B_ij| plus the FP32 tolerance, and the starts with no
  ambiguous row within the relative tolerance of their own gradient norm;
* Phi per start within the summed forward bound plus the relative tolerance;
* the Adam update per start, from the kernel's own gradient, within the
  relative tolerance of that start's norm."""
import numpy as np

from oracle import mape_oracle as O


def dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def per_start_rel(a, b, floor=1e-30):
    """Per row p: ||a_p - b_p||_2 / ||b_p||_2 (rows with ||b_p|| = 0 compare
    ||a_p|| against `floor`).  Returns the array of per-start errors."""
    a = np.asarray(a, np.float64).reshape(len(a), -1)
    b = np.asarray(b, np.float64).reshape(len(b), -1)
    num = np.linalg.norm(a - b, axis=1)
    den = np.maximum(np.linalg.norm(b, axis=1), floor)
    return num / den


def forward_error_bound(B, Z, bits, abs_err=None):
    """[P x n] bound on |fl(B z)_i - (B z)_i| for z carried to `bits`
    significant bits and d products summed in FP32, with 1% slack.
    abs_err [P], if given, is an absolute error per element of z on top of the
    relative one (the subnormal range of a narrow format)."""
    Bf = np.abs(np.asarray(B, np.float64))
    Zf = np.abs(np.asarray(Z, np.float64))
    d = Bf.shape[1]
    bound = (2.0 ** -bits + d * 2.0 ** -23) * (Zf @ Bf.T) * 1.01 + 1e-6
    if abs_err is not None:
        bound += np.asarray(abs_err, np.float64)[:, None] * Bf.sum(axis=1)[None, :] * 1.01
    return bound


def e4m3_abs_err(Z):
    """Per start, the absolute error of an element of z in the FP8 forward
    product beyond the relative 2^-4: half the e4m3 subnormal step (2^-10) in
    units of z, whose per-start scale is 2^(8 - e) with max |z| < 2^e."""
    zinf = np.abs(np.asarray(Z, np.float64)).max(axis=1)
    e = np.where(zinf > 0, np.frexp(np.where(zinf > 0, zinf, 1.0))[1], 0)
    scale = np.where(zinf > 0, np.ldexp(1.0, np.clip(8 - e, -100, 100)), 1.0)
    return 2.0 ** -10 / scale


def check_phi_grad(B, Z, phi, grad, bits, tol=1e-5, lam1=0.85, lam2=1.0, abs_err=None):
    """Checks the kernel's Phi [P] and gradient [P x d] at the points Z against
    the FP64 oracle, start by start, under the rules in this module's
    docstring.  Returns statistics: the share of starts with an ambiguous row,
    the mean number of ambiguous rows per start, the largest per-start
    relative gradient error on the starts without one, and the largest
    coordinate error over the allowance on all starts (<= 0 passes)."""
    Bf = np.asarray(B, np.float64)
    Zf = np.asarray(Z, np.float64)
    grad = np.asarray(grad, np.float64)
    phi = np.asarray(phi, np.float64)
    Y = Zf @ Bf.T
    eb = forward_error_bound(B, Z, bits, abs_err)
    amb = np.abs(Y) <= eb
    go = O.phi_grad(B, Zf, lam1, lam2)
    po = O.phi(B, Zf, lam1, lam2)
    # gradient: every start, coordinate-wise
    allow = 2.0 * amb.astype(np.float64) @ np.abs(Bf)
    scale = np.maximum(np.abs(go).max(axis=1, initial=0.0), 1.0)[:, None]
    excess = np.abs(grad - go) - (allow + tol * scale)
    worst = float(excess.max(initial=-np.inf))
    assert worst <= 0.0, f"gradient beyond the per-start allowance by {worst}"
    determined = ~amb.any(axis=1)
    rel = per_start_rel(grad[determined], go[determined]) if determined.any() else np.zeros(0)
    assert np.all(rel <= tol), f"per-start gradient error {rel.max()} on a start without ambiguous rows"
    # Phi: per start (+inf exactly where the oracle has +inf, z = 0)
    inf = np.isinf(po)
    assert np.array_equal(np.isinf(phi), inf)
    pb = eb.sum(axis=1)
    dphi = np.abs(phi[~inf] - po[~inf])
    assert np.all(dphi <= pb[~inf] + tol * np.abs(po[~inf]) + 1e-5), "Phi beyond the per-start bound"
    return {"ambiguous_share": float(amb.any(axis=1).mean()), "ambiguous_rows_per_start": float(amb.sum(1).mean()),
            "max_rel_grad": float(rel.max(initial=0.0)), "worst_excess": worst}


def check_adam(z, m, v, grad, t, z1, m1, v1, tol=1e-5, lr=0.003):
    """The kernel's Adam step t (1-based) from (z, m, v) with its own gradient
    against the oracle's, per start within `tol` relative."""
    zo, mo, vo = O.adam_update(np.asarray(z, np.float64), np.asarray(m, np.float64), np.asarray(v, np.float64),
                               np.asarray(grad, np.float64), t, lr)
    for got, want, name in ((z1, zo, "z"), (m1, mo, "m"), (v1, vo, "v")):
        err = per_start_rel(got, want)
        nz = np.linalg.norm(np.asarray(want, np.float64).reshape(len(want), -1), axis=1) > 0
        assert np.all(err[nz] <= tol), f"Adam {name}: per-start error {err[nz].max()}"
        assert np.all(np.asarray(got)[~nz] == 0), f"Adam {name}: nonzero where the oracle is zero"


def rows_set(G, n):
    G = np.asarray(G)
    return {tuple(int(v) for v in r[:n]) for r in G}


def check_steps(inst, states, grads, phis, bits, tol=1e-5, fp8=False):
    """Per-step parity of a run of single steps (states[t] = ((z, m, v) before,
    (z, m, v) after), grads/phis the kernel's debug outputs at the input
    point): Phi and gradient by check_phi_grad, Adam by check_adam, and the
    oracle's collection of the kernel's own iterates.  Returns (the union of
    the collected sets, the share of start-steps with an ambiguous row, the
    mean ambiguous rows per start-step, the largest per-start gradient error
    on start-steps without one)."""
    expect = set()
    shares, rows, worst = [], [], 0.0
    for t, ((z, m, v), (z1, m1, v1)) in enumerate(states):
        st = check_phi_grad(inst.B, z, phis[t], grads[t], bits, tol, abs_err=e4m3_abs_err(z) if fp8 else None)
        check_adam(z, m, v, grads[t], t + 1, z1, m1, v1, tol)
        shares.append(st["ambiguous_share"])
        rows.append(st["ambiguous_rows_per_start"])
        worst = max(worst, st["max_rel_grad"])
        expect |= O.collect(inst.A, inst.B, inst.l, inst.u, z1)
    return expect, float(np.mean(shares)), float(np.mean(rows)), worst


def report(case, **values):
    """Prints one line of observed figures (shown with pytest -s, or by -rA
    for failures) and appends it to the file named by MAPE_TEST_REPORT, if
    set."""
    import json
    import os
    line = json.dumps({"case": case, **values})
    print(line)
    path = os.environ.get("MAPE_TEST_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(line + "\n")
