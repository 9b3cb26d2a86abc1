"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/mape.h declares; its struct layouts match the ctypes binding; argument
checks answer before any device work.  CPU only (no compute calls)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mape.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2412_13576_gb300 import mape
    return mape.lib(build_if_missing=True)


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(mape_[a-z0-9_]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


def test_every_declared_symbol_is_exported(lib):
    from paper_2412_13576_gb300 import mape
    out = subprocess.run(["nm", "-D", "--defined-only", mape.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mape_\w+)", out))
    declared = _declared()
    assert len(declared) >= 25
    missing = [n for n in declared if n not in exported]
    assert not missing, missing


def test_struct_layouts_match_binding(tmp_path, lib):
    from paper_2412_13576_gb300 import mape
    prog = tmp_path / "sizes.c"
    prog.write_text('#include "mape.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){'
                    'printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(mape_config), sizeof(mape_extract_args),'
                    'sizeof(mape_augment_args), sizeof(mape_problem), sizeof(mape_status),'
                    'offsetof(mape_extract_args, cand_count), offsetof(mape_augment_args, max_iters));return 0;}')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()))
    expect = [ctypes.sizeof(mape.Config), ctypes.sizeof(mape.ExtractArgs), ctypes.sizeof(mape.AugmentArgs),
              ctypes.sizeof(mape.Problem), ctypes.sizeof(mape.Status), mape.ExtractArgs.cand_count.offset,
              mape.AugmentArgs.max_iters.offset]
    assert got == expect


def test_server_struct_layouts_match_binding(tmp_path, lib):
    from paper_2412_13576_gb300 import mape
    prog = tmp_path / "sizes2.c"
    prog.write_text('#include "mape.h"\n#include <stdio.h>\n#include <stddef.h>\nint main(void){'
                    'printf("%zu %zu %zu %zu %zu\\n", sizeof(mape_server_config), sizeof(mape_request_info),'
                    'sizeof(mape_server_stats), offsetof(mape_server_config, max_slots),'
                    'offsetof(mape_request_info, t_first_improve_ms));return 0;}')
    exe = tmp_path / "sizes2"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()))
    expect = [ctypes.sizeof(mape.ServerConfig), ctypes.sizeof(mape.RequestInfo), ctypes.sizeof(mape.ServerStats),
              mape.ServerConfig.max_slots.offset, mape.RequestInfo.t_first_improve_ms.offset]
    assert got == expect


def test_request_bytes_estimate(lib):
    """The admission estimate covers at least the FP32 state and the two
    candidate buffers, grows with P and n, and is 0 for invalid sizes."""
    from paper_2412_13576_gb300 import mape
    cfg = mape.default_config(T=1000)
    n, m, P = 500, 100, 1024
    b = mape.request_bytes(n, m, P, 1, cfg)
    ldg = 512
    cap = min(P * 1001, 1 << 23, (1 << 31) // ldg)
    assert b >= 3 * P * (n - m) * 4 + 2 * cap * ldg
    assert mape.request_bytes(n, m, 2 * P, 1, cfg) > b
    assert mape.request_bytes(2 * n, 2 * m, P, 1, cfg) > b
    assert mape.request_bytes(n, m, P, 8, cfg) > b
    small = mape.default_config(T=1000, cand_capacity=4096)
    assert mape.request_bytes(n, m, P, 1, small) < b
    assert mape.request_bytes(n, n, P, 1, cfg) == 0
    assert mape.request_bytes(n, m, 0, 1, cfg) == 0
    assert lib.mape_request_bytes(n, m, P, 1, None) == 0


def test_server_argument_checks_without_device(lib):
    from paper_2412_13576_gb300 import mape
    h = ctypes.c_void_p()
    assert lib.mape_server_create(None, ctypes.byref(h)) == -1
    sc = mape.ServerConfig()
    sc.cfg = mape.default_config()
    sc.mem_cap_bytes, sc.max_slots = 1 << 30, 0
    assert lib.mape_server_create(ctypes.byref(sc), ctypes.byref(h)) == -1
    rid = ctypes.c_uint64(0)
    assert lib.mape_server_submit(None, None, None, None, None, None, None, 1, None, None, None, 1,
                                  ctypes.byref(rid)) == -1
    assert lib.mape_server_poll(None, 1, None) == -1
    assert lib.mape_server_wait_all(None, 0) == -1
    lib.mape_server_destroy(None)


def test_default_config_is_the_papers(lib):
    from paper_2412_13576_gb300 import mape
    c = mape.default_config()
    assert (round(c.lambda1, 6), c.lambda2, round(c.lr, 6)) == (0.85, 1.0, 0.003)
    assert (round(c.beta1, 6), round(c.beta2, 6), c.period) == (0.9, 0.999, 1)


def test_argument_checks_without_device(lib):
    from paper_2412_13576_gb300 import mape
    assert lib.mape_extract(None, None) == -1
    assert lib.mape_augment_run(None, None, None) == -1
    h = ctypes.c_void_p()
    assert lib.mape_create_instance(None, None, None, None, None, None, None, None, ctypes.byref(h)) == -1
    K = ctypes.c_int64(5)
    assert lib.mape_dedup(None, 0, 4, 16, None, 0, ctypes.byref(K), None, 0, None) == 0 and K.value == 0
    assert lib.mape_dedup(None, 0, 4, 15, None, 0, ctypes.byref(K), None, 0, None) == -1
    assert lib.mape_poll(None, None) == -1
    assert lib.mape_wait(None, 0) == -1
    lib.mape_destroy(None)
    assert lib.mape_project_workspace_bytes(10, 5) > 100
    assert lib.mape_dedup_workspace_bytes(1000, 32) > 1000 * 8


def test_augment_batch_argument_checks(lib):
    """Algorithm 1's batched and tuned entry points refuse bad arguments
    before any device work: no items, a lane count that is not a power of two
    up to 32, a null output."""
    from paper_2412_13576_gb300 import mape
    it = (ctypes.c_int64 * 2)()
    assert lib.mape_augment_run_batch(None, 2, it, None, 0, None, None, None) == -1
    A = (mape.AugmentArgs * 1)()
    A[0].n, A[0].S, A[0].K, A[0].ldg, A[0].score_lanes = 4, 0, 0, 16, 3
    assert lib.mape_augment_run_batch(A, 1, it, None, 0, None, None, None) == -1
    assert lib.mape_augment_run(ctypes.byref(A[0]), it, None) == -1
    A[0].score_lanes = 0
    assert lib.mape_augment_run_batch(A, 0, it, None, 0, None, None, None) == -1
    assert lib.mape_augment_run_batch_workspace_bytes(0) == 0
    assert lib.mape_augment_run_batch_workspace_bytes(8) > 8 * 64
    assert lib.mape_augment_tune_lookup(4, 1, 1, 0, None) == -1
    assert mape.augment_tune_lookup(12345, 1, 1, False) is None
    assert lib.mape_augment_batch(None, 1, None, None) == -1
    # 1024 partial minima per start at most, whatever K
    assert lib.mape_augment_workspace_bytes(200, 4, 1 << 30) == lib.mape_augment_workspace_bytes(200, 4, 1 << 20)


def test_bounds_rejected_before_upload(lib):
    """u - l > 127 cannot be stored as int8 directions: BOUNDS, no device work."""
    import numpy as np
    from paper_2412_13576_gb300 import mape
    n, m = 4, 1
    A = np.array([[1, 1, 1, 1]], np.int32)
    B = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [-1, -1, -1]], np.int32)
    b = np.zeros(1, np.int64)
    l = np.zeros(n, np.int32)
    u = np.array([1, 1, 1, 200], np.int32)
    Q = np.eye(n, dtype=np.int32)
    c = np.zeros(n, np.int32)
    prob = mape.Problem(n, m, ctypes.c_void_p(Q.ctypes.data), ctypes.c_void_p(c.ctypes.data), None)
    cfg = mape.default_config()
    h = ctypes.c_void_p()
    rc = lib.mape_create_instance(ctypes.c_void_p(A.ctypes.data), ctypes.c_void_p(b.ctypes.data),
                                  ctypes.c_void_p(l.ctypes.data), ctypes.c_void_p(u.ctypes.data), ctypes.byref(prob),
                                  ctypes.c_void_p(B.ctypes.data), ctypes.byref(cfg), None, ctypes.byref(h))
    assert rc == -4


def test_inequality_extension_matches_oracle(lib):
    """mape_inequality_extension (host-only) writes the oracle's equality form
    of G x >= h: [A 0; G -I], (b, h), slack bounds, [B; G B]."""
    import numpy as np
    from oracle import mape_oracle as O
    from paper_2412_13576_gb300 import instances as I
    from paper_2412_13576_gb300 import mape
    for inst, seed in ((I.tiny_graver_case(), 1), (I.small_dense(), 2), (I.medium_sparse(), 3)):
        rng = np.random.default_rng(seed)
        G = rng.integers(-2, 3, size=(3, inst.n))
        h = G @ inst.xbar.astype(np.int64) - rng.integers(0, 4, size=3)
        e = mape.inequality_extension(inst, G, h)
        A2, b2, l2, u2, B2 = O.inequality_extension(inst.A, inst.b, inst.l, inst.u, G, h, inst.B)
        for got, want in ((e.A, A2), (e.b, b2), (e.l, l2), (e.u, u2), (e.B, B2)):
            assert np.array_equal(got, want)
        assert np.all(e.A.astype(np.int64) @ e.B == 0)
        assert np.array_equal(e.A.astype(np.int64) @ e.xbar, e.b)
        # Corollary 3.3's objective and point: f ignores the slacks, and xbar
        # carries them (G xbar - h), inside the slack bounds
        n = inst.n
        assert np.array_equal(e.xbar[:n], inst.xbar)
        assert np.array_equal(e.xbar[n:], G @ inst.xbar.astype(np.int64) - h)
        assert O.in_feasible_region(e.A, e.b, e.l, e.u, e.xbar)
        assert np.all(e.Q[n:] == 0) and np.all(e.Q[:, n:] == 0) and np.array_equal(e.Q[:n, :n], inst.Q)
        assert np.all(e.c[n:] == 0) and np.array_equal(e.c[:n], inst.c)
        assert O.f_value(e.Q, e.c, e.w, e.xbar) == O.f_value(inst.Q, inst.c, inst.w, inst.xbar)
    inst = I.tiny_graver_case()
    with pytest.raises(mape.MapeError) as err:
        mape.inequality_extension(inst, np.ones((1, inst.n), np.int32), [10 ** 6])
    assert err.value.code == -4


def test_inequality_extension_objective_and_points(lib):
    """The objective (with the quartic weights) and several points of the
    extended instance through the C ABI: w2 = (w, 0); a point that violates
    G x >= h has no slack and is refused with MAPE_ERR_BOUNDS."""
    import ctypes

    import numpy as np
    from oracle import mape_oracle as O
    from paper_2412_13576_gb300 import instances as I
    from paper_2412_13576_gb300 import mape
    inst = I.make_instance("quartic_n12_m3", 12, 3, c_k=2, c_density=0.5, lo=-4, hi=4, q_k=3, q_density=0.3,
                           lin_k=5, w_max=3, seed=41)
    rng = np.random.default_rng(5)
    n, m2 = inst.n, 2
    G = rng.integers(-2, 3, size=(m2, n)).astype(np.int32)
    h = (G @ inst.xbar.astype(np.int64) - 3).astype(np.int64)
    e = mape.inequality_extension(inst, G, h)
    assert np.array_equal(e.w[:n], inst.w) and np.all(e.w[n:] == 0)
    X = np.stack([inst.xbar, inst.xbar]).astype(np.int32)
    X2 = np.empty((2, n + m2), np.int32)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    assert lib.mape_inequality_extension_points(n, m2, ptr(G), ptr(h), ptr(X), 2, ptr(X2)) == 0
    for r in range(2):
        assert np.array_equal(X2[r], e.xbar)
        assert O.f_value(e.Q, e.c, e.w, X2[r]) == O.f_value(inst.Q, inst.c, inst.w, X[r])
    # a point below one inequality: G x - h < 0
    hb = h.copy()
    hb[1] = G[1] @ inst.xbar.astype(np.int64) + 1
    assert lib.mape_inequality_extension_points(n, m2, ptr(G), ptr(hb), ptr(X), 2, ptr(X2)) == -4


def test_kernel_basis_matches_oracle(lib):
    """mape_kernel_basis (host-only): the HNF basis equals the oracle's exactly,
    the LLL-reduced one equals the oracle's exact-rational LLL on these
    matrices and satisfies Appendix A's conditions; A B = 0; a rank-deficient
    A is refused."""
    import numpy as np
    from oracle import mape_oracle as O
    from paper_2412_13576_gb300 import instances as I
    from paper_2412_13576_gb300 import mape
    for A in (np.array([[2, 3, -1, 4], [1, -2, 5, 0]]), I.tiny_graver_case().A, I.small_dense().A,
              I.general_instance().A, I.general_instance(n=20, m=6, seed=3).A):
        Bo, _ = O.hnf_kernel_basis(A)
        if max(abs(int(v)) for v in Bo.ravel()) <= 2 ** 31 - 1:
            assert np.array_equal(mape.kernel_basis(A, reduce=False), np.array(Bo, dtype=np.int64))
        else:  # the unreduced basis does not fit the int32 output
            with pytest.raises(mape.MapeError):
                mape.kernel_basis(A, reduce=False)
        B = mape.kernel_basis(A, reduce=True)
        assert np.all(A.astype(np.int64) @ B == 0)
        assert np.array_equal(B, np.array(O.lll_reduce(Bo), dtype=np.int64))
        assert O.lll_conditions(B) == (True, True)
    with pytest.raises(mape.MapeError) as err:
        mape.kernel_basis(np.array([[1, 2, 3], [2, 4, 6]]))
    assert err.value.code == -1


def test_mma_issue_probe_refuses_bad_arguments(lib):
    """Argument checks of the measurement entry point run before any CUDA call."""
    import ctypes
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    for args in ((2, 128, 256, 1, 64), (0, 96, 256, 1, 64), (0, 128, 8, 1, 64), (0, 128, 264, 1, 64),
                 (0, 128, 256, 3, 64), (0, 128, 512, 2, 64), (0, 128, 256, 1, 0)):
        assert lib.mape_mma_issue_probe(*args, ctypes.byref(a), ctypes.byref(b)) == -1
