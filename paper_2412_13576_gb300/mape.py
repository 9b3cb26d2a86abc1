"""Python binding of libmape (ctypes).  Argument marshalling only: every step
of the path runs in the library's CUDA kernels.  Names follow include/mape.h.

Device buffers are torch tensors (torch is used for device memory and
streams); the handle API takes host numpy arrays.  If the library is missing
or cannot be loaded, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK = 0
ERR = {
    -1: "INVALID_ARG", -2: "SHAPE", -3: "NOT_KERNEL_BASIS", -4: "BOUNDS", -5: "INFEASIBLE",
    -6: "OVERFLOW", -7: "CAPACITY", -8: "CUDA", -9: "TIMEOUT", -10: "STATE", -11: "OOM",
    -12: "KERNEL_TEST", -13: "NUMERIC", -14: "CANCELLED",
}
PREC_FP32 = 0
PREC_BF16 = 1
PREC_BF16X1 = 2
PREC_SPARSE = 3
PREC_FP8 = 4
PREC_STREAMED = 0x100   # OR into a BF16 precision: force the streamed tensor-core kernels
PREC_AUTOTUNE = 0x200   # OR into a BF16 precision: choose the implementation and tile widths by timing
PREC_SPARSE_FWD = 0x400  # OR into MAPE_PREC_BF16: the CUDA-core sparse forward product on the streamed path
PHASES = ["IDLE", "EXTRACTING", "FILTERING", "AUGMENTING", "DONE", "ERROR"]


class MapeError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        name = ERR.get(code, str(code))
        extra = ""
        if code == -8 and _LIB is not None:
            extra = ": " + _LIB.mape_last_cuda_error().decode()
        super().__init__(f"{where} failed with MAPE_ERR_{name}{extra}")


P_ = C.c_void_p
I32 = C.c_int32
I64 = C.c_int64
F32 = C.c_float


class Config(C.Structure):
    _fields_ = [("lambda1", F32), ("lambda2", F32), ("lr", F32), ("eps", F32), ("beta1", C.c_double),
                ("beta2", C.c_double), ("T", I32), ("period", I32), ("precision", I32), ("reserved", I32),
                ("cand_capacity", I64), ("max_aug_iters", I64)]


class ExtractArgs(C.Structure):
    _fields_ = [("n", I32), ("d", I32), ("P", I32), ("B", P_), ("span", P_), ("Z", P_), ("M", P_),
                ("V", P_), ("t0", I32), ("T", I32), ("period", I32), ("precision", I32),
                ("lambda1", F32), ("lambda2", F32), ("lr", F32), ("eps", F32), ("beta1", C.c_double),
                ("beta2", C.c_double), ("cand", P_), ("ldc", I32), ("pad0", I32), ("cand_cap", I64),
                ("cand_count", P_), ("flags", P_), ("dbg_phi", P_), ("dbg_grad", P_),
                ("workspace", P_), ("workspace_bytes", C.c_size_t)]


class InitArgs(C.Structure):
    _fields_ = [("n", I32), ("m", I32), ("P", I32), ("pad0", I32), ("A", P_), ("b", P_), ("l", P_), ("u", P_),
                ("X", P_), ("M", P_), ("V", P_), ("t0", I32), ("T", I32), ("period", I32), ("lambda3", F32),
                ("lr", F32), ("eps", F32), ("beta1", C.c_double), ("beta2", C.c_double), ("sol", P_),
                ("lds", I32), ("pad1", I32), ("sol_cap", I64), ("sol_count", P_), ("flags", P_),
                ("dbg_f", P_), ("dbg_grad", P_), ("workspace", P_), ("workspace_bytes", C.c_size_t)]


class DedupItem(C.Structure):
    _fields_ = [("cand", P_), ("count", I64), ("n", I32), ("ldc", I32), ("uniq", P_), ("uniq_cap", I64),
                ("K", I64), ("status", I32), ("pad0", I32), ("workspace", P_), ("workspace_bytes", C.c_size_t)]


class KernelTestItem(C.Structure):
    _fields_ = [("A", P_), ("m", I32), ("n", I32), ("G", P_), ("K", I64), ("ldg", I32), ("pad0", I32), ("ok", P_),
                ("fail_count", I64), ("workspace", P_), ("workspace_bytes", C.c_size_t)]


class MinimalItem(C.Structure):
    _fields_ = [("G", P_), ("K", I64), ("n", I32), ("ldg", I32), ("valid", P_), ("keep", P_), ("out", P_),
                ("K_out", I64), ("workspace", P_), ("workspace_bytes", C.c_size_t)]


class CoeffsItem(C.Structure):
    _fields_ = [("q_row", P_), ("q_col", P_), ("q_val", P_), ("nnz", I32), ("n", I32), ("w", P_), ("G", P_),
                ("K", I64), ("ldg", I32), ("pad0", I32), ("a", P_), ("q4", P_)]


class AugTuneInfo(C.Structure):
    _fields_ = [("lanes", I32), ("candidates", I32), ("cand_lanes", I32 * 8), ("probe_ms", F32 * 8)]


class AugmentArgs(C.Structure):
    _fields_ = [("n", I32), ("S", I32), ("K", I64), ("G", P_), ("ldg", I32), ("score_lanes", I32),
                ("a", P_), ("q4", P_), ("q_row", P_), ("q_col", P_), ("q_val", P_), ("nnz", I32),
                ("pad1", I32), ("c", P_), ("w", P_), ("l", P_), ("u", P_), ("X", P_), ("fval", P_),
                ("moves", P_), ("nmoves", P_), ("moves_cap", I32), ("pad2", I32),
                ("max_iters", I64), ("workspace", P_), ("workspace_bytes", C.c_size_t)]


class TuneInfo(C.Structure):
    _fields_ = [("path", I32), ("wF", I32), ("wG", I32), ("candidates", I32), ("probe_steps", I32),
                ("cand_path", I32 * 16), ("cand_wF", I32 * 16), ("cand_wG", I32 * 16), ("probe_ms", F32 * 16)]

    def as_dict(self):
        k = self.candidates
        names = ("resident", "streamed", "streamed_sparse_forward")
        return {"path": names[self.path], "wF": self.wF, "wG": self.wG,
                "probe_steps": self.probe_steps,
                "candidates": [{"path": names[self.cand_path[i]], "wF": self.cand_wF[i],
                                "wG": self.cand_wG[i], "ms": self.probe_ms[i]} for i in range(k)]}


class Problem(C.Structure):
    _fields_ = [("n", I32), ("m", I32), ("Q", P_), ("c", P_), ("w", P_)]


class Status(C.Structure):
    _fields_ = [("phase", I32), ("error", I32), ("candidates", I64), ("unique", I64),
                ("kernel_failures", I64), ("directions", I64), ("aug_iters", I64), ("best_f", I64),
                ("best_start", I32), ("pad0", I32), ("extract_ms", C.c_double),
                ("filter_ms", C.c_double), ("augment_ms", C.c_double),
                ("first_improve_ms", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("pad")}
        d["phase"] = PHASES[self.phase] if 0 <= self.phase < len(PHASES) else self.phase
        return d


class ServerConfig(C.Structure):
    _fields_ = [("cfg", Config), ("mem_cap_bytes", C.c_size_t), ("max_slots", I32), ("keep_directions", I32),
                ("batch_extraction", I32), ("reserved", I32)]


class RequestInfo(C.Structure):
    _fields_ = [("state", I32), ("error", I32), ("n", I32), ("m", I32), ("P", I32), ("pad0", I32),
                ("directions", I64), ("best_f", I64), ("aug_iters", I64), ("bytes", C.c_size_t),
                ("t_submit_ms", C.c_double), ("t_admit_ms", C.c_double), ("t_extracted_ms", C.c_double),
                ("t_first_improve_ms", C.c_double), ("t_done_ms", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("pad")}
        d["state"] = REQ_STATES[self.state] if 0 <= self.state < len(REQ_STATES) else self.state
        return d


class ServerStats(C.Structure):
    _fields_ = [("submitted", I64), ("completed", I64), ("failed", I64), ("queued", I64), ("running", I64),
                ("peak_running", I64), ("mem_in_use", C.c_size_t), ("mem_peak", C.c_size_t),
                ("mem_cap", C.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


REQ_STATES = ("QUEUED", "RUNNING", "DONE", "FAILED")

_LIB = None

_SIGS = {
    "mape_default_config": (None, [C.POINTER(Config)]),
    "mape_version": (C.c_char_p, []),
    "mape_last_cuda_error": (C.c_char_p, []),
    "mape_launch_count": (C.c_ulonglong, []),
    "mape_project_workspace_bytes": (C.c_size_t, [I32, I32]),
    "mape_project_starts": (C.c_int, [P_, I32, I32, P_, I32, P_, P_, C.c_size_t, P_]),
    "mape_project_prepare_workspace_bytes": (C.c_size_t, [I32, I32]),
    "mape_project_prepare": (C.c_int, [P_, I32, I32, P_, P_, C.c_size_t, P_]),
    "mape_project_apply": (C.c_int, [P_, I32, I32, P_, I32, P_, P_]),
    "mape_phi_grad": (C.c_int, [P_, I32, I32, P_, I32, F32, F32, P_, P_, P_]),
    "mape_extract_workspace_bytes": (C.c_size_t, [I32, I32, I32, I32]),
    "mape_extract": (C.c_int, [C.POINTER(ExtractArgs), P_]),
    "mape_initial_solutions_workspace_bytes": (C.c_size_t, [I32, I32, I32]),
    "mape_initial_solutions": (C.c_int, [C.POINTER(InitArgs), P_]),
    "mape_autotune_lookup": (C.c_int, [I32, I32, I32, I32, C.POINTER(TuneInfo)]),
    "mape_autotune_clear": (None, []),
    "mape_dedup_workspace_bytes": (C.c_size_t, [I64, I32]),
    "mape_dedup": (C.c_int, [P_, I64, I32, I32, P_, I64, C.POINTER(I64), P_, C.c_size_t, P_]),
    "mape_kernel_test_batch_workspace_bytes": (C.c_size_t, [I32]),
    "mape_kernel_test_batch": (C.c_int, [C.POINTER(KernelTestItem), I32, P_, C.c_size_t, P_]),
    "mape_minimal_filter_batch_workspace_bytes": (C.c_size_t, [C.POINTER(MinimalItem), I32]),
    "mape_minimal_filter_batch": (C.c_int, [C.POINTER(MinimalItem), I32, P_, C.c_size_t, P_]),
    "mape_direction_coeffs_batch_workspace_bytes": (C.c_size_t, [I32]),
    "mape_direction_coeffs_batch": (C.c_int, [C.POINTER(CoeffsItem), I32, P_, C.c_size_t, P_]),
    "mape_dedup_batch_workspace_bytes": (C.c_size_t, [I32]),
    "mape_dedup_batch": (C.c_int, [C.POINTER(DedupItem), I32, P_, C.c_size_t, P_]),
    "mape_dedup_static_max_rows": (I64, []),
    "mape_dedup_static": (C.c_int, [P_, I64, I32, I32, P_, I64, C.POINTER(I64), P_]),
    "mape_kernel_test_workspace_bytes": (C.c_size_t, [I32, I32]),
    "mape_kernel_test": (C.c_int, [P_, I32, I32, P_, I64, I32, P_, C.POINTER(I64), P_, C.c_size_t, P_]),
    "mape_minimal_workspace_bytes": (C.c_size_t, [I64, I32]),
    "mape_minimal_filter": (C.c_int, [P_, I64, I32, I32, P_, P_, P_, C.POINTER(I64), P_, C.c_size_t, P_]),
    "mape_direction_coeffs": (C.c_int, [P_, P_, P_, I32, P_, I32, P_, I64, I32, P_, P_, P_]),
    "mape_augment_workspace_bytes": (C.c_size_t, [I32, I32, I64]),
    "mape_augment_run": (C.c_int, [C.POINTER(AugmentArgs), C.POINTER(I64), P_]),
    "mape_augment_run_batch_workspace_bytes": (C.c_size_t, [I32]),
    "mape_augment_run_batch": (C.c_int, [C.POINTER(AugmentArgs), I32, C.POINTER(I64), P_, C.c_size_t, P_, P_, P_]),
    "mape_augment_tune_lookup": (C.c_int, [I32, I64, I32, I32, C.POINTER(AugTuneInfo)]),
    "mape_augment_batch": (C.c_int, [C.POINTER(P_), I32, C.POINTER(P_), C.POINTER(I32)]),
    "mape_set_allocator": (C.c_int, [P_, P_, P_]),
    "mape_trim_memory": (C.c_int, []),
    "mape_create_instance": (C.c_int, [P_, P_, P_, P_, C.POINTER(Problem), P_, C.POINTER(Config), P_,
                                       C.POINTER(P_)]),
    "mape_extract_directions": (C.c_int, [P_, I32, P_, P_]),
    "mape_extract_directions_batch": (C.c_int, [C.POINTER(P_), I32, C.POINTER(I32), C.POINTER(P_), C.POINTER(P_)]),
    "mape_augment": (C.c_int, [P_, P_, I32, C.POINTER(Problem)]),
    "mape_poll": (C.c_int, [P_, C.POINTER(Status)]),
    "mape_wait": (C.c_int, [P_, I64]),
    "mape_cancel": (C.c_int, [P_]),
    "mape_get_directions": (C.c_int, [P_, P_, I64, C.POINTER(I64)]),
    "mape_get_directions_i8": (C.c_int, [P_, P_, I64, I64, C.POINTER(I64)]),
    "mape_get_solution": (C.c_int, [P_, P_, C.POINTER(I64)]),
    "mape_get_solutions": (C.c_int, [P_, P_, P_, I32]),
    "mape_destroy": (None, [P_]),
    "mape_inequality_extension": (C.c_int, [I32, I32, I32, P_, P_, P_, P_, P_, P_, P_, P_, P_, P_, P_, P_]),
    "mape_kernel_basis": (C.c_int, [I32, I32, P_, I32, P_]),
    "mape_inequality_extension_objective": (C.c_int, [I32, I32, P_, P_, P_, P_, P_, P_]),
    "mape_inequality_extension_points": (C.c_int, [I32, I32, P_, P_, P_, I32, P_]),
    "mape_find_initial_solutions": (C.c_int, [P_, I32, P_, I32, I32, P_, I32, C.POINTER(I32)]),
    "mape_request_bytes": (C.c_size_t, [I32, I32, I32, I32, C.POINTER(Config)]),
    "mape_server_create": (C.c_int, [C.POINTER(ServerConfig), C.POINTER(P_)]),
    "mape_server_submit": (C.c_int, [P_, P_, P_, P_, P_, C.POINTER(Problem), P_, I32, P_, P_, P_, I32,
                                     C.POINTER(C.c_uint64)]),
    "mape_server_poll": (C.c_int, [P_, C.c_uint64, C.POINTER(RequestInfo)]),
    "mape_server_wait": (C.c_int, [P_, C.c_uint64, I64]),
    "mape_server_wait_all": (C.c_int, [P_, I64]),
    "mape_server_result": (C.c_int, [P_, C.c_uint64, P_, C.POINTER(I64), P_, I64, C.POINTER(I64)]),
    "mape_server_release": (C.c_int, [P_, C.c_uint64]),
    "mape_server_get_stats": (C.c_int, [P_, C.POINTER(ServerStats)]),
    "mape_server_destroy": (None, [P_]),
    "mape_launch_timing": (C.c_int, [I32]),
    "mape_mma_issue_probe": (C.c_int, [I32, I32, I32, I32, I32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mape_launch_timing_read": (C.c_int, [C.POINTER(C.c_double), C.POINTER(I64)]),
}


def library_path() -> str:
    """The in-tree build, unless MAPE_LIBRARY names another build of libmape."""
    return os.environ.get("MAPE_LIBRARY", _build.LIB)


def lib(build_if_missing: bool = False):
    """The loaded libmape.  Raises if it is not built (or build_if_missing).
    On a machine with a CUDA device, the handles' device memory is routed
    through PyTorch's caching allocator (use_torch_allocator)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if build_if_missing:
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libmape is not built ({path}); run __graft_entry__.build()")
    L = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    try:
        import torch
        if torch.cuda.is_available():
            use_torch_allocator(True)
    except ImportError:
        pass
    return L


# ---- device memory of the handles: PyTorch's caching allocator ---------------

_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


def _torch_alloc(nbytes, stream, ctx):
    # runs on the thread that creates or feeds a handle (a server's scheduler
    # thread included), whose current device is the handle's; NULL = OOM
    try:
        import torch
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:
        return None


def _torch_free(ptr, nbytes, stream, ctx):
    try:
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:
        pass


_TORCH_HOOKS = (_ALLOC_FN(_torch_alloc), _FREE_FN(_torch_free))  # kept alive for the process


def use_torch_allocator(enable: bool = True):
    """Routes the device memory of every handle created afterwards through
    PyTorch's caching allocator on the handle's stream (mape_set_allocator),
    so that it is counted by torch.cuda.memory_allocated() and reused by
    torch; enable=False restores the library's own memory pool."""
    L = lib()
    if enable:
        _check(L.mape_set_allocator(C.cast(_TORCH_HOOKS[0], C.c_void_p), C.cast(_TORCH_HOOKS[1], C.c_void_p), None),
               "mape_set_allocator")
    else:
        _check(L.mape_set_allocator(None, None, None), "mape_set_allocator")


def _check(rc, where):
    if rc != OK:
        raise MapeError(rc, where)
    return rc


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def default_config(**over) -> Config:
    cfg = Config()
    lib().mape_default_config(C.byref(cfg))
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


def round16(n: int) -> int:
    return (n + 15) // 16 * 16


def _workspace(nbytes, device):
    import torch
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)


# ---- stage entry points (torch device tensors) ------------------------------

def project_starts(B, G0, stream=None):
    """a2: Z0 = (B^T B)^{-1} B^T g per row of G0.  B int32 [n,d], G0 f32 [P,n]."""
    import torch
    n, d = B.shape
    P = G0.shape[0]
    Z0 = torch.empty((P, d), dtype=torch.float32, device=B.device)
    ws = _workspace(lib().mape_project_workspace_bytes(n, d), B.device)
    _check(lib().mape_project_starts(_ptr(B), n, d, _ptr(G0), P, _ptr(Z0), _ptr(ws), ws.numel(),
                                     _stream(stream)), "mape_project_starts")
    return Z0


def phi_grad(B, Z, lambda1=0.85, lambda2=1.0, stream=None):
    """a3-a5 in FP32: (phi [P], grad [P,d])."""
    import torch
    n, d = B.shape
    P = Z.shape[0]
    phi = torch.empty(P, dtype=torch.float32, device=B.device)
    grad = torch.empty((P, d), dtype=torch.float32, device=B.device)
    _check(lib().mape_phi_grad(_ptr(B), n, d, _ptr(Z), P, lambda1, lambda2, _ptr(phi), _ptr(grad),
                               _stream(stream)), "mape_phi_grad")
    return phi, grad


def _extract_args(B, span, Z, M, V, *, t0, T, cfg: Config, cand, cand_count, flags, ldc,
                  dbg_phi=None, dbg_grad=None, workspace=None):
    n, d = B.shape
    P = Z.shape[0]
    a = ExtractArgs()
    a.n, a.d, a.P = n, d, P
    a.B, a.span, a.Z, a.M, a.V = _ptr(B), _ptr(span), _ptr(Z), _ptr(M), _ptr(V)
    a.t0, a.T, a.period, a.precision = t0, T, cfg.period, cfg.precision
    a.lambda1, a.lambda2, a.lr = cfg.lambda1, cfg.lambda2, cfg.lr
    a.beta1, a.beta2, a.eps = cfg.beta1, cfg.beta2, cfg.eps
    a.cand = _ptr(cand)
    a.ldc = ldc
    a.cand_cap = cand.shape[0] if cand is not None else 0
    a.cand_count, a.flags = _ptr(cand_count), _ptr(flags)
    a.dbg_phi, a.dbg_grad = _ptr(dbg_phi), _ptr(dbg_grad)
    if workspace is None:
        workspace = _workspace(lib().mape_extract_workspace_bytes(n, d, P, cfg.precision), B.device)
    a.workspace, a.workspace_bytes = _ptr(workspace), workspace.numel()
    return a, workspace


def extract_batch(calls, *, t0, T, cfg: Config, stream=None):
    """a3-a8 for many instances in one batched, graph-captured run.  calls:
    dicts with the keyword arguments of extract() except t0, T, cfg (B, span,
    Z, M, V, cand, cand_count, flags, ldc)."""
    keep = []
    arr = (ExtractArgs * len(calls))()
    for i, c in enumerate(calls):
        a, ws = _extract_args(t0=t0, T=T, cfg=cfg, **c)
        arr[i] = a
        keep.append(ws)
    nb = lib().mape_extract_batch_workspace_bytes(arr, len(calls))
    dev = calls[0]["B"].device
    bws = _workspace(max(nb, 16), dev)
    _check(lib().mape_extract_batch(arr, len(calls), _ptr(bws), bws.numel(), _stream(stream)), "mape_extract_batch")
    return keep


def initial_solutions(A, b, l, u, X, M, V, *, t0, T, sol, sol_count, flags, lds, lambda3=0.1, lr=0.003,
                      period=1, dbg_f=None, dbg_grad=None, stream=None):
    """Eq. (4): T projected Adam steps in place on X/M/V (device tensors);
    appends the exactly feasible roundings to sol as bytes round(x) - l."""
    m, n = A.shape
    a = InitArgs()
    a.n, a.m, a.P = n, m, X.shape[0]
    a.A, a.b, a.l, a.u, a.X, a.M, a.V = _ptr(A), _ptr(b), _ptr(l), _ptr(u), _ptr(X), _ptr(M), _ptr(V)
    a.t0, a.T, a.period, a.lambda3, a.lr, a.eps = t0, T, period, lambda3, lr, 1e-8
    a.beta1, a.beta2 = 0.9, 0.999
    a.sol, a.lds, a.sol_cap = _ptr(sol), lds, sol.shape[0]
    a.sol_count, a.flags, a.dbg_f, a.dbg_grad = _ptr(sol_count), _ptr(flags), _ptr(dbg_f), _ptr(dbg_grad)
    ws = _workspace(max(16, lib().mape_initial_solutions_workspace_bytes(n, m, T)), X.device)
    a.workspace, a.workspace_bytes = _ptr(ws), ws.numel()
    _check(lib().mape_initial_solutions(C.byref(a), _stream(stream)), "mape_initial_solutions")
    return ws


def extract(B, span, Z, M, V, *, t0, T, cfg: Config, cand, cand_count, flags, ldc,
            dbg_phi=None, dbg_grad=None, workspace=None, stream=None):
    """a3-a8: T Adam steps of Algorithm 2 in place on Z/M/V; appends to cand."""
    n, d = B.shape
    P = Z.shape[0]
    a = ExtractArgs()
    a.n, a.d, a.P = n, d, P
    a.B, a.span, a.Z, a.M, a.V = _ptr(B), _ptr(span), _ptr(Z), _ptr(M), _ptr(V)
    a.t0, a.T, a.period, a.precision = t0, T, cfg.period, cfg.precision
    a.lambda1, a.lambda2, a.lr = cfg.lambda1, cfg.lambda2, cfg.lr
    a.beta1, a.beta2, a.eps = cfg.beta1, cfg.beta2, cfg.eps
    a.cand = _ptr(cand)
    a.ldc = ldc
    a.cand_cap = cand.shape[0] if cand is not None else 0
    a.cand_count, a.flags = _ptr(cand_count), _ptr(flags)
    a.dbg_phi, a.dbg_grad = _ptr(dbg_phi), _ptr(dbg_grad)
    if workspace is None:
        workspace = _workspace(lib().mape_extract_workspace_bytes(n, d, P, cfg.precision), B.device)
    a.workspace, a.workspace_bytes = _ptr(workspace), workspace.numel()
    _check(lib().mape_extract(C.byref(a), _stream(stream)), "mape_extract")


def dedup(cand, count, n, stream=None):
    """a10: distinct rows of cand[:count], sorted lexicographically."""
    import torch
    ldc = cand.shape[1]
    uniq = torch.empty((max(count, 1), ldc), dtype=torch.int8, device=cand.device)
    ws = _workspace(lib().mape_dedup_workspace_bytes(count, ldc), cand.device)
    K = I64(0)
    _check(lib().mape_dedup(_ptr(cand), count, n, ldc, _ptr(uniq), uniq.shape[0], C.byref(K), _ptr(ws),
                            ws.numel(), _stream(stream)), "mape_dedup")
    return uniq[:K.value]


def dedup_batch(sets, stream=None):
    """mape_dedup_batch: a10 for several candidate sets in one sequence of
    launches.  sets: (cand [rows x ldc] int8 CUDA tensor, count, n, uniq_cap
    or None for count).  Returns one (distinct rows, K, status) per set (the
    rows empty when the status is not OK)."""
    import torch
    k = len(sets)
    items = (DedupItem * k)()
    keep = []
    for i, (cand, count, n, cap) in enumerate(sets):
        ldc = cand.shape[1]
        cap = count if cap is None else cap
        uniq = torch.zeros((max(cap, 1), ldc), dtype=torch.int8, device=cand.device)
        ws = _workspace(lib().mape_dedup_workspace_bytes(count, ldc), cand.device)
        keep.append((uniq, ws))
        it = items[i]
        it.cand, it.count, it.n, it.ldc = _ptr(cand), count, n, ldc
        it.uniq, it.uniq_cap = _ptr(uniq), cap
        it.workspace, it.workspace_bytes = _ptr(ws), ws.numel()
    dev = sets[0][0].device
    bws = _workspace(lib().mape_dedup_batch_workspace_bytes(k), dev)
    rc = lib().mape_dedup_batch(items, k, _ptr(bws), bws.numel(), _stream(stream))
    if rc not in (OK, -7):  # CAPACITY is reported per set
        _check(rc, "mape_dedup_batch")
    return [(keep[i][0][: items[i].K] if items[i].status == OK else keep[i][0][:0], items[i].K, items[i].status)
            for i in range(k)]


def kernel_test_batch(cases, stream=None):
    """mape_kernel_test_batch: a9 for several instances in one sequence of
    launches.  cases: (A [m x n] int32, G [K x ldg] int8, n) CUDA tensors.
    Returns one (ok [K] uint8, failures) per case."""
    import torch
    k = len(cases)
    items = (KernelTestItem * k)()
    keep = []
    for i, (A, G, n) in enumerate(cases):
        m, K = A.shape[0], G.shape[0]
        ok = torch.empty(max(K, 1), dtype=torch.uint8, device=G.device)
        ws = _workspace(lib().mape_kernel_test_workspace_bytes(m, n), G.device)
        keep.append((ok, ws))
        it = items[i]
        it.A, it.m, it.n, it.G, it.K, it.ldg, it.ok = _ptr(A), m, n, _ptr(G), K, G.shape[1], _ptr(ok)
        it.workspace, it.workspace_bytes = _ptr(ws), ws.numel()
    bws = _workspace(lib().mape_kernel_test_batch_workspace_bytes(k), cases[0][1].device)
    _check(lib().mape_kernel_test_batch(items, k, _ptr(bws), bws.numel(), _stream(stream)), "mape_kernel_test_batch")
    return [(keep[i][0][: cases[i][1].shape[0]], items[i].fail_count) for i in range(k)]


def minimal_filter_batch(cases, stream=None):
    """mape_minimal_filter_batch: a11 for several instances.  cases: (G [K x
    ldg] int8 CUDA tensor, n, valid [K] uint8 tensor or None).  Returns one
    (keep [K] uint8, kept rows [K_out x ldg]) per case."""
    import torch
    k = len(cases)
    items = (MinimalItem * k)()
    keep = []
    for i, (G, n, valid) in enumerate(cases):
        K, ldg = G.shape
        kp = torch.empty(max(K, 1), dtype=torch.uint8, device=G.device)
        out = torch.empty((max(K, 1), ldg), dtype=torch.int8, device=G.device)
        ws = _workspace(lib().mape_minimal_workspace_bytes(K, n), G.device)
        keep.append((kp, out, ws))
        it = items[i]
        it.G, it.K, it.n, it.ldg, it.valid = _ptr(G), K, n, ldg, _ptr(valid)
        it.keep, it.out, it.workspace, it.workspace_bytes = _ptr(kp), _ptr(out), _ptr(ws), ws.numel()
    bws = _workspace(lib().mape_minimal_filter_batch_workspace_bytes(items, k), cases[0][0].device)
    _check(lib().mape_minimal_filter_batch(items, k, _ptr(bws), bws.numel(), _stream(stream)),
           "mape_minimal_filter_batch")
    return [(keep[i][0][: cases[i][0].shape[0]], keep[i][1][: items[i].K_out]) for i in range(k)]


def direction_coeffs_batch(cases, stream=None):
    """mape_direction_coeffs_batch: a12 for several instances.  cases: (qr,
    qc, qv, w or None, n, G) CUDA tensors.  Returns one (a, q4) per case."""
    import torch
    k = len(cases)
    items = (CoeffsItem * k)()
    keep = []
    for i, (qr, qc, qv, w, n, G) in enumerate(cases):
        K, ldg = G.shape
        a = torch.empty(max(K, 1), dtype=torch.int64, device=G.device)
        q4 = torch.empty(max(K, 1), dtype=torch.int64, device=G.device)
        keep.append((a, q4))
        it = items[i]
        it.q_row, it.q_col, it.q_val, it.nnz, it.n, it.w = _ptr(qr), _ptr(qc), _ptr(qv), qv.numel(), n, _ptr(w)
        it.G, it.K, it.ldg, it.a, it.q4 = _ptr(G), K, ldg, _ptr(a), _ptr(q4)
    bws = _workspace(lib().mape_direction_coeffs_batch_workspace_bytes(k), cases[0][5].device)
    _check(lib().mape_direction_coeffs_batch(items, k, _ptr(bws), bws.numel(), _stream(stream)),
           "mape_direction_coeffs_batch")
    torch.cuda.synchronize()
    return [(keep[i][0][: cases[i][5].shape[0]], keep[i][1][: cases[i][5].shape[0]]) for i in range(k)]


def kernel_test(A, G, n, stream=None):
    """a9: (ok [K] uint8, failures)."""
    import torch
    m = A.shape[0]
    K = G.shape[0]
    ok = torch.empty(max(K, 1), dtype=torch.uint8, device=G.device)
    ws = _workspace(lib().mape_kernel_test_workspace_bytes(m, n), G.device)
    fails = I64(0)
    _check(lib().mape_kernel_test(_ptr(A), m, n, _ptr(G), K, G.shape[1], _ptr(ok), C.byref(fails), _ptr(ws),
                                  ws.numel(), _stream(stream)), "mape_kernel_test")
    return ok[:K], fails.value


def minimal_filter(G, n, valid=None, stream=None):
    """a11: (keep [K] uint8, kept rows in input order)."""
    import torch
    K, ldg = G.shape
    keep = torch.empty(max(K, 1), dtype=torch.uint8, device=G.device)
    out = torch.empty((max(K, 1), ldg), dtype=torch.int8, device=G.device)
    ws = _workspace(lib().mape_minimal_workspace_bytes(K, n), G.device)
    Ko = I64(0)
    _check(lib().mape_minimal_filter(_ptr(G), K, n, ldg, _ptr(valid), _ptr(keep), _ptr(out), C.byref(Ko),
                                     _ptr(ws), ws.numel(), _stream(stream)), "mape_minimal_filter")
    return keep[:K], out[:Ko.value]


def coo_upper(Q):
    """Upper triangle (incl. diagonal) of a symmetric numpy matrix as COO int32 arrays."""
    Q = np.asarray(Q)
    r, c = np.nonzero(np.triu(Q))
    return r.astype(np.int32), c.astype(np.int32), Q[r, c].astype(np.int32)


def direction_coeffs(qr, qc, qv, w, n, G, stream=None):
    """a12: (a [K] int64, q4 [K] int64)."""
    import torch
    K, ldg = G.shape
    a = torch.empty(max(K, 1), dtype=torch.int64, device=G.device)
    q4 = torch.empty(max(K, 1), dtype=torch.int64, device=G.device)
    _check(lib().mape_direction_coeffs(_ptr(qr), _ptr(qc), _ptr(qv), qv.numel(), _ptr(w), n, _ptr(G), K, ldg,
                                       _ptr(a), _ptr(q4), _stream(stream)), "mape_direction_coeffs")
    return a[:K], q4[:K]


def _augment_args(G, n, a, q4, qr, qc, qv, c, w, l, u, X, max_iters, moves_cap, lanes):
    """The arguments of one Algorithm 1 run and the output tensors it fills
    (fval, moves, nmoves) and its workspace."""
    import torch
    K, ldg = G.shape
    S = X.shape[0]
    dev = X.device
    fval = torch.empty(S, dtype=torch.int64, device=dev)
    moves = torch.zeros((S, moves_cap, 4), dtype=torch.int64, device=dev) if moves_cap else None
    nmoves = torch.zeros(S, dtype=torch.int32, device=dev)
    ws = _workspace(lib().mape_augment_workspace_bytes(n, S, K), dev)
    A = AugmentArgs()
    A.n, A.S, A.K, A.G, A.ldg, A.score_lanes = n, S, K, _ptr(G), ldg, lanes
    A.a, A.q4 = _ptr(a), _ptr(q4)
    A.q_row, A.q_col, A.q_val, A.nnz = _ptr(qr), _ptr(qc), _ptr(qv), qv.numel()
    A.c, A.w, A.l, A.u = _ptr(c), _ptr(w), _ptr(l), _ptr(u)
    A.X, A.fval = _ptr(X), _ptr(fval)
    A.moves, A.nmoves, A.moves_cap = _ptr(moves), _ptr(nmoves), moves_cap
    A.max_iters = max_iters
    A.workspace, A.workspace_bytes = _ptr(ws), ws.numel()
    return A, (fval, moves, nmoves, ws)


def augment_run(G, n, a, q4, qr, qc, qv, c, w, l, u, X, *, max_iters=10 ** 6, moves_cap=0, lanes=0, stream=None):
    """a13-a14: Algorithm 1 in place on X [S,n]; returns (fval, iters, moves,
    nmoves).  lanes: lanes per direction of the scoring pass (0: autotuned)."""
    A, (fval, moves, nmoves, _ws) = _augment_args(G, n, a, q4, qr, qc, qv, c, w, l, u, X, max_iters, moves_cap,
                                                  lanes)
    iters = I64(0)
    _check(lib().mape_augment_run(C.byref(A), C.byref(iters), _stream(stream)), "mape_augment_run")
    return fval, iters.value, moves, nmoves


_DONE_FN = C.CFUNCTYPE(None, I32, I64, C.c_void_p)


def augment_run_batch(runs, *, stream=None, on_done=None):
    """mape_augment_run_batch: Algorithm 1 for several instances in one
    sequence of launches.  runs: dicts of augment_run's arguments (G, n, a,
    q4, qr, qc, qv, c, w, l, u, X, and optionally max_iters, moves_cap,
    lanes).  on_done(item, iters) is called as each run's iterations end.
    Returns one (fval, iters, moves, nmoves) per run."""
    k = len(runs)
    args, outs = [], []
    for r in runs:
        A, o = _augment_args(r["G"], r["n"], r["a"], r["q4"], r["qr"], r["qc"], r["qv"], r["c"], r["w"], r["l"],
                             r["u"], r["X"], r.get("max_iters", 10 ** 6), r.get("moves_cap", 0), r.get("lanes", 0))
        args.append(A)
        outs.append(o)
    items = (AugmentArgs * k)(*args)
    iters = (I64 * k)()
    dev = runs[0]["X"].device
    ws = _workspace(lib().mape_augment_run_batch_workspace_bytes(k), dev)
    cb = _DONE_FN(lambda i, it, _ctx: on_done(int(i), int(it))) if on_done is not None else None
    _check(lib().mape_augment_run_batch(items, k, iters, _ptr(ws), ws.numel(), _stream(stream),
                                        C.cast(cb, C.c_void_p) if cb is not None else None, None),
           "mape_augment_run_batch")
    return [(fval, int(iters[i]), moves, nmoves) for i, (fval, moves, nmoves, _w) in enumerate(outs)]


def augment_tune_lookup(n, K, S, quartic):
    """The autotuned lane count of the scoring pass for a shape, or None."""
    info = AugTuneInfo()
    rc = lib().mape_augment_tune_lookup(n, K, S, 1 if quartic else 0, C.byref(info))
    if rc != OK:
        return None
    c = info.candidates
    return {"lanes": info.lanes, "cand_lanes": list(info.cand_lanes[:c]), "probe_ms": list(info.probe_ms[:c])}


# ---- instance handle (host numpy arrays) ------------------------------------

def _np(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _host(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def extract_directions_batch(handles, starts):
    """mape_extract_directions_batch: Algorithm 2 for several Instance handles
    at once.  starts: one (P, Z0, G0) per handle (host float32 arrays, one of
    Z0 / G0 None)."""
    k = len(handles)
    hs = (P_ * k)(*[h.h for h in handles])
    Ps = (I32 * k)(*[int(P) for P, _, _ in starts])
    keep = []

    def arr(x):
        if x is None:
            return None
        x = _np(x, np.float32)
        keep.append(x)
        return x.ctypes.data

    Z = (P_ * k)(*[arr(z) for _, z, _ in starts])
    G = (P_ * k)(*[arr(g) for _, _, g in starts])
    for h, x in zip(handles, keep):
        h._keep["batch_start"] = x
    for h in handles:
        h._keep["batch_starts_all"] = keep
    _check(lib().mape_extract_directions_batch(hs, k, Ps, Z, G), "mape_extract_directions_batch")


def augment_batch(handles, starts):
    """mape_augment_batch: Algorithm 1 for several Instance handles at once.
    starts: one X0 [S x n] int32 host array per handle."""
    k = len(handles)
    hs = (P_ * k)(*[h.h for h in handles])
    keep = [_np(np.atleast_2d(x), np.int32) for x in starts]
    X = (P_ * k)(*[x.ctypes.data for x in keep])
    S = (I32 * k)(*[x.shape[0] for x in keep])
    for h, x in zip(handles, keep):
        h._keep["x0"] = x
    _check(lib().mape_augment_batch(hs, k, X, S), "mape_augment_batch")


class Instance:
    """mape_create_instance ... mape_destroy over host arrays."""

    def __init__(self, A, b, l, u, Q, c, w, B, cfg: Config | None = None, stream=None):
        self._keep = {}
        self.m, self.n = A.shape
        self.cfg = cfg if cfg is not None else default_config()
        arrs = dict(A=_np(A, np.int32), b=_np(b, np.int64), l=_np(l, np.int32), u=_np(u, np.int32),
                    B=_np(B, np.int32))
        self._keep.update(arrs)
        prob = self._problem(Q, c, w)
        h = C.c_void_p()
        st = C.c_void_p(stream.cuda_stream) if stream is not None else None
        _check(lib().mape_create_instance(_host(arrs["A"]), _host(arrs["b"]), _host(arrs["l"]),
                                          _host(arrs["u"]), C.byref(prob), _host(arrs["B"]),
                                          C.byref(self.cfg), st, C.byref(h)), "mape_create_instance")
        self.h = h

    def _problem(self, Q, c, w):
        Qa, ca = _np(Q, np.int32), _np(c, np.int32)
        wa = None if w is None else _np(w, np.int32)
        self._keep.update(Q=Qa, c=ca, w=wa)
        return Problem(self.n, self.m, _host(Qa), _host(ca), _host(wa))

    @classmethod
    def from_generated(cls, inst, cfg=None, stream=None):
        return cls(inst.A, inst.b, inst.l, inst.u, inst.Q, inst.c, inst.w, inst.B, cfg, stream)

    def extract_directions(self, P, Z0=None, G0=None):
        """Z0/G0: host numpy float32 arrays or CUDA torch tensors."""
        def arg(x):
            if x is None:
                return None
            if hasattr(x, "data_ptr"):
                self._keep["start_dev"] = x
                return C.c_void_p(x.data_ptr())
            x = _np(x, np.float32)
            self._keep["start"] = x
            return _host(x)
        _check(lib().mape_extract_directions(self.h, P, arg(Z0), arg(G0)), "mape_extract_directions")

    def augment(self, X0, f=None):
        if hasattr(X0, "data_ptr"):
            self._keep["x0_dev"] = X0
            ptr, S = C.c_void_p(X0.data_ptr()), X0.shape[0]
        else:
            X0 = _np(np.atleast_2d(X0), np.int32)
            self._keep["x0"] = X0
            ptr, S = _host(X0), X0.shape[0]
        prob = None if f is None else C.byref(self._problem(*f))
        _check(lib().mape_augment(self.h, ptr, S, prob), "mape_augment")

    def poll(self) -> dict:
        st = Status()
        _check(lib().mape_poll(self.h, C.byref(st)), "mape_poll")
        return st.as_dict()

    def wait(self, timeout_s: float = 600.0):
        rc = lib().mape_wait(self.h, int(timeout_s * 1e9))
        _check(rc, "mape_wait")

    def cancel(self):
        _check(lib().mape_cancel(self.h), "mape_cancel")

    def directions(self) -> np.ndarray:
        K = I64(0)
        rc = lib().mape_get_directions(self.h, None, 0, C.byref(K))
        if rc not in (OK, -7):
            _check(rc, "mape_get_directions")
        out = np.empty((K.value, self.n), dtype=np.int32)
        _check(lib().mape_get_directions(self.h, _host(out), K.value, C.byref(K)), "mape_get_directions")
        return out

    def directions_i8(self, out=None) -> np.ndarray:
        """The direction set as int8 rows [K x n] (no conversion on the
        device).  `out` may be a caller-owned host array (e.g. the numpy view
        of a pinned torch tensor) with at least K rows of at least n int8;
        the rows are written there and a view of the first K is returned."""
        K = I64(0)
        rc = lib().mape_get_directions_i8(self.h, None, 0, self.n, C.byref(K))
        if rc not in (OK, -7):
            _check(rc, "mape_get_directions_i8")
        if out is None:
            out = np.empty((K.value, self.n), dtype=np.int8)
        if out.dtype != np.int8 or out.ndim != 2 or out.shape[0] < K.value or out.shape[1] < self.n \
                or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous int8 array of at least K x n")
        _check(lib().mape_get_directions_i8(self.h, out.ctypes.data_as(C.c_void_p), out.shape[0], out.shape[1],
                                            C.byref(K)), "mape_get_directions_i8")
        return out[: K.value, : self.n]

    def initial_solutions(self, X0, T=1000, period=1):
        """Eq. (4) from the starts X0 [P x n] (host float32): the distinct
        feasible points found, [S x n] int32."""
        X0 = _np(X0, np.float32)
        S = I32(0)
        cap = min(X0.shape[0] * (T // period + 1), 1 << 16)
        out = np.empty((cap, self.n), dtype=np.int32)
        rc = lib().mape_find_initial_solutions(self.h, X0.shape[0], _host(X0), T, period, _host(out), cap, C.byref(S))
        if rc == -7 and S.value > cap:  # more distinct points than the first buffer held: run again with room
            out = np.empty((S.value, self.n), dtype=np.int32)
            rc = lib().mape_find_initial_solutions(self.h, X0.shape[0], _host(X0), T, period, _host(out), S.value,
                                                   C.byref(S))
        _check(rc, "mape_find_initial_solutions")
        return out[: S.value]

    def solution(self):
        x = np.empty(self.n, dtype=np.int32)
        f = I64(0)
        _check(lib().mape_get_solution(self.h, _host(x), C.byref(f)), "mape_get_solution")
        return x, f.value

    def solutions(self, S):
        X = np.empty((S, self.n), dtype=np.int32)
        f = np.empty(S, dtype=np.int64)
        _check(lib().mape_get_solutions(self.h, _host(X), _host(f), S), "mape_get_solutions")
        return X, f

    def close(self):
        if getattr(self, "h", None):
            lib().mape_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- request server (host numpy arrays) --------------------------------------

class Server:
    """mape_server_create ... mape_server_destroy: continuous batching of
    instances on one GPU, admitted by device memory."""

    def __init__(self, cfg: Config | None = None, mem_cap_bytes: int = 150 << 30, max_slots: int = 8,
                 keep_directions: bool = False, batch_extraction: bool = False):
        sc = ServerConfig()
        sc.cfg = cfg if cfg is not None else default_config()
        sc.mem_cap_bytes, sc.max_slots, sc.keep_directions = int(mem_cap_bytes), int(max_slots), int(keep_directions)
        sc.batch_extraction = int(batch_extraction)
        self.cfg = sc.cfg
        h = C.c_void_p()
        _check(lib().mape_server_create(C.byref(sc), C.byref(h)), "mape_server_create")
        self.h = h
        self._n = {}

    def submit(self, inst, P, Z0=None, G0=None, X0=None) -> int:
        """Queues a generated instance with P starts (Z0 [P x d] or G0 [P x n])
        and augmentation starts X0 [S x n] (default: x̄)."""
        A, b, l, u, B = (_np(inst.A, np.int32), _np(inst.b, np.int64), _np(inst.l, np.int32),
                         _np(inst.u, np.int32), _np(inst.B, np.int32))
        Q, c = _np(inst.Q, np.int32), _np(inst.c, np.int32)
        w = None if inst.w is None else _np(inst.w, np.int32)
        X0 = _np(np.atleast_2d(inst.xbar if X0 is None else X0), np.int32)
        Z0 = None if Z0 is None else _np(Z0, np.float32)
        G0 = None if G0 is None else _np(G0, np.float32)
        m, n = A.shape
        prob = Problem(n, m, _host(Q), _host(c), _host(w))
        rid = C.c_uint64(0)
        _check(lib().mape_server_submit(self.h, _host(A), _host(b), _host(l), _host(u), C.byref(prob), _host(B), P,
                                        _host(Z0), _host(G0), _host(X0), X0.shape[0], C.byref(rid)),
               "mape_server_submit")
        self._n[rid.value] = n
        return rid.value

    def info(self, rid) -> dict:
        st = RequestInfo()
        _check(lib().mape_server_poll(self.h, rid, C.byref(st)), "mape_server_poll")
        return st.as_dict()

    def wait(self, rid, timeout_s: float = 600.0):
        _check(lib().mape_server_wait(self.h, rid, int(timeout_s * 1e9)), "mape_server_wait")

    def wait_all(self, timeout_s: float = 3600.0):
        _check(lib().mape_server_wait_all(self.h, int(timeout_s * 1e9)), "mape_server_wait_all")

    def result(self, rid, directions: bool = False):
        n = self._n[rid]
        x = np.empty(n, dtype=np.int32)
        f = I64(0)
        K = I64(0)
        _check(lib().mape_server_result(self.h, rid, _host(x), C.byref(f), None, 0, C.byref(K)), "mape_server_result")
        if not directions:
            return x, f.value
        G = np.empty((K.value, n), dtype=np.int8)
        _check(lib().mape_server_result(self.h, rid, None, None, _host(G), K.value, C.byref(K)), "mape_server_result")
        return x, f.value, G

    def release(self, rid):
        _check(lib().mape_server_release(self.h, rid), "mape_server_release")

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().mape_server_get_stats(self.h, C.byref(st)), "mape_server_get_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            lib().mape_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


TIMED_KINDS = ("stream_fwd", "stream_collect", "stream_grad", "resident")


def launch_timing(enable: bool):
    """Switches the library's per-launch CUDA-event timing of the extraction
    kernels on or off (mape_launch_timing) and clears its sums."""
    _check(lib().mape_launch_timing(int(enable)), "mape_launch_timing")


def launch_timing_read() -> dict:
    """{kind: (summed ms, launches)} of the timed launches so far
    (mape_launch_timing_read; synchronises on the recorded events)."""
    ms = (C.c_double * len(TIMED_KINDS))()
    cnt = (I64 * len(TIMED_KINDS))()
    _check(lib().mape_launch_timing_read(ms, cnt), "mape_launch_timing_read")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(TIMED_KINDS)}


def mma_issue_probe(kind, M, N, accumulators=1, chain=512):
    """SM cycles per tcgen05.mma instruction (issue, issue + completion) for a
    chain of `chain` instructions (mape_mma_issue_probe; kind 0 BF16 K = 16,
    kind 1 e4m3 K = 32)."""
    a, b = C.c_double(0), C.c_double(0)
    _check(lib().mape_mma_issue_probe(kind, M, N, accumulators, chain, C.byref(a), C.byref(b)),
           "mape_mma_issue_probe")
    return a.value, b.value


def trim_memory():
    """Hands back the memory that the library's pool on the current device
    keeps reserved beyond the live handles (mape_trim_memory)."""
    _check(lib().mape_trim_memory(), "mape_trim_memory")


def request_bytes(n, m, P, S, cfg: Config | None = None) -> int:
    cfg = cfg if cfg is not None else default_config()
    return int(lib().mape_request_bytes(n, m, P, S, C.byref(cfg)))


def inequality_extension(inst, G, h):
    """The instance with G x >= h added, in equality form with slacks
    (mape_inequality_extension, _objective and _points): a copy of `inst` with
    n + m2 variables whose objective ignores the slacks and whose xbar carries
    the slacks G xbar - h."""
    import dataclasses
    G = _np(np.atleast_2d(G), np.int32)
    h = _np(np.atleast_1d(h), np.int64)
    n, m, m2, d = inst.n, inst.m, G.shape[0], inst.d
    A, b, l, u, B = (_np(inst.A, np.int32), _np(inst.b, np.int64), _np(inst.l, np.int32), _np(inst.u, np.int32),
                     _np(inst.B, np.int32))
    A2 = np.empty((m + m2, n + m2), np.int32)
    b2 = np.empty(m + m2, np.int64)
    l2 = np.empty(n + m2, np.int32)
    u2 = np.empty(n + m2, np.int32)
    B2 = np.empty((n + m2, d), np.int32)
    _check(lib().mape_inequality_extension(n, m, m2, _host(A), _host(b), _host(l), _host(u), _host(G), _host(h),
                                           _host(B), _host(A2), _host(b2), _host(l2), _host(u2), _host(B2)),
           "mape_inequality_extension")
    Q, c = _np(inst.Q, np.int32), _np(inst.c, np.int32)
    w = None if inst.w is None else _np(inst.w, np.int32)
    Q2 = np.empty((n + m2, n + m2), np.int32)
    c2 = np.empty(n + m2, np.int32)
    w2 = None if w is None else np.empty(n + m2, np.int32)
    _check(lib().mape_inequality_extension_objective(n, m2, _host(Q), _host(c), _host(w), _host(Q2), _host(c2),
                                                     _host(w2)), "mape_inequality_extension_objective")
    x = _np(inst.xbar[None, :], np.int32)
    x2 = np.empty((1, n + m2), np.int32)
    _check(lib().mape_inequality_extension_points(n, m2, _host(G), _host(h), _host(x), 1, _host(x2)),
           "mape_inequality_extension_points")
    return dataclasses.replace(inst, name=inst.name + f"_ineq{m2}", n=n + m2, m=m + m2, A=A2, b=b2, l=l2, u=u2,
                               B=B2, Q=Q2, c=c2, w=w2, xbar=x2[0])


def kernel_basis(A, reduce: bool = True) -> np.ndarray:
    """A basis of Ker_Z(A) for a general full-row-rank A (mape_kernel_basis):
    [n x (n - m)] int32, LLL-reduced unless reduce=False."""
    A = _np(np.atleast_2d(A), np.int32)
    m, n = A.shape
    B = np.empty((n, n - m), np.int32)
    _check(lib().mape_kernel_basis(m, n, _host(A), int(reduce), _host(B)), "mape_kernel_basis")
    return B


def autotune_info(n, d, P, precision=PREC_BF16):
    """The autotuned choice for a shape (mape_autotune_lookup), or None."""
    info = TuneInfo()
    rc = lib().mape_autotune_lookup(n, d, P, precision, C.byref(info))
    return None if rc != OK else info.as_dict()
