"""Thin ctypes binding of libtileqr (include/tileqr.h).

Argument marshalling only: every step of the factorization, Q^T application
and solve runs in the library's CUDA kernels.  PyTorch provides the device
memory (the caller-side workspace) and the current CUDA stream.  There is no
CPU fallback: if the compiled library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtileqr.so")

TILEQR_FP64, TILEQR_TF32, TILEQR_SPLIT_BF16 = 0, 1, 2
TILEQR_SCHED_DAG, TILEQR_SCHED_BULK = 0, 1
TILEQR_FLAG_NONE, TILEQR_FLAG_TEST_WITHHOLD_LAST_TASK, TILEQR_FLAG_TEST_RANDOM_DELAYS = 0, 1, 2
TILEQR_ERR_CUDA = 1001
TILEQR_ERR_TIMEOUT = 1002
TILEQR_ERR_NONFINITE = 1003
TILEQR_ERR_WORKSPACE = 1004
TILEQR_ERR_SINGULAR = 1005
TILEQR_ERR_UNSUPPORTED = 1006
TILEQR_ERR_SCRATCH_LIMIT = 1007
TILEQR_ERR_NOT_SPD = 1008
TILEQR_UPDATE_LARFB, TILEQR_UPDATE_SSRFB = 0, 1
TILEQR_MIXED_UPDATE_WS_BYTES = 388 * 1024

EXPORTED = [
    "tileqr_workspace_size", "tileqr_factor", "tileqr_status", "tileqr_get_R",
    "tileqr_get_factors", "tileqr_apply_workspace_size", "tileqr_apply_qt", "tileqr_solve_ls",
    "tileqr_strerror", "tileqr_launch_count", "tileqr_reset_launch_count",
    "tileqr_set_profile_events", "tileqr_factor_noalloc", "tileqr_set_trace", "tileqr_trace_count",
    "tileqr_refine_workspace_size", "tileqr_solve_refine",
    "tileqr_batched_workspace_size", "tileqr_batched_prepare", "tileqr_factor_batched",
    "tileqr_batched_status", "tileqr_batched_get",
    "tileqr_workspace_size_tree", "tileqr_factor_tree", "tileqr_get_tree_T", "tileqr_task_graph",
    "tileqr_apply_q", "tileqr_form_q",
    "tileqr_cholesky_workspace_size", "tileqr_cholesky", "tileqr_cholesky_get_L", "tileqr_cholesky_info",
    "tileqr_lu_workspace_size", "tileqr_lu", "tileqr_lu_info", "tileqr_lu_get_factors",
    "tileqr_lu_solve_workspace_size", "tileqr_lu_solve", "tileqr_mixed_update_tile",
    "tileqr_ls_refine_workspace_size", "tileqr_solve_ls_refine",
    "tileqr_batched_ls_workspace_size", "tileqr_batched_solve_ls", "tileqr_measure_fp64_rates",
    "tileqr_apply_mixed_workspace_size", "tileqr_apply_mixed",
]


class tileqr_desc(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64), ("n", ctypes.c_int64),
        ("nb", ctypes.c_int32), ("ib", ctypes.c_int32),
        ("p", ctypes.c_int32), ("q", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("schedule", ctypes.c_int32),
        ("tiles", ctypes.c_void_p), ("T", ctypes.c_void_p),
        ("sched", ctypes.c_void_p), ("sched_bytes", ctypes.c_size_t),
        ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
        ("domain", ctypes.c_int32), ("reserved", ctypes.c_int32), ("T2", ctypes.c_void_p),
    ]


class tileqr_refine_info(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("inner_iterations", ctypes.c_int), ("method", ctypes.c_int),
        ("converged", ctypes.c_int), ("initial_rel_residual", ctypes.c_double),
        ("rel_residual", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class tileqr_batch(ctypes.Structure):
    _fields_ = [
        ("count", ctypes.c_int), ("nb", ctypes.c_int), ("ib", ctypes.c_int), ("precision", ctypes.c_int),
        ("total_tasks", ctypes.c_uint64), ("cap", ctypes.c_uint32 * 4),
        ("off_ctrl", ctypes.c_size_t), ("off_cnt", ctypes.c_size_t), ("off_q", ctypes.c_size_t * 4),
        ("off_mats", ctypes.c_size_t), ("sched_bytes", ctypes.c_size_t),
        ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t), ("flops", ctypes.c_double),
    ]


class TileQRError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {code} ({strerror(code)})")


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libtileqr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libtileqr.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    i64, i32, vp, sz = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t
    dp = ctypes.POINTER(tileqr_desc)
    sig = {
        "tileqr_workspace_size": (i32, [i64, i64, i32, i32, i32, ctypes.POINTER(sz)]),
        "tileqr_factor": (i32, [i64, i64, vp, i64, i32, i32, i32, i32, i32, vp, sz, vp, dp]),
        "tileqr_status": (i32, [dp, vp]),
        "tileqr_get_R": (i32, [dp, vp, i64, vp]),
        "tileqr_get_factors": (i32, [dp, vp, i64, vp, i64, vp]),
        "tileqr_apply_workspace_size": (i32, [dp, i64, ctypes.POINTER(sz)]),
        "tileqr_apply_qt": (i32, [dp, vp, i64, i64, vp, sz, vp]),
        "tileqr_apply_mixed_workspace_size": (i32, [dp, i64, ctypes.POINTER(sz)]),
        "tileqr_apply_mixed": (i32, [dp, i32, vp, i64, i64, vp, sz, vp]),
        "tileqr_solve_ls": (i32, [dp, vp, i64, i64, vp, sz, vp]),
        "tileqr_strerror": (ctypes.c_char_p, [i32]),
        "tileqr_launch_count": (ctypes.c_uint64, []),
        "tileqr_reset_launch_count": (None, []),
        "tileqr_set_profile_events": (None, [vp, vp]),
        "tileqr_factor_noalloc": (i32, [i64, i64, vp, i64, i32, i32, vp, sz, vp, sz, vp, dp]),
        "tileqr_set_trace": (None, [vp, ctypes.c_uint64]),
        "tileqr_refine_workspace_size": (i32, [dp, ctypes.POINTER(sz)]),
        "tileqr_batched_workspace_size": (i32, [i32, vp, vp, i32, i32, i32, ctypes.POINTER(sz)]),
        "tileqr_batched_prepare": (i32, [i32, vp, vp, vp, vp, i32, i32, i32, vp, sz, vp,
                                         ctypes.POINTER(tileqr_batch)]),
        "tileqr_factor_batched": (i32, [ctypes.POINTER(tileqr_batch), vp]),
        "tileqr_batched_status": (i32, [ctypes.POINTER(tileqr_batch), vp]),
        "tileqr_batched_get": (i32, [ctypes.POINTER(tileqr_batch), i32, dp]),
        "tileqr_solve_refine": (i32, [dp, vp, i64, vp, vp, i32, ctypes.c_double, vp, sz, vp,
                                      ctypes.POINTER(tileqr_refine_info)]),
        "tileqr_trace_count": (i32, [dp, vp, ctypes.POINTER(ctypes.c_uint64)]),
        "tileqr_workspace_size_tree": (i32, [i64, i64, i32, i32, i32, i32, ctypes.POINTER(sz)]),
        "tileqr_factor_tree": (i32, [i64, i64, vp, i64, i32, i32, i32, i32, i32, vp, sz, vp, dp]),
        "tileqr_get_tree_T": (i32, [dp, vp, i64, vp]),
        "tileqr_apply_q": (i32, [dp, vp, i64, i64, vp, sz, vp]),
        "tileqr_form_q": (i32, [dp, vp, i64, i64, vp, sz, vp]),
        "tileqr_cholesky_workspace_size": (i32, [i64, i32, ctypes.POINTER(sz)]),
        "tileqr_cholesky": (i32, [i64, vp, i64, i32, i32, vp, sz, vp, dp]),
        "tileqr_cholesky_get_L": (i32, [dp, vp, i64, vp]),
        "tileqr_cholesky_info": (i32, [dp, vp, ctypes.POINTER(i64)]),
        "tileqr_lu_workspace_size": (i32, [i64, i32, i32, ctypes.POINTER(sz)]),
        "tileqr_lu": (i32, [i64, vp, i64, i32, i32, i32, vp, sz, vp, dp]),
        "tileqr_lu_info": (i32, [dp, vp, ctypes.POINTER(i64)]),
        "tileqr_lu_get_factors": (i32, [dp, vp, i64, vp, i64, vp, i64, vp]),
        "tileqr_lu_solve_workspace_size": (i32, [dp, i64, ctypes.POINTER(sz)]),
        "tileqr_lu_solve": (i32, [dp, vp, i64, i64, vp, sz, vp]),
        "tileqr_mixed_update_tile": (i32, [i32, i32, vp, vp, vp, vp, vp, sz, vp]),
        "tileqr_measure_fp64_rates": (i32, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]),
        "tileqr_ls_refine_workspace_size": (i32, [dp, i64, ctypes.POINTER(sz)]),
        "tileqr_batched_ls_workspace_size": (i32, [ctypes.POINTER(tileqr_batch), ctypes.POINTER(sz)]),
        "tileqr_batched_solve_ls": (i32, [ctypes.POINTER(tileqr_batch), vp, vp, i32, ctypes.c_double, vp, sz, vp,
                                          ctypes.POINTER(tileqr_refine_info)]),
        "tileqr_solve_ls_refine": (i32, [dp, vp, i64, vp, i64, i64, vp, i64, vp, i64, i32, ctypes.c_double, vp,
                                         sz, vp, ctypes.POINTER(tileqr_refine_info)]),
        "tileqr_task_graph": (i32, [i64, i64, i32, i32, i32, vp, vp, vp, vp, ctypes.POINTER(i64),
                                    ctypes.POINTER(i64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load().tileqr_strerror(int(code)).decode()
    except ImportError:
        return "library not loaded"


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(rc: int, where: str):
    if rc != 0:
        raise TileQRError(rc, where)


def as_colmajor(A: torch.Tensor) -> torch.Tensor:
    """A float64 CUDA tensor of shape (m, n) laid out column-major (stride (1, ld))."""
    if A.dim() == 1:
        A = A.reshape(-1, 1)
    if A.dtype != torch.float64:
        raise TypeError("tileqr works on float64 matrices")
    if not A.is_cuda:
        raise TypeError("tileqr needs CUDA tensors")
    m, n = A.shape
    if A.stride(0) == 1 and (n <= 1 or A.stride(1) >= max(m, 1)):
        return A
    return A.t().contiguous().t()


def colmajor_empty(m: int, n: int, device="cuda") -> torch.Tensor:
    return torch.empty((n, m), dtype=torch.float64, device=device).t()


def to_device_colmajor(a, device="cuda") -> torch.Tensor:
    """Copy a host matrix (numpy or torch) into a column-major device tensor."""
    t = torch.as_tensor(a, dtype=torch.float64)
    if t.dim() == 1:
        t = t.reshape(-1, 1)
    m, n = t.shape
    out = colmajor_empty(m, n, device)
    out.copy_(t)
    return out


def _ld(A: torch.Tensor) -> int:
    return max(int(A.stride(1)) if A.shape[1] > 1 else A.shape[0], 1)


# ---------------------------------------------------------------------------
# The C entry points, same names.
def tileqr_workspace_size(m: int, n: int, nb: int, ib: int, precision: int = TILEQR_FP64) -> int:
    out = ctypes.c_size_t(0)
    _check(load().tileqr_workspace_size(m, n, nb, ib, precision, ctypes.byref(out)), "tileqr_workspace_size")
    return out.value


def tileqr_factor(A: torch.Tensor, nb: int, ib: int, precision: int = TILEQR_FP64,
                  schedule: int = TILEQR_SCHED_DAG, flags: int = 0, workspace: torch.Tensor | None = None,
                  stream=None) -> "Factorization":
    A = as_colmajor(A)
    m, n = A.shape
    need = tileqr_workspace_size(m, n, nb, ib, precision)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=A.device)
    d = tileqr_desc()
    rc = load().tileqr_factor(m, n, ctypes.c_void_p(A.data_ptr()), _ld(A), nb, ib, precision, schedule,
                              flags, ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                              _stream_ptr(stream), ctypes.byref(d))
    _check(rc, "tileqr_factor")
    return Factorization(d, workspace, A.device)


def tileqr_workspace_size_tree(m: int, n: int, nb: int, ib: int, precision: int = TILEQR_FP64,
                               domain: int = 0) -> int:
    out = ctypes.c_size_t(0)
    _check(load().tileqr_workspace_size_tree(m, n, nb, ib, precision, domain, ctypes.byref(out)),
           "tileqr_workspace_size_tree")
    return out.value


def tileqr_factor_tree(A: torch.Tensor, nb: int, ib: int, domain: int, precision: int = TILEQR_FP64,
                       flags: int = 0, workspace: torch.Tensor | None = None, stream=None) -> "Factorization":
    """Tree form (domains of `domain` tile rows, heads merged pairwise)."""
    A = as_colmajor(A)
    m, n = A.shape
    need = tileqr_workspace_size_tree(m, n, nb, ib, precision, domain)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=A.device)
    d = tileqr_desc()
    rc = load().tileqr_factor_tree(m, n, ctypes.c_void_p(A.data_ptr()), _ld(A), nb, ib, domain, precision, flags,
                                   ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream_ptr(stream),
                                   ctypes.byref(d))
    _check(rc, "tileqr_factor_tree")
    return Factorization(d, workspace, A.device)


def tileqr_task_graph(m: int, n: int, nb: int, domain: int = 0, what: int = 0):
    """(tasks, ndeps, succ_ptr, succ) of the executed task graph, as numpy
    arrays (host only; no GPU needed)."""
    import numpy as np
    lib = load()
    nt, ne = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib.tileqr_task_graph(m, n, nb, domain, what, None, None, None, None, ctypes.byref(nt),
                                 ctypes.byref(ne)), "tileqr_task_graph")
    tasks = np.zeros((nt.value, 4), dtype=np.int32)
    ndeps = np.zeros(nt.value, dtype=np.int32)
    ptr = np.zeros(nt.value + 1, dtype=np.int64)
    succ = np.zeros(max(ne.value, 1), dtype=np.int64)
    vp = ctypes.c_void_p
    _check(lib.tileqr_task_graph(m, n, nb, domain, what, vp(tasks.ctypes.data), vp(ndeps.ctypes.data),
                                 vp(ptr.ctypes.data), vp(succ.ctypes.data), ctypes.byref(nt), ctypes.byref(ne)),
           "tileqr_task_graph")
    return tasks, ndeps, ptr, succ[:ne.value]


def tileqr_cholesky_workspace_size(n: int, nb: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().tileqr_cholesky_workspace_size(n, nb, ctypes.byref(out)), "tileqr_cholesky_workspace_size")
    return out.value


def tileqr_cholesky(A: torch.Tensor, nb: int = 128, workspace: torch.Tensor | None = None,
                    stream=None) -> "CholeskyFactorization":
    """Tiled Cholesky A = L L^T of an SPD matrix (only its lower triangle is read)."""
    A = as_colmajor(A)
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("tileqr_cholesky needs a square matrix")
    need = tileqr_cholesky_workspace_size(n, nb)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=A.device)
    d = tileqr_desc()
    rc = load().tileqr_cholesky(n, ctypes.c_void_p(A.data_ptr()), _ld(A), nb, 0,
                                ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream_ptr(stream),
                                ctypes.byref(d))
    _check(rc, "tileqr_cholesky")
    return CholeskyFactorization(d, workspace, A.device)


class CholeskyFactorization:
    """A tiled Cholesky factorization in a caller-owned (torch) workspace."""

    def __init__(self, desc: tileqr_desc, workspace: torch.Tensor, device):
        self.desc, self.workspace, self.device = desc, workspace, device

    def status(self, stream=None) -> int:
        return load().tileqr_status(ctypes.byref(self.desc), _stream_ptr(stream))

    def check(self, stream=None):
        _check(self.status(stream), "tileqr_cholesky")
        return self

    def info(self, stream=None) -> int:
        out = ctypes.c_int64(0)
        _check(load().tileqr_cholesky_info(ctypes.byref(self.desc), _stream_ptr(stream), ctypes.byref(out)),
               "tileqr_cholesky_info")
        return int(out.value)

    def L(self, stream=None) -> torch.Tensor:
        n = self.desc.n
        L = colmajor_empty(n, n, self.device)
        _check(load().tileqr_cholesky_get_L(ctypes.byref(self.desc), ctypes.c_void_p(L.data_ptr()), max(n, 1),
                                            _stream_ptr(stream)), "tileqr_cholesky_get_L")
        return L


def tileqr_lu_workspace_size(n: int, nb: int, ib: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().tileqr_lu_workspace_size(n, nb, ib, ctypes.byref(out)), "tileqr_lu_workspace_size")
    return out.value


def tileqr_lu(A: torch.Tensor, nb: int = 128, ib: int = 16, workspace: torch.Tensor | None = None,
              stream=None, flags: int = 0) -> "LUFactorization":
    """Tiled LU with tiled pairwise pivoting (Algorithm 3) of a square FP64 matrix."""
    A = as_colmajor(A)
    n = A.shape[0]
    if A.shape[1] != n:
        raise ValueError("tileqr_lu needs a square matrix")
    need = tileqr_lu_workspace_size(n, nb, ib)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=A.device)
    d = tileqr_desc()
    rc = load().tileqr_lu(n, ctypes.c_void_p(A.data_ptr()), _ld(A), nb, ib, flags,
                          ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream_ptr(stream),
                          ctypes.byref(d))
    _check(rc, "tileqr_lu")
    return LUFactorization(d, workspace, A.device)


class LUFactorization:
    """A tiled LU factorization (N U = A) in a caller-owned (torch) workspace."""

    def __init__(self, desc: tileqr_desc, workspace: torch.Tensor, device):
        self.desc, self.workspace, self.device = desc, workspace, device
        self._solve_ws = None

    def status(self, stream=None) -> int:
        return load().tileqr_status(ctypes.byref(self.desc), _stream_ptr(stream))

    def check(self, stream=None):
        _check(self.status(stream), "tileqr_lu")
        return self

    def info(self, stream=None) -> int:
        out = ctypes.c_int64(0)
        _check(load().tileqr_lu_info(ctypes.byref(self.desc), _stream_ptr(stream), ctypes.byref(out)),
               "tileqr_lu_info")
        return int(out.value)

    def factors(self, stream=None):
        """(F, Lx, piv): F n x n (U and the multipliers), Lx (p*ib) x n, piv
        p x n int32, all column-major device tensors."""
        d = self.desc
        n, p, ib = d.n, d.p, d.ib
        F = colmajor_empty(n, n, self.device)
        Lx = colmajor_empty(max(p * ib, 1), n, self.device)
        piv = torch.empty((n, max(p, 1)), dtype=torch.int32, device=self.device).t()
        _check(load().tileqr_lu_get_factors(ctypes.byref(d), ctypes.c_void_p(F.data_ptr()), max(n, 1),
                                            ctypes.c_void_p(Lx.data_ptr()), max(p * ib, 1),
                                            ctypes.c_void_p(piv.data_ptr()), max(p, 1), _stream_ptr(stream)),
               "tileqr_lu_get_factors")
        return F, Lx, piv

    def solve(self, B: torch.Tensor, stream=None) -> torch.Tensor:
        """A^{-1} B (B: n x nrhs or n, FP64 on the device), in a new tensor."""
        vec = B.dim() == 1
        Bm = as_colmajor(B.reshape(-1, 1) if vec else B)
        X = colmajor_empty(Bm.shape[0], Bm.shape[1], self.device)
        X.copy_(Bm)
        nrhs = X.shape[1]
        need = ctypes.c_size_t(0)
        _check(load().tileqr_lu_solve_workspace_size(ctypes.byref(self.desc), nrhs, ctypes.byref(need)),
               "tileqr_lu_solve_workspace_size")
        if self._solve_ws is None or self._solve_ws.numel() < need.value:
            self._solve_ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device=self.device)
        _check(load().tileqr_lu_solve(ctypes.byref(self.desc), ctypes.c_void_p(X.data_ptr()), _ld(X), nrhs,
                                      ctypes.c_void_p(self._solve_ws.data_ptr()), self._solve_ws.numel(),
                                      _stream_ptr(stream)), "tileqr_lu_solve")
        return X.reshape(-1) if vec else X


class Factorization:
    """A factorization living in a caller-owned (torch) workspace."""

    def __init__(self, desc: tileqr_desc, workspace: torch.Tensor, device):
        self.desc, self.workspace, self.device = desc, workspace, device
        self._apply_ws = None

    @property
    def m(self):
        return self.desc.m

    @property
    def n(self):
        return self.desc.n

    def status(self, stream=None) -> int:
        """Synchronise and return the device-side status (0 = success)."""
        return load().tileqr_status(ctypes.byref(self.desc), _stream_ptr(stream))

    def check(self, stream=None):
        _check(self.status(stream), "tileqr factorization")
        return self

    def R(self, stream=None) -> torch.Tensor:
        k = min(self.m, self.n)
        R = colmajor_empty(k, self.n, self.device)
        _check(load().tileqr_get_R(ctypes.byref(self.desc), ctypes.c_void_p(R.data_ptr()), max(k, 1),
                                   _stream_ptr(stream)), "tileqr_get_R")
        return R

    def factors(self, stream=None):
        """(AV, T): LAPACK-style in-place factors and the (p*ib) x n T strips."""
        d = self.desc
        AV = colmajor_empty(d.m, d.n, self.device)
        T = colmajor_empty(d.p * d.ib, d.n, self.device)
        _check(load().tileqr_get_factors(ctypes.byref(d), ctypes.c_void_p(AV.data_ptr()), max(d.m, 1),
                                         ctypes.c_void_p(T.data_ptr()), max(d.p * d.ib, 1),
                                         _stream_ptr(stream)), "tileqr_get_factors")
        return AV, T

    def tree_T(self, stream=None) -> torch.Tensor:
        """The DTTQRT T strips of a tree-form factorization, (p*ib) x n."""
        d = self.desc
        T2 = colmajor_empty(d.p * d.ib, d.n, self.device)
        _check(load().tileqr_get_tree_T(ctypes.byref(d), ctypes.c_void_p(T2.data_ptr()), max(d.p * d.ib, 1),
                                        _stream_ptr(stream)), "tileqr_get_tree_T")
        return T2

    def _apply_workspace(self, nrhs: int) -> torch.Tensor:
        out = ctypes.c_size_t(0)
        _check(load().tileqr_apply_workspace_size(ctypes.byref(self.desc), nrhs, ctypes.byref(out)),
               "tileqr_apply_workspace_size")
        if self._apply_ws is None or self._apply_ws.numel() < out.value:
            self._apply_ws = torch.empty(max(out.value, 256), dtype=torch.uint8, device=self.device)
        return self._apply_ws

    def apply_qt(self, B: torch.Tensor, stream=None) -> torch.Tensor:
        """Q^T B in place (B column-major m x nrhs); returns B."""
        B = as_colmajor(B)
        ws = self._apply_workspace(B.shape[1])
        _check(load().tileqr_apply_qt(ctypes.byref(self.desc), ctypes.c_void_p(B.data_ptr()), _ld(B),
                                      B.shape[1], ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                      _stream_ptr(stream)), "tileqr_apply_qt")
        return B

    def apply_q(self, B: torch.Tensor, stream=None) -> torch.Tensor:
        """Q B in place (Q itself); returns B."""
        B = as_colmajor(B)
        ws = self._apply_workspace(B.shape[1])
        _check(load().tileqr_apply_q(ctypes.byref(self.desc), ctypes.c_void_p(B.data_ptr()), _ld(B), B.shape[1],
                                     ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)),
               "tileqr_apply_q")
        return B

    def apply_mixed(self, B: torch.Tensor, trans: bool = True, stream=None) -> torch.Tensor:
        """Q^T B (trans) or Q B on the tensor cores, in place, for a
        TILEQR_TF32 factorization with nb 128 (3xTF32: about 2^-19 relative
        per column, not FP64); synchronous; returns B."""
        B = as_colmajor(B)
        out = ctypes.c_size_t(0)
        _check(load().tileqr_apply_mixed_workspace_size(ctypes.byref(self.desc), B.shape[1], ctypes.byref(out)),
               "tileqr_apply_mixed_workspace_size")
        ws = torch.empty(max(out.value, 256), dtype=torch.uint8, device=self.device)
        _check(load().tileqr_apply_mixed(ctypes.byref(self.desc), 1 if trans else 0, ctypes.c_void_p(B.data_ptr()),
                                         _ld(B), B.shape[1], ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                         _stream_ptr(stream)), "tileqr_apply_mixed")
        return B

    def form_q(self, ncols: int | None = None, stream=None) -> torch.Tensor:
        """The leading ncols (default min(m, n)) columns of Q, m x ncols."""
        k = min(self.m, self.n) if ncols is None else ncols
        Q = colmajor_empty(self.m, k, self.device)
        ws = self._apply_workspace(k)
        _check(load().tileqr_form_q(ctypes.byref(self.desc), ctypes.c_void_p(Q.data_ptr()), max(self.m, 1), k,
                                    ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)),
               "tileqr_form_q")
        return Q

    def solve_refine(self, A: torch.Tensor, b: torch.Tensor, max_iter: int = 30, tol: float = 1e-12,
                     stream=None):
        """x with ||b - A x|| / ||b|| <= tol by FP64 iterative refinement on
        this factorization of A (see tileqr_solve_refine); returns (x, info)."""
        A = as_colmajor(A)
        b = b.reshape(-1).contiguous()
        need = ctypes.c_size_t(0)
        _check(load().tileqr_refine_workspace_size(ctypes.byref(self.desc), ctypes.byref(need)),
               "tileqr_refine_workspace_size")
        ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device=self.device)
        x = torch.empty(self.n, dtype=torch.float64, device=self.device)
        info = tileqr_refine_info()
        _check(load().tileqr_solve_refine(ctypes.byref(self.desc), ctypes.c_void_p(A.data_ptr()), _ld(A),
                                          ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), max_iter,
                                          tol, ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream),
                                          ctypes.byref(info)), "tileqr_solve_refine")
        return x, info

    def solve_ls_refine(self, A: torch.Tensor, B: torch.Tensor, max_iter: int = 10, tol: float = 1e-14,
                        residual: bool = False, stream=None):
        """min ||A X - B|| refined in FP64 on the augmented system (see
        tileqr_solve_ls_refine); B is not modified.  Returns (X, info), or
        (X, R, info) with the residuals B - A X if residual is True."""
        A = as_colmajor(A)
        B = as_colmajor(B)
        nrhs = B.shape[1]
        need = ctypes.c_size_t(0)
        _check(load().tileqr_ls_refine_workspace_size(ctypes.byref(self.desc), nrhs, ctypes.byref(need)),
               "tileqr_ls_refine_workspace_size")
        ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device=self.device)
        X = colmajor_empty(self.n, nrhs, self.device)
        R = colmajor_empty(self.m, nrhs, self.device) if residual else None
        info = tileqr_refine_info()
        _check(load().tileqr_solve_ls_refine(ctypes.byref(self.desc), ctypes.c_void_p(A.data_ptr()), _ld(A),
                                             ctypes.c_void_p(B.data_ptr()), _ld(B), nrhs,
                                             ctypes.c_void_p(X.data_ptr()), _ld(X),
                                             ctypes.c_void_p(R.data_ptr()) if R is not None else None,
                                             _ld(R) if R is not None else 1, max_iter, tol,
                                             ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream),
                                             ctypes.byref(info)), "tileqr_solve_ls_refine")
        return (X, R, info) if residual else (X, info)

    def solve_ls(self, B: torch.Tensor, stream=None) -> torch.Tensor:
        """min ||A X - B||: B overwritten (X in its first n rows); returns X."""
        B = as_colmajor(B)
        ws = self._apply_workspace(B.shape[1])
        _check(load().tileqr_solve_ls(ctypes.byref(self.desc), ctypes.c_void_p(B.data_ptr()), _ld(B),
                                      B.shape[1], ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                      _stream_ptr(stream)), "tileqr_solve_ls")
        return B[: self.n]


def tileqr_status(f: Factorization, stream=None) -> int:
    return f.status(stream)


def tileqr_get_R(f: Factorization, stream=None) -> torch.Tensor:
    return f.R(stream)


def tileqr_get_factors(f: Factorization, stream=None):
    return f.factors(stream)


def tileqr_apply_qt(f: Factorization, B: torch.Tensor, stream=None) -> torch.Tensor:
    return f.apply_qt(B, stream)


def tileqr_solve_ls(f: Factorization, B: torch.Tensor, stream=None) -> torch.Tensor:
    return f.solve_ls(B, stream)


def tileqr_mixed_update_tile(kind: int, ib: int, V: torch.Tensor, T: torch.Tensor, B: torch.Tensor | None,
                             C: torch.Tensor, stream=None) -> None:
    """One TILEQR_TF32 update task (DLARFB or DSSRFB) on 128 x 128 column-
    major float64 CUDA tiles, B and C updated in place; T is the ib x 128 strip
    (column-major)."""
    for t in (V, T, C) + ((B,) if B is not None else ()):
        assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    ws = torch.empty(TILEQR_MIXED_UPDATE_WS_BYTES, dtype=torch.uint8, device=C.device)
    _check(load().tileqr_mixed_update_tile(kind, ib, ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                           ctypes.c_void_p(B.data_ptr()) if B is not None else None,
                                           ctypes.c_void_p(C.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                           ws.numel(), _stream_ptr(stream)), "tileqr_mixed_update_tile")


def tileqr_measure_fp64_rates(stream=None):
    """(DFMA GFLOP/s, FP64 mma.sync GFLOP/s) measured on the current GPU."""
    a, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().tileqr_measure_fp64_rates(ctypes.byref(a), ctypes.byref(b), _stream_ptr(stream)),
           "tileqr_measure_fp64_rates")
    return a.value, b.value


def tileqr_launch_count() -> int:
    return int(load().tileqr_launch_count())


def tileqr_reset_launch_count() -> None:
    load().tileqr_reset_launch_count()


def tileqr_set_profile_events(before=None, after=None) -> None:
    """Record torch.cuda.Event pair around the task-graph launches of later
    factorizations (None, None disables)."""
    # torch creates the CUDA event on its first record(): record once here so
    # the handle exists (the library re-records it around each launch)
    for e in (before, after):
        if e is not None and e.cuda_event == 0:
            e.record()
    b = ctypes.c_void_p(before.cuda_event) if before is not None else None
    a = ctypes.c_void_p(after.cuda_event) if after is not None else None
    load().tileqr_set_profile_events(b, a)


def tileqr_set_trace(records: torch.Tensor | None) -> None:
    """Trace every task of later factorizations into `records` (an int64 CUDA
    tensor of shape (capacity, 4)); None disables tracing."""
    if records is None:
        load().tileqr_set_trace(None, 0)
        return
    assert records.dtype == torch.int64 and records.is_cuda and records.dim() == 2 and records.shape[1] == 4
    load().tileqr_set_trace(ctypes.c_void_p(records.data_ptr()), records.shape[0])


def tileqr_trace_count(f: "Factorization", stream=None) -> int:
    out = ctypes.c_uint64(0)
    _check(load().tileqr_trace_count(ctypes.byref(f.desc), _stream_ptr(stream), ctypes.byref(out)),
           "tileqr_trace_count")
    return int(out.value)


class Batch:
    """A prepared batch of independent factorizations (tileqr_batched_prepare).

    `mats` are column-major float64 CUDA tensors; they must stay alive while
    the batch is used.  run() enqueues the factorization of all of them
    (graph-capturable); get(b) returns the Factorization of matrix b."""

    def __init__(self, mats, nb: int, ib: int, precision: int = TILEQR_FP64, stream=None):
        import numpy as np
        self.mats = [as_colmajor(a) for a in mats]
        count = len(self.mats)
        self._m = np.array([a.shape[0] for a in self.mats], dtype=np.int64)
        self._n = np.array([a.shape[1] for a in self.mats], dtype=np.int64)
        self._lda = np.array([_ld(a) for a in self.mats], dtype=np.int64)
        self._ptrs = (ctypes.c_void_p * max(count, 1))(*[a.data_ptr() for a in self.mats])
        need = ctypes.c_size_t(0)
        mp = self._m.ctypes.data_as(ctypes.c_void_p)
        np_ = self._n.ctypes.data_as(ctypes.c_void_p)
        _check(load().tileqr_batched_workspace_size(count, mp, np_, nb, ib, precision, ctypes.byref(need)),
               "tileqr_batched_workspace_size")
        dev = self.mats[0].device if count else torch.device("cuda")
        self.workspace = torch.empty(max(need.value, 256), dtype=torch.uint8, device=dev)
        self.device = dev
        self.bt = tileqr_batch()
        _check(load().tileqr_batched_prepare(count, mp, np_, self._ptrs, self._lda.ctypes.data_as(ctypes.c_void_p),
                                             nb, ib, precision, ctypes.c_void_p(self.workspace.data_ptr()),
                                             self.workspace.numel(), _stream_ptr(stream), ctypes.byref(self.bt)),
               "tileqr_batched_prepare")

    @property
    def flops(self) -> float:
        return self.bt.flops

    def run(self, stream=None) -> None:
        _check(load().tileqr_factor_batched(ctypes.byref(self.bt), _stream_ptr(stream)), "tileqr_factor_batched")

    def status(self, stream=None) -> int:
        return load().tileqr_batched_status(ctypes.byref(self.bt), _stream_ptr(stream))

    def get(self, b: int) -> "Factorization":
        d = tileqr_desc()
        _check(load().tileqr_batched_get(ctypes.byref(self.bt), b, ctypes.byref(d)), "tileqr_batched_get")
        return Factorization(d, self.workspace, self.device)

    def solve_ls(self, bs, max_iter: int = 8, tol: float = 1e-14, stream=None):
        """Least squares per matrix (one right-hand side each, bs[b] of m_b
        entries) refined in FP64 on the augmented system, all matrices in one
        launch (tileqr_batched_solve_ls); max_iter = 1 is the plain solve.
        Returns ([x_b], summary info)."""
        count = len(self.mats)
        bs = [b.reshape(-1).contiguous() for b in bs]
        xs = [torch.empty(int(n), dtype=torch.float64, device=self.device) for n in self._n]
        need = ctypes.c_size_t(0)
        _check(load().tileqr_batched_ls_workspace_size(ctypes.byref(self.bt), ctypes.byref(need)),
               "tileqr_batched_ls_workspace_size")
        ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device=self.device)
        bp = (ctypes.c_void_p * max(count, 1))(*[b.data_ptr() for b in bs])
        xp = (ctypes.c_void_p * max(count, 1))(*[x.data_ptr() for x in xs])
        info = tileqr_refine_info()
        _check(load().tileqr_batched_solve_ls(ctypes.byref(self.bt), bp, xp, max_iter, tol,
                                              ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream),
                                              ctypes.byref(info)), "tileqr_batched_solve_ls")
        return xs, info
