"""CPU oracle for the tiled Householder QR -- TEST INFRASTRUCTURE ONLY.

Plain, slow FP64 implementation of Algorithm 2 of Buttari, Langou, Kurzak and
Dongarra (the four tile kernels of Sec. 3.2.1 with the inner blocking of
Sec. 3.2.3), an independent unblocked Householder QR, Q^T application and the
least-squares solve, all in ``tileqr_oracle.c`` and called here through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and the CUDA library never calls it.

Every pinned function is checked in ``tests/test_oracle_*.py`` against
closed forms, LAPACK's own tile kernels (dgeqrt, dgemqrt, dtpqrt, dtpmqrt),
invariants, and brute force; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tileqr_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "cholesky_oracle.c"), os.path.join(_HERE, "lu_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")

TASK_GEQRT, TASK_TSQRT, TASK_LARFB, TASK_SSRFB = 0, 1, 2, 3


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")


def _compile(lib: str, extra, force: bool) -> str:
    if (not force and os.path.exists(lib)
            and os.path.getmtime(lib) >= max(os.path.getmtime(x) for x in _SRCS)):
        return lib
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC"] + extra + \
        ["-shared", "-o", tmp] + _SRCS + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no FMA contraction, no -march):
    the single-threaded library the tests use, and the same sources built
    with OpenMP (liboracle_omp.so), whose only parallel code is the level-by-
    level driver of tiled_qr_levels (the CPU baseline)."""
    _compile(_LIB_OMP, ["-fopenmp"], force)
    return _compile(_LIB, [], force)


_lib = None
_lib_omp = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        lib.oracle_tiled_qr.argtypes = [i64, i64, dp, i64, i32, i32, dp, i64]
        lib.oracle_tiled_qr_ordered.argtypes = [i64, i64, dp, i64, i32, i32, dp, i64, i64,
                                                ctypes.POINTER(ctypes.c_int32)]
        lib.oracle_apply_qt.argtypes = [i64, i64, dp, i64, i32, i32, dp, i64, i64, dp, i64]
        lib.oracle_solve_ls.argtypes = [i64, i64, dp, i64, i32, i32, dp, i64, i64, dp, i64]
        lib.oracle_unblocked_qr.argtypes = [i64, i64, dp, i64]
        lib.oracle_tiled_qr_tree.argtypes = [i64, i64, dp, i64, i32, i32, i32, dp, i64, dp, i64]
        lib.oracle_tiled_qr_tree_ordered.argtypes = [i64, i64, dp, i64, i32, i32, i32, dp, i64, dp, i64,
                                                     i64, ctypes.POINTER(ctypes.c_int32)]
        lib.oracle_apply_qt_tree.argtypes = [i64, i64, dp, i64, i32, i32, i32, dp, i64, dp, i64, i64, dp,
                                             i64]
        lib.oracle_apply_q_tree.argtypes = [i64, i64, dp, i64, i32, i32, i32, dp, i64, dp, i64, i64, dp, i64]
        lib.oracle_tiled_cholesky.argtypes = [i64, dp, i64, i32]
        lib.oracle_tiled_cholesky_ordered.argtypes = [i64, dp, i64, i32, i64, ctypes.POINTER(ctypes.c_int32)]
        lib.oracle_tiled_cholesky.restype = ctypes.c_int
        lib.oracle_tiled_cholesky_ordered.restype = ctypes.c_int
        lib.chol_set_mutation.argtypes = [i32]
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_tiled_lu.argtypes = [i64, dp, i64, i32, i32, dp, i64, ip]
        lib.oracle_tiled_lu_ordered.argtypes = [i64, dp, i64, i32, i32, dp, i64, ip, i64,
                                                ctypes.POINTER(ctypes.c_int32)]
        lib.oracle_lu_apply.argtypes = [i64, dp, i64, i32, i32, dp, i64, ip, i64, dp, i64, i32]
        lib.oracle_lu_unapply.argtypes = [i64, dp, i64, i32, i32, dp, i64, ip, i64, dp, i64]
        for f in (lib.oracle_tiled_lu, lib.oracle_tiled_lu_ordered, lib.oracle_lu_apply, lib.oracle_lu_unapply):
            f.restype = ctypes.c_int
        lib.lu_set_mutation.argtypes = [i32]
        lib.lu_flops.restype = ctypes.c_double
        lib.chol_flops.restype = ctypes.c_double
        lib.oracle_flops.restype = ctypes.c_double
        lib.oracle_set_mutation.argtypes = [i32]
        for f in (lib.oracle_tiled_qr, lib.oracle_tiled_qr_ordered, lib.oracle_apply_qt,
                  lib.oracle_solve_ls, lib.oracle_unblocked_qr, lib.oracle_tiled_qr_tree,
                  lib.oracle_tiled_qr_tree_ordered, lib.oracle_apply_qt_tree, lib.oracle_apply_q_tree):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fortran(a) -> np.ndarray:
    return np.array(a, dtype=np.float64, order="F", copy=True)


def geometry(m: int, n: int, nb: int):
    """Tile grid p x q and the partial-tile extents (Sec. 3.2.1 with ragged edges)."""
    p, q = -(-m // nb), -(-n // nb)
    mr = [min(nb, m - i * nb) for i in range(p)]
    nc = [min(nb, n - j * nb) for j in range(q)]
    return p, q, mr, nc


class Factored:
    """Result of the tiled factorization: A overwritten by R and V, plus T.

    ``A`` is m x n column-major; ``T`` is (p*ib) x n column-major, the strip of
    tile (i, k) being rows i*ib..i*ib+ib-1 and columns k*nb..k*nb+nc(k)-1.
    """

    def __init__(self, A, T, m, n, nb, ib, T2=None, h=0):
        self.A, self.T, self.m, self.n, self.nb, self.ib = A, T, m, n, nb, ib
        self.T2, self.h = T2, h   # tree variant: DTTQRT T strips and domain size

    def R(self) -> np.ndarray:
        """The min(m,n) x n upper-trapezoidal R factor."""
        k = min(self.m, self.n)
        return np.triu(self.A[:k, :])

    def tile(self, i, j):
        nb = self.nb
        return self.A[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb]

    def tstrip(self, i, k):
        nb, ib = self.nb, self.ib
        return self.T[i * ib:(i + 1) * ib, k * nb:(k + 1) * nb]

    def tstrip2(self, i, k):
        nb, ib = self.nb, self.ib
        return self.T2[i * ib:(i + 1) * ib, k * nb:(k + 1) * nb]


def tiled_qr(A, nb: int, ib: int) -> Factored:
    """Algorithm 2 on a copy of A, tasks in the printed loop order."""
    lib = _load()
    A = _fortran(A)
    m, n = A.shape
    p = -(-m // nb) if m else 0
    T = np.zeros((max(p * ib, 1), max(n, 1)), dtype=np.float64, order="F")
    rc = lib.oracle_tiled_qr(m, n, _dp(A), max(m, 1), nb, ib, _dp(T), T.shape[0])
    if rc:
        raise ValueError(f"oracle_tiled_qr: illegal argument {rc}")
    return Factored(A, T, m, n, nb, ib)


def tiled_qr_levels(A, nb: int, ib: int, threads: int = 1):
    """Algorithm 2 run level by level of its task graph, the tasks of a level
    spread over `threads` OpenMP threads (the same tile kernels; identical
    bits to tiled_qr).  Returns (Factored, number of levels)."""
    global _lib_omp
    if _lib_omp is None:
        build()
        lib = ctypes.CDLL(_LIB_OMP)
        lib.oracle_tiled_qr_levels.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                               ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)]
        lib.oracle_tiled_qr_levels.restype = ctypes.c_int
        _lib_omp = lib
    A = _fortran(A)
    m, n = A.shape
    p = -(-m // nb) if m else 0
    T = np.zeros((max(p * ib, 1), max(n, 1)), dtype=np.float64, order="F")
    nlev = ctypes.c_int(0)
    rc = _lib_omp.oracle_tiled_qr_levels(m, n, _dp(A), max(m, 1), nb, ib, _dp(T), T.shape[0], int(threads),
                                         ctypes.byref(nlev))
    if rc:
        raise ValueError(f"oracle_tiled_qr_levels: error {rc}")
    return Factored(A, T, m, n, nb, ib), nlev.value


def tiled_qr_ordered(A, nb: int, ib: int, tasks) -> Factored:
    """Algorithm 2 with its tasks run in the given order (rows {kind,i,j,k})."""
    lib = _load()
    A = _fortran(A)
    m, n = A.shape
    p = -(-m // nb)
    T = np.zeros((max(p * ib, 1), max(n, 1)), dtype=np.float64, order="F")
    tk = np.ascontiguousarray(np.asarray(tasks, dtype=np.int32).reshape(-1, 4))
    rc = lib.oracle_tiled_qr_ordered(m, n, _dp(A), max(m, 1), nb, ib, _dp(T), T.shape[0],
                                     tk.shape[0],
                                     tk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc:
        raise ValueError(f"oracle_tiled_qr_ordered: illegal argument {rc}")
    return Factored(A, T, m, n, nb, ib)


def _tree_arrays(m, n, nb, ib):
    p = -(-m // nb) if m else 0
    T = np.zeros((max(p * ib, 1), max(n, 1)), dtype=np.float64, order="F")
    return T, np.zeros_like(T, order="F")


def tiled_qr_tree(A, nb: int, ib: int, h: int) -> Factored:
    """The tree variant on a copy of A: domains of h tile rows per step,
    heads merged pairwise by DTTQRT (h <= 0 or h >= p: Algorithm 2)."""
    lib = _load()
    A = _fortran(A)
    m, n = A.shape
    T, T2 = _tree_arrays(m, n, nb, ib)
    rc = lib.oracle_tiled_qr_tree(m, n, _dp(A), max(m, 1), nb, ib, int(h), _dp(T), T.shape[0], _dp(T2),
                                  T2.shape[0])
    if rc:
        raise ValueError(f"oracle_tiled_qr_tree: illegal argument {rc}")
    return Factored(A, T, m, n, nb, ib, T2, h)


def tiled_qr_tree_ordered(A, nb: int, ib: int, h: int, tasks) -> Factored:
    """The tree variant with its tasks run in the given order (rows {kind,i,j,k})."""
    lib = _load()
    A = _fortran(A)
    m, n = A.shape
    T, T2 = _tree_arrays(m, n, nb, ib)
    tk = np.ascontiguousarray(np.asarray(tasks, dtype=np.int32).reshape(-1, 4))
    rc = lib.oracle_tiled_qr_tree_ordered(m, n, _dp(A), max(m, 1), nb, ib, int(h), _dp(T), T.shape[0],
                                          _dp(T2), T2.shape[0], tk.shape[0],
                                          tk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if rc:
        raise ValueError(f"oracle_tiled_qr_tree_ordered: illegal argument {rc}")
    return Factored(A, T, m, n, nb, ib, T2, h)


def apply_qt(f: Factored, B) -> np.ndarray:
    """Q^T B for the Q held (as V and T) in a Factored result."""
    lib = _load()
    B = _fortran(B)
    if B.ndim == 1:
        B = B.reshape(-1, 1, order="F")
    if f.T2 is not None:
        rc = lib.oracle_apply_qt_tree(f.m, f.n, _dp(f.A), max(f.m, 1), f.nb, f.ib, int(f.h), _dp(f.T),
                                      f.T.shape[0], _dp(f.T2), f.T2.shape[0], B.shape[1], _dp(B),
                                      max(f.m, 1))
        if rc:
            raise ValueError(f"oracle_apply_qt_tree: illegal argument {rc}")
        return B
    rc = lib.oracle_apply_qt(f.m, f.n, _dp(f.A), max(f.m, 1), f.nb, f.ib, _dp(f.T),
                             f.T.shape[0], B.shape[1], _dp(B), max(f.m, 1))
    if rc:
        raise ValueError(f"oracle_apply_qt: illegal argument {rc}")
    return B


def apply_q(f: Factored, B) -> np.ndarray:
    """Q B (Q itself, not Q^T) for the Q held in a Factored result: the
    update transformations replayed in reverse order, each with its inner
    blocks reversed and T_l instead of T_l^T."""
    lib = _load()
    B = _fortran(B)
    if B.ndim == 1:
        B = B.reshape(-1, 1, order="F")
    T2 = f.T2 if f.T2 is not None else np.zeros((1, 1), order="F")
    rc = lib.oracle_apply_q_tree(f.m, f.n, _dp(f.A), max(f.m, 1), f.nb, f.ib, int(f.h), _dp(f.T), f.T.shape[0],
                                 _dp(T2), T2.shape[0], B.shape[1], _dp(B), max(f.m, 1))
    if rc:
        raise ValueError(f"oracle_apply_q_tree: illegal argument {rc}")
    return B


def form_q(f: Factored, ncols: int | None = None) -> np.ndarray:
    """The first ncols (default min(m, n)) columns of Q, m x ncols: Q applied
    to the leading columns of the identity."""
    k = min(f.m, f.n) if ncols is None else ncols
    E = np.zeros((f.m, k), order="F")
    E[np.arange(min(f.m, k)), np.arange(min(f.m, k))] = 1.0
    return apply_q(f, E)


def solve_ls(f: Factored, B) -> np.ndarray:
    """argmin_X ||A X - B||_F for m >= n: Q^T B then back substitution with R."""
    if f.T2 is not None:
        # tree variant: Q^T B, then the triangular solve (library routine)
        import scipy.linalg
        if f.m < f.n:
            raise ValueError("solve_ls needs m >= n")
        Y = apply_qt(f, B)
        R = f.A[:f.n, :f.n]
        d = np.diag(R)
        if np.any(d == 0.0):
            raise np.linalg.LinAlgError(f"R({int(np.argmax(d == 0.0))},...) is exactly zero")
        return scipy.linalg.solve_triangular(np.triu(R), Y[:f.n, :], lower=False)
    lib = _load()
    B = _fortran(B)
    if B.ndim == 1:
        B = B.reshape(-1, 1, order="F")
    rc = lib.oracle_solve_ls(f.m, f.n, _dp(f.A), max(f.m, 1), f.nb, f.ib, _dp(f.T),
                             f.T.shape[0], B.shape[1], _dp(B), max(f.m, 1))
    if rc < 0:
        raise ValueError(f"oracle_solve_ls: illegal argument {rc}")
    if rc > 0:
        raise np.linalg.LinAlgError(f"R({rc - 1},{rc - 1}) is exactly zero")
    return B[:f.n, :].copy(order="F")


def refine_ls_augmented(f: Factored, A, b, max_iter: int = 20, tol: float = 1e-14):
    """Least squares min ||A x - b|| for m >= n, refined in FP64 on top of a
    (possibly inexact) factorization f of A: Bjorck's iterative refinement of
    the augmented system [I A; A^T 0] [r; x] = [b; 0] (A. Bjorck, "Iterative
    refinement of linear least squares solutions I", BIT 7, 1967).  Not part
    of the paper; the oracle of the refinement for inconsistent systems.

    Each step forms the augmented residuals in FP64, u = b - r - A x and
    w = -A^T r, and solves the augmented system for the correction with the
    factors (A ~ Q [R; 0]): h = R^{-T} w, [d1; d2] = Q^T u,
    dx = R^{-1} (d1 - h), dr = Q [h; d2].  Refining x alone (x += R^{-1}
    (Q^T (b - A x))(0:n)) stalls at an error proportional to the factors'
    error times the residual; the augmented form converges to the FP64
    solution.  Stops when ||dx|| <= tol ||x|| or when ||dx|| no longer halves.
    Returns (x, r, steps)."""
    import scipy.linalg
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    m, n = A.shape
    if m < n:
        raise ValueError("refine_ls_augmented needs m >= n")
    R = np.triu(f.R()[:n, :n])
    x = solve_ls(f, b.copy()).reshape(-1)
    r = b - A @ x
    steps = 0
    prev = np.inf
    for steps in range(1, max_iter + 1):
        u = b - r - A @ x
        w = -(A.T @ r)
        h = scipy.linalg.solve_triangular(R, w, trans="T", lower=False)
        d = apply_qt(f, u.copy()).reshape(-1)
        dx = scipy.linalg.solve_triangular(R, d[:n] - h, lower=False)
        z = np.concatenate([h, d[n:]])
        dr = apply_q(f, z.copy()).reshape(-1)
        x = x + dx
        r = r + dr
        # stop once the correction is negligible, or no longer halves (it
        # has reached the rounding level of the FP64 residuals)
        ndx = np.linalg.norm(dx)
        if ndx <= tol * np.linalg.norm(x) or ndx > 0.5 * prev:
            break
        prev = ndx
    return x, r, steps


def unblocked_qr(A) -> np.ndarray:
    """R of the textbook unblocked Householder QR (independent of the tiled code)."""
    lib = _load()
    A = _fortran(A)
    m, n = A.shape
    rc = lib.oracle_unblocked_qr(m, n, _dp(A), max(m, 1))
    if rc:
        raise ValueError("oracle_unblocked_qr: illegal argument")
    return np.triu(A[:min(m, n), :])


def flops() -> float:
    return _load().oracle_flops()


def reset_flops() -> None:
    _load().oracle_reset_flops()


def set_mutation(code: int) -> None:
    """Plant a deliberate mistake in the oracle's arithmetic (tests only)."""
    _load().oracle_set_mutation(int(code))


# ---------------------------------------------------------------------------
# Task graph of Algorithm 2 (Sec. 4).
def task_list(m: int, n: int, nb: int):
    """Tasks {kind, i, j, k} in the printed loop order of Algorithm 2."""
    p, q, _, _ = geometry(m, n, nb)
    out = []
    for k in range(min(p, q)):
        out.append((TASK_GEQRT, k, k, k))
        for j in range(k + 1, q):
            out.append((TASK_LARFB, k, j, k))
        for i in range(k + 1, p):
            out.append((TASK_TSQRT, i, k, k))
            for j in range(k + 1, q):
                out.append((TASK_SSRFB, i, j, k))
    return out


TASK_TTQRT, TASK_TTSSRFB = 4, 5


def _domain(p: int, h: int) -> int:
    return p if (h <= 0 or h > p) else h


def tt_partner(k: int, H: int, e: int) -> int:
    """Head row that domain head e is merged into at step k (level ctz(d))."""
    d = (e - k) // H
    lev = (d & -d).bit_length() - 1
    return k + (d - (1 << lev)) * H


def task_list_tree(m: int, n: int, nb: int, h: int):
    """Tasks {kind, i, j, k} of the tree variant in the oracle's sequential
    order (oracle_tiled_qr_tree); h <= 0 or h >= p gives task_list."""
    p, q, _, _ = geometry(m, n, nb)
    H = _domain(p, h)
    out = []
    for k in range(min(p, q)):
        ndom = -(-(p - k) // H)
        for d in range(ndom):
            hd = k + d * H
            last = min(hd + H, p) - 1
            out.append((TASK_GEQRT, hd, k, k))
            for j in range(k + 1, q):
                out.append((TASK_LARFB, hd, j, k))
            for i in range(hd + 1, last + 1):
                out.append((TASK_TSQRT, i, k, k))
                for j in range(k + 1, q):
                    out.append((TASK_SSRFB, i, j, k))
        lev = 0
        while (1 << lev) < ndom:
            for d in range(0, ndom - (1 << lev), 2 << lev):
                e = k + (d + (1 << lev)) * H
                out.append((TASK_TTQRT, e, k, k))
                for j in range(k + 1, q):
                    out.append((TASK_TTSSRFB, e, j, k))
            lev += 1
    return out


def task_access_tree(kind: int, i: int, j: int, k: int, H: int):
    """(reads, writes) of a task of the tree variant.  A head tile's upper
    triangle ('R', r, k) holds its R (then the DTTQRT reflectors), its strict
    lower part ('V', r, k) the DGEQRT reflectors; ('T2', r, k) is the DTTQRT
    T strip."""
    if kind == TASK_GEQRT:
        return {("A", i, k)}, {("R", i, k), ("V", i, k), ("T", i, k)}
    if kind == TASK_LARFB:
        return {("V", i, k), ("T", i, k)}, {("A", i, j)}
    if kind == TASK_TSQRT:
        return set(), {("R", k + ((i - k) // H) * H, k), ("A", i, k), ("T", i, k)}
    if kind == TASK_SSRFB:
        return {("A", i, k), ("T", i, k)}, {("A", k + ((i - k) // H) * H, j), ("A", i, j)}
    if kind == TASK_TTQRT:
        return set(), {("R", tt_partner(k, H, i), k), ("R", i, k), ("T2", i, k)}
    return {("R", i, k), ("T2", i, k)}, {("A", tt_partner(k, H, i), j), ("A", i, j)}


def _mechanical_deps(tasks, access):
    last_w, readers = {}, {}
    preds = {}
    for t in tasks:
        r, w = access(t)
        ps = set()
        for d in r | w:
            if d in last_w:
                ps.add(last_w[d])
        for d in w:
            ps |= readers.get(d, set())
        preds[t] = ps - {t}
        for d in r:
            readers.setdefault(d, set()).add(t)
        for d in w:
            last_w[d] = t
            readers[d] = set()
    return preds


def dependencies_tree(m: int, n: int, nb: int, h: int):
    """Predecessor sets of the tree variant, derived from the reads and
    writes of its sequential order exactly as dependencies() does."""
    p, _, _, _ = geometry(m, n, nb)
    H = _domain(p, h)
    tasks = task_list_tree(m, n, nb, h)
    return tasks, _mechanical_deps(tasks, lambda t: task_access_tree(*t, H))


def apply_task_list_tree(m: int, n: int, nb: int, h: int):
    """Q^T applied to one block column of right-hand sides: the update tasks
    of the tree variant replayed on the row blocks of B, as {kind, i, k}
    (kind TASK_LARFB / TASK_SSRFB / TASK_TTSSRFB) in sequential order."""
    p, q, _, _ = geometry(m, n, nb)
    H = _domain(p, h)
    out = []
    for k in range(min(p, q)):
        ndom = -(-(p - k) // H)
        for d in range(ndom):
            hd = k + d * H
            last = min(hd + H, p) - 1
            out.append((TASK_LARFB, hd, k))
            for i in range(hd + 1, last + 1):
                out.append((TASK_SSRFB, i, k))
        lev = 0
        while (1 << lev) < ndom:
            for d in range(0, ndom - (1 << lev), 2 << lev):
                out.append((TASK_TTSSRFB, k + (d + (1 << lev)) * H, k))
            lev += 1
    return out


def apply_dependencies_tree(m: int, n: int, nb: int, h: int, reverse: bool = False):
    """Predecessor sets of the Q^T application on one block column (reverse:
    of the Q application, which runs the same tasks in reverse order), from
    the row blocks of B each task reads and writes."""
    p, _, _, _ = geometry(m, n, nb)
    H = _domain(p, h)
    tasks = apply_task_list_tree(m, n, nb, h)
    if reverse:
        tasks = tasks[::-1]

    def access(t):
        kind, i, k = t
        if kind == TASK_LARFB:
            return set(), {("B", i)}
        if kind == TASK_SSRFB:
            return set(), {("B", k + ((i - k) // H) * H), ("B", i)}
        return set(), {("B", tt_partner(k, H, i)), ("B", i)}

    return tasks, _mechanical_deps(tasks, access)


def task_access(kind: int, i: int, j: int, k: int):
    """(reads, writes) of one task as sets of data items, from the kernel
    definitions of Sec. 3.2.1.  The diagonal tile is split into its R part
    ('R', k, k) (upper triangle) and its V part ('V', k, k) (strict lower);
    ('T', i, k) is the T strip."""
    if kind == TASK_GEQRT:
        # consumes the whole diagonal tile as last written by the previous step
        return {("A", k, k)}, {("R", k, k), ("V", k, k), ("T", k, k)}
    if kind == TASK_LARFB:
        return {("V", k, k), ("T", k, k)}, {("A", k, j)}
    if kind == TASK_TSQRT:
        return set(), {("R", k, k), ("A", i, k), ("T", i, k)}
    return {("A", i, k), ("T", i, k)}, {("A", k, j), ("A", i, j)}


def dependencies(m: int, n: int, nb: int):
    """Predecessor sets derived mechanically from the reads/writes of the
    sequential order: a task depends on the last writer of everything it
    touches, and a writer also waits for the readers since that write."""
    tasks = task_list(m, n, nb)
    last_w, readers = {}, {}
    preds = {}
    for t in tasks:
        r, w = task_access(*t)
        # the read-modify-write of tiles: a written tile is also read unless the
        # task creates it outright (GEQRT/TSQRT start from the prior contents)
        touched = r | w
        ps = set()
        for d in touched:
            if d in last_w:
                ps.add(last_w[d])
        for d in w:
            ps |= readers.get(d, set())
        preds[t] = ps - {t}
        for d in r:
            readers.setdefault(d, set()).add(t)
        for d in w:
            last_w[d] = t
            readers[d] = set()
    return tasks, preds


def random_topological_order(m: int, n: int, nb: int, rng: np.random.Generator, h: int = 0):
    tasks, preds = dependencies_tree(m, n, nb, h) if h > 0 else dependencies(m, n, nb)
    succ = {t: [] for t in tasks}
    indeg = {t: len(preds[t]) for t in tasks}
    for t, ps in preds.items():
        for s in ps:
            succ[s].append(t)
    ready = [t for t in tasks if indeg[t] == 0]
    order = []
    while ready:
        t = ready.pop(int(rng.integers(len(ready))))
        order.append(t)
        for s in succ[t]:
            indeg[s] -= 1
            if indeg[s] == 0:
                ready.append(s)
    assert len(order) == len(tasks)
    return order


# ---------------------------------------------------------------------------
# Checks used by the tests.
def sign_normalize(R: np.ndarray) -> np.ndarray:
    """D R with D = diag(sign(R_jj)), sign(0) = +1."""
    k = min(R.shape)
    d = np.where(np.diag(R[:k, :k]) < 0, -1.0, 1.0)
    out = R.copy()
    out[:k, :] *= d[:, None]
    return out


def explicit_qt(f: Factored) -> np.ndarray:
    """The m x m matrix Q^T, by applying Q^T to the identity."""
    return apply_qt(f, np.eye(f.m))


def invariants(A0: np.ndarray, f: Factored):
    """(||Q^T Q - I||_F, ||A - QR||_F / ||A||_F, max |strict lower of R|)."""
    Qt = explicit_qt(f)
    Q = Qt.T
    m, n = A0.shape
    k = min(m, n)
    R = f.R()
    orth = np.linalg.norm(Q.T @ Q - np.eye(m))
    back = np.linalg.norm(A0 - Q[:, :k] @ R) / max(np.linalg.norm(A0), 1e-300)
    return orth, back, float(np.max(np.abs(np.tril(R, -1)))) if R.size else 0.0


def lapack_opcount(m: int, n: int) -> float:
    """LAPACK's Householder QR operation count 2 n^2 (m - n/3) (Sec. 5)."""
    return 2.0 * n * n * (m - n / 3.0)


def tiled_flop_model(m: int, n: int, nb: int, ib: int) -> float:
    """Sec. 3.2.3: 2 n^2 (m - n/3) (1 + s/(4b)) for the DSSRFB-dominated cost."""
    return lapack_opcount(m, n) * (1.0 + ib / (4.0 * nb))


# ---------------------------------------------------------------------------
# Tiled Cholesky (Sec. 3.1, Algorithm 1): DPOTF2, DTRSM, DGSMM.
TASK_POTF2, TASK_TRSM, TASK_GSMM = 0, 1, 2


def tiled_cholesky(A, nb: int):
    """(L, info): Algorithm 1 on a copy of the SPD matrix A; L is the lower
    Cholesky factor (strict upper part zero).  info = 0, or the 1-based
    global column of the first non-positive pivot (L then partial)."""
    lib = _load()
    A = _fortran(A)
    n = A.shape[0]
    info = lib.oracle_tiled_cholesky(n, _dp(A), max(n, 1), nb)
    if info < 0:
        raise ValueError(f"oracle_tiled_cholesky: illegal argument {info}")
    return np.tril(A), info


def tiled_cholesky_ordered(A, nb: int, tasks):
    lib = _load()
    A = _fortran(A)
    n = A.shape[0]
    tk = np.ascontiguousarray(np.asarray(tasks, dtype=np.int32).reshape(-1, 4))
    info = lib.oracle_tiled_cholesky_ordered(n, _dp(A), max(n, 1), nb, tk.shape[0],
                                             tk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if info < 0:
        raise ValueError(f"oracle_tiled_cholesky_ordered: illegal argument {info}")
    return np.tril(A), info


def cholesky_flops() -> float:
    return _load().chol_flops()


def cholesky_reset_flops() -> None:
    _load().chol_reset_flops()


def cholesky_set_mutation(code: int) -> None:
    _load().chol_set_mutation(int(code))


def cholesky_task_list(n: int, nb: int):
    """Tasks {kind, i, j, k} of Algorithm 1 in its printed loop order."""
    p = -(-n // nb)
    out = []
    for k in range(p):
        out.append((TASK_POTF2, k, k, k))
        for i in range(k + 1, p):
            out.append((TASK_TRSM, i, k, k))
        for i in range(k + 1, p):
            for j in range(k + 1, i + 1):
                out.append((TASK_GSMM, i, j, k))
    return out


def cholesky_dependencies(n: int, nb: int):
    """Predecessor sets of Algorithm 1 from the tiles each kernel reads and
    writes (Sec. 3.1): DPOTF2 rewrites A_kk, DTRSM reads L_kk and rewrites
    A_ik, DGSMM reads L_ik and L_jk and rewrites A_ij."""

    def access(t):
        kind, i, j, k = t
        if kind == TASK_POTF2:
            return set(), {("A", k, k)}
        if kind == TASK_TRSM:
            return {("A", k, k)}, {("A", i, k)}
        return {("A", i, k), ("A", j, k)}, {("A", i, j)}

    tasks = cholesky_task_list(n, nb)
    return tasks, _mechanical_deps(tasks, access)


def cholesky_random_order(n: int, nb: int, rng: np.random.Generator):
    tasks, preds = cholesky_dependencies(n, nb)
    succ = {t: [] for t in tasks}
    indeg = {t: len(preds[t]) for t in tasks}
    for t, ps in preds.items():
        for x in ps:
            succ[x].append(t)
    ready = [t for t in tasks if indeg[t] == 0]
    order = []
    while ready:
        t = ready.pop(int(rng.integers(len(ready))))
        order.append(t)
        for x in succ[t]:
            indeg[x] -= 1
            if indeg[x] == 0:
                ready.append(x)
    assert len(order) == len(tasks)
    return order


# ---------------------------------------------------------------------------
# Tiled LU with tiled pairwise pivoting (Sec. 3.2.2, Algorithm 3; GETWP).
TASK_GETRF, TASK_GESSM, TASK_TSTRF, TASK_SSSSM = 0, 1, 2, 3


class LUFactored:
    """A (n x n, U and multipliers in place), Lx ((p*ib) x n: the L1 blocks of
    each DTSTRF), piv (p x n ints: the pivots), info (first zero-pivot
    column + 1, or 0)."""

    def __init__(self, A, Lx, piv, n, nb, ib, info):
        self.A, self.Lx, self.piv, self.n, self.nb, self.ib, self.info = A, Lx, piv, n, nb, ib, info

    def U(self) -> np.ndarray:
        return np.triu(self.A)

    def _ip(self):
        return self.piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int))

    def apply(self, Y, solve: bool = False) -> np.ndarray:
        """The factorization's transformations applied to Y (Algorithm 3's
        order); with solve, followed by the back substitution with U: A^{-1} Y."""
        lib = _load()
        Y = _fortran(Y)
        if Y.ndim == 1:
            Y = Y.reshape(-1, 1, order="F")
        rc = lib.oracle_lu_apply(self.n, _dp(self.A), max(self.n, 1), self.nb, self.ib, _dp(self.Lx),
                                 self.Lx.shape[0], self._ip(), Y.shape[1], _dp(Y), max(self.n, 1), int(solve))
        if rc:
            raise ValueError(f"oracle_lu_apply: {rc}")
        return Y

    def solve(self, Y) -> np.ndarray:
        return self.apply(Y, solve=True)

    def N_times(self, X) -> np.ndarray:
        """N X, with N the inverse of the factorization's transformations
        (Sec. 3.2.4): N U reconstructs A."""
        lib = _load()
        X = _fortran(X)
        rc = lib.oracle_lu_unapply(self.n, _dp(self.A), max(self.n, 1), self.nb, self.ib, _dp(self.Lx),
                                   self.Lx.shape[0], self._ip(), X.shape[1], _dp(X), max(self.n, 1))
        if rc:
            raise ValueError(f"oracle_lu_unapply: {rc}")
        return X


def _lu_arrays(n, nb, ib):
    p = n // nb
    Lx = np.zeros((max(p * ib, 1), max(n, 1)), order="F")
    piv = np.zeros((max(p, 1), max(n, 1)), dtype=np.int32, order="F")
    return Lx, piv


def tiled_lu(A, nb: int, ib: int) -> LUFactored:
    """Algorithm 3 on a copy of A (n x n, n a multiple of nb)."""
    lib = _load()
    A = _fortran(A)
    n = A.shape[0]
    Lx, piv = _lu_arrays(n, nb, ib)
    info = lib.oracle_tiled_lu(n, _dp(A), max(n, 1), nb, ib, _dp(Lx), Lx.shape[0],
                               piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if info < 0:
        raise ValueError(f"oracle_tiled_lu: illegal argument {info}")
    return LUFactored(A, Lx, piv, n, nb, ib, info)


def tiled_lu_ordered(A, nb: int, ib: int, tasks) -> LUFactored:
    lib = _load()
    A = _fortran(A)
    n = A.shape[0]
    Lx, piv = _lu_arrays(n, nb, ib)
    tk = np.ascontiguousarray(np.asarray(tasks, dtype=np.int32).reshape(-1, 4))
    info = lib.oracle_tiled_lu_ordered(n, _dp(A), max(n, 1), nb, ib, _dp(Lx), Lx.shape[0],
                                       piv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), tk.shape[0],
                                       tk.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    if info < 0:
        raise ValueError(f"oracle_tiled_lu_ordered: illegal argument {info}")
    return LUFactored(A, Lx, piv, n, nb, ib, info)


def lu_set_mutation(code: int) -> None:
    _load().lu_set_mutation(int(code))


def lu_flops() -> float:
    return _load().lu_flops()


def lu_reset_flops() -> None:
    _load().lu_reset_flops()


def lu_task_list(n: int, nb: int):
    """Tasks {kind, i, j, k} of Algorithm 3 in its printed loop order."""
    p = n // nb
    out = []
    for k in range(p):
        out.append((TASK_GETRF, k, k, k))
        for j in range(k + 1, p):
            out.append((TASK_GESSM, k, j, k))
        for i in range(k + 1, p):
            out.append((TASK_TSTRF, i, k, k))
            for j in range(k + 1, p):
                out.append((TASK_SSSSM, i, j, k))
    return out


def lu_dependencies(n: int, nb: int):
    """Predecessor sets of Algorithm 3 from the tiles each kernel reads and
    writes (Sec. 3.2.2): the diagonal tile is split into its U part ('U')
    and its DGETRF multipliers ('L'); ('X', i, k) are the DTSTRF pivots and
    L1 blocks."""

    def access(t):
        kind, i, j, k = t
        if kind == TASK_GETRF:
            return {("A", k, k)}, {("U", k, k), ("L", k, k)}
        if kind == TASK_GESSM:
            return {("L", k, k)}, {("A", k, j)}
        if kind == TASK_TSTRF:
            return set(), {("U", k, k), ("A", i, k), ("X", i, k)}
        return {("A", i, k), ("X", i, k)}, {("A", k, j), ("A", i, j)}

    tasks = lu_task_list(n, nb)
    return tasks, _mechanical_deps(tasks, access)


def lu_random_order(n: int, nb: int, rng: np.random.Generator):
    tasks, preds = lu_dependencies(n, nb)
    succ = {t: [] for t in tasks}
    indeg = {t: len(preds[t]) for t in tasks}
    for t, ps in preds.items():
        for x in ps:
            succ[x].append(t)
    ready = [t for t in tasks if indeg[t] == 0]
    order = []
    while ready:
        t = ready.pop(int(rng.integers(len(ready))))
        order.append(t)
        for x in succ[t]:
            indeg[x] -= 1
            if indeg[x] == 0:
                ready.append(x)
    assert len(order) == len(tasks)
    return order


def lu_stability(A0: np.ndarray, f: "LUFactored", y=None) -> dict:
    """The measures of Sec. 3.2.4 (infinity norms): backward error of the
    factorization ||A - N U|| / ||A||, of the solution ||y - A x|| / (||A||
    ||x||) for a right-hand side y, ||N||, ||U|| and || |N| |U| ||."""
    n = f.n
    U = f.U()
    N = f.N_times(np.eye(n))
    inf = lambda M: float(np.abs(M).sum(axis=1).max()) if M.size else 0.0
    nA = inf(A0)
    out = {"fact_backward": inf(A0 - N @ U) / nA, "norm_N": inf(N), "norm_U": inf(U),
           "norm_absN_absU": inf(np.abs(N) @ np.abs(U))}
    if y is not None:
        x = f.solve(y)
        out["solve_backward"] = inf(y - A0 @ x) / (nA * inf(x))
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
