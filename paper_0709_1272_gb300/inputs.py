"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the factorization: it only draws matrices
with the distributions and shapes of the workloads (dense random matrices as
in the experiments of Sec. 5, which factor randn/uniform matrices; a
matrix with prescribed singular values; a ragged batch of shapes).  numpy's
Philox bit generator keyed by the seed makes every draw reproducible on any
host.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20070709


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed) & (2**64 - 1)))


def uniform_matrix(m: int, n: int, seed: int) -> np.ndarray:
    """m x n, entries iid uniform[-1, 1), column-major float64."""
    return _rng(seed).uniform(-1.0, 1.0, size=(n, m)).T


def normal_matrix(m: int, n: int, seed: int) -> np.ndarray:
    """m x n, entries iid N(0, 1), column-major float64."""
    return _rng(seed).standard_normal(size=(n, m)).T


def kappa_matrix(n: int, kappa: float, seed: int):
    """A = (I - 2 u u^T) diag(s) (I - 2 v v^T) with unit u, v drawn from N(0,1)
    and s_i = kappa^(-(i)/(n-1)), i = 0..n-1 (geometric from 1 to 1/kappa).

    The singular values of A are exactly s, so cond_2(A) = kappa.  Returns
    (A column-major, s, u, v).  Formed as D - 2 u (u^T D) - 2 (D v) v^T
    + 4 (u^T D v) u v^T, O(n^2) work.
    """
    g = _rng(seed)
    u = g.standard_normal(n)
    u /= np.linalg.norm(u)
    v = g.standard_normal(n)
    v /= np.linalg.norm(v)
    s = kappa ** (-np.arange(n, dtype=np.float64) / max(n - 1, 1))
    su = s * u          # D u  (= D^T u)
    sv = s * v          # D v
    c = float(u @ sv)   # u^T D v
    A = np.zeros((n, n), dtype=np.float64, order="F")
    A[np.arange(n), np.arange(n)] = s
    A -= 2.0 * np.outer(u, su)
    A -= 2.0 * np.outer(sv, v)
    A += 4.0 * c * np.outer(u, v)
    return A, s, u, v


def kappa_factors(n: int, kappa: float, seed: int):
    """(s, u, v) of kappa_matrix(n, kappa, seed), without forming A: the same
    draws, so A = (I - 2uu^T) diag(s) (I - 2vv^T) can be formed elsewhere
    (e.g. on the device) from them."""
    g = _rng(seed)
    u = g.standard_normal(n)
    u /= np.linalg.norm(u)
    v = g.standard_normal(n)
    v /= np.linalg.norm(v)
    s = kappa ** (-np.arange(n, dtype=np.float64) / max(n - 1, 1))
    return s, u, v


def kappa_columns(n: int, kappa: float, seed: int, j0: int, j1: int) -> np.ndarray:
    """Columns j0..j1-1 of kappa_matrix(n, kappa, seed) (n x (j1-j0),
    column-major), formed entry by entry from the same (s, u, v)."""
    s, u, v = kappa_factors(n, kappa, seed)
    c = float(u @ (s * v))
    cols = np.arange(j0, j1)
    A = np.zeros((n, j1 - j0), dtype=np.float64, order="F")
    A[cols, np.arange(j1 - j0)] = s[cols]
    A -= 2.0 * np.outer(u, (s * u)[cols])
    A -= 2.0 * np.outer(s * v, v[cols])
    A += 4.0 * c * np.outer(u, v[cols])
    return A


def spd_matrix(n: int, seed: int) -> np.ndarray:
    """Symmetric positive definite n x n: (G + G^T)/2 + n I with G uniform[-1,1)
    (column-major).  Each row's off-diagonal absolute sum is about n/2 < n, so
    the matrix is strictly diagonally dominant with a positive diagonal
    (Gershgorin: SPD, condition number at most about 3)."""
    G = _rng(seed).uniform(-1.0, 1.0, size=(n, n))
    A = 0.5 * (G + G.T)
    A[np.arange(n), np.arange(n)] += n
    return np.asfortranarray(A)


def batch_shapes(count: int, seed: int, m_lo: int = 64, m_hi: int = 2048, n_lo: int = 32):
    """Ragged batch: m uniform in [m_lo, m_hi], n uniform in [n_lo, m]."""
    g = _rng(seed)
    ms = g.integers(m_lo, m_hi + 1, size=count)
    ns = np.array([g.integers(n_lo, int(m) + 1) for m in ms], dtype=np.int64)
    return [(int(m), int(n)) for m, n in zip(ms, ns)]


def batch_matrices(shapes, seed: int):
    """One uniform[-1,1) matrix per shape, item b drawn from seed + 1 + b."""
    return [uniform_matrix(m, n, seed + 1 + b) for b, (m, n) in enumerate(shapes)]


def batch_pool(shapes, seed: int, threads: int | None = None):
    """All matrices of a batch in one flat float64 buffer (matrix b occupies
    m_b * n_b consecutive values, column-major), drawn exactly as
    batch_matrices(shapes, seed) would draw them, in parallel threads (numpy's
    generators release the GIL).  Returns (pool, offsets)."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    offsets, tot = [], 0
    for (m, n) in shapes:
        offsets.append(tot)
        tot += m * n
    pool = np.empty(tot, dtype=np.float64)

    def fill(b):
        m, n = shapes[b]
        pool[offsets[b]:offsets[b] + m * n] = _rng(seed + 1 + b).uniform(-1.0, 1.0, size=m * n)

    with ThreadPoolExecutor(threads or os.cpu_count() or 4) as ex:
        list(ex.map(fill, range(len(shapes))))
    return pool, offsets
