"""Tiled Cholesky (Sec. 3.1, Algorithm 1) on the GPU against the CPU oracle,
element by element through the C ABI (relative Frobenius 1e-12 on L; both
sides run DPOTF2 / DTRSM / DGSMM on the same tiles, so they differ only in
rounding order), plus the failure paths (not positive definite, non-finite
input, an unread upper triangle) and a large case checked by properties
that hold at any size: L_00 is the Cholesky factor of A_00, the first block
column solves L_i0 L_00^T = A_i0, and L L^T = A to rounding."""
import numpy as np
import pytest
import torch

import oracle
from paper_0709_1272_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12
EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def tq():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    tileqr.load()
    return tileqr


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("n,nb", [(512, 64), (1000, 128), (777, 64), (129, 128), (64, 64), (1, 64), (3000, 128)])
def test_cholesky_matches_oracle(tq, n, nb):
    A = inputs.spd_matrix(n, seed=1000 + n)
    f = tq.tileqr_cholesky(tq.to_device_colmajor(A), nb).check()
    assert f.info() == 0
    L = f.L().cpu().numpy()
    Lo, info = oracle.tiled_cholesky(A, nb)
    assert info == 0
    assert _rel(L, Lo) <= TOL
    assert np.array_equal(L, np.tril(L))
    assert np.abs(L @ L.T - A).max() <= 10 * n * EPS * np.abs(A).max()


def test_not_positive_definite(tq):
    n = 700
    A = inputs.spd_matrix(n, seed=7)
    A[300, 300] = -5.0
    f = tq.tileqr_cholesky(tq.to_device_colmajor(A), 64)
    assert f.status() == tq.TILEQR_ERR_NOT_SPD
    _, info = oracle.tiled_cholesky(A, 64)
    assert f.info() == info and 1 <= info <= 301
    # the context stays usable
    B = inputs.spd_matrix(300, seed=8)
    g = tq.tileqr_cholesky(tq.to_device_colmajor(B), 64).check()
    assert _rel(g.L().cpu().numpy(), oracle.tiled_cholesky(B, 64)[0]) <= TOL


def test_upper_triangle_not_read_and_nonfinite_lower_reported(tq):
    n = 500
    A = inputs.spd_matrix(n, seed=9)
    B = A.copy(order="F")
    B[np.triu_indices(n, 1)] = np.nan
    f = tq.tileqr_cholesky(tq.to_device_colmajor(B), 128).check()
    assert _rel(f.L().cpu().numpy(), oracle.tiled_cholesky(A, 128)[0]) <= TOL
    C = A.copy(order="F")
    C[400, 10] = np.inf
    g = tq.tileqr_cholesky(tq.to_device_colmajor(C), 128)
    assert g.status() == tq.TILEQR_ERR_NONFINITE


def test_cholesky_8192_properties(tq):
    n, nb = 8192, 128
    A = inputs.spd_matrix(n, seed=20070714)
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_cholesky(Ad, nb).check()
    L = f.L()
    Ln = L[:, :nb].cpu().numpy()
    L00 = np.linalg.cholesky(A[:nb, :nb])
    assert _rel(Ln[:nb], L00) <= TOL
    # first block column: L_i0 L_00^T = A_i0
    assert np.abs(Ln[nb:] @ L00.T - A[nb:, :nb]).max() <= 20 * nb * EPS * np.abs(A[nb:, :nb]).max()
    Lt = torch.tril(L)
    err = (torch.linalg.matrix_norm(Lt @ Lt.t() - torch.tril(Ad) - torch.tril(Ad, -1).t()) /
           torch.linalg.matrix_norm(Ad)).item()
    assert err <= 10 * n * EPS


def test_cholesky_trace_respects_dependencies(tq):
    # the persistent kernel's trace honours the Algorithm 1 dependencies
    n, nb = 1280, 128
    A = inputs.spd_matrix(n, seed=11)
    tasks, preds = oracle.cholesky_dependencies(n, nb)
    rec = torch.zeros((len(tasks) + 16, 4), dtype=torch.int64, device="cuda")
    tq.tileqr_set_trace(rec)
    try:
        f = tq.tileqr_cholesky(tq.to_device_colmajor(A), nb).check()
        cnt = tq.tileqr_trace_count(f)
    finally:
        tq.tileqr_set_trace(None)
    r = rec.cpu().numpy()
    assert cnt == len(tasks)
    code = r[:cnt, 0].astype(np.uint64)
    k = ((code >> np.uint64(42)) & np.uint64(0x1FFFFF)).astype(int)
    i = ((code >> np.uint64(21)) & np.uint64(0x1FFFFF)).astype(int)
    j = (code & np.uint64(0x1FFFFF)).astype(int)
    seen = {}
    for t in range(cnt):
        kind = 0 if (i[t] == k[t] and j[t] == k[t]) else (1 if j[t] == k[t] else 2)
        seen[(kind, int(i[t]), int(j[t]), int(k[t]))] = (int(r[t, 1]), int(r[t, 2]))
    assert set(seen) == set(tasks)
    for t in tasks:
        for pr in preds[t]:
            assert seen[pr][1] <= seen[t][0]


def test_full_16384(tq):
    """The benchmarked launch: 16384 x 16384 SPD (G + G^T)/2 + n I with the
    benchmark's seed, nb 128.  Properties at full size: L is lower triangular
    with a positive diagonal, and (L L^T)[rows, :] = A[rows, :] to rounding
    on 64 sampled rows."""
    n, nb = 16384, 128
    A = inputs.spd_matrix(n, seed=20070709 + 7)
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_cholesky(Ad, nb).check()
    assert f.info() == 0
    L = f.L()
    assert torch.count_nonzero(torch.triu(L, 1)).item() == 0
    assert (torch.diagonal(L) > 0).all().item()
    rows = torch.from_numpy(np.random.Generator(np.random.Philox(key=5)).choice(n, 64, replace=False)).cuda()
    LLt = L[rows] @ L.t()
    err = (LLt - Ad[rows]).abs().max().item()
    assert err <= 10 * n * EPS * np.abs(A).max()
