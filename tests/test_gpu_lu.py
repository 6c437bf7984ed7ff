"""Tiled LU with tiled pairwise pivoting (Sec. 3.2.2, Algorithm 3) on the GPU
against the CPU oracle, element by element through the C ABI.

Both sides run DGETRF / DGESSM / DTSTRF / DSSSSM on the same tiles with the
same pivot rule, so they differ only in rounding order: the pivots (an
argmax, decided in FP64 on both sides) must be identical on these seeded
inputs, the factors agree to TOL relative to their largest entry.  TOL comes
from the arithmetic: every entry is a sum of at most n products formed in a
different order, ~n eps of the largest intermediate (growth stays below 10
on these inputs), so 64 n eps with n <= 640 gives 1e-11.
Sizes that are not a multiple of nb are compared with the oracle run on the
identity-padded matrix diag(A, I), which is what the library factors.
The full-size case (16384, nb 128, ib 16: the benchmark's launch) is checked
by properties that hold at any size: the multipliers are bounded by 1, the
pivots are valid candidates, and the solve reaches rounding-level backward
error (Sec. 3.2.4's measure)."""
import numpy as np
import pytest
import torch

import oracle
from paper_0709_1272_gb300 import inputs

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
TOL = 1e-11


@pytest.fixture(scope="module")
def tq():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    tileqr.load()
    return tileqr


def _padded(A, nb):
    n = A.shape[0]
    p = -(-n // nb)
    Ap = np.eye(p * nb)
    Ap[:n, :n] = A
    return Ap


def _compare(tq, A, nb, ib):
    n = A.shape[0]
    f = tq.tileqr_lu(tq.to_device_colmajor(A), nb, ib).check()
    F, Lx, piv = (t.cpu().numpy() for t in f.factors())
    o = oracle.tiled_lu(_padded(A, nb), nb, ib)
    assert np.array_equal(piv, o.piv[:, :n])
    scale = max(np.abs(o.A[:n, :n]).max(), 1e-300)
    assert np.abs(F - o.A[:n, :n]).max() <= TOL * scale
    assert np.abs(Lx - o.Lx[:, :n]).max() <= TOL
    assert f.info() == o.info
    return f, o


@pytest.mark.parametrize("n,nb,ib", [(256, 64, 16), (320, 64, 32), (384, 128, 16), (512, 128, 32),
                                     (640, 128, 16), (200, 64, 16), (130, 128, 16), (64, 64, 16), (1, 64, 16)])
def test_lu_matches_oracle(tq, n, nb, ib):
    A = inputs.normal_matrix(n, n, seed=3000 + n + nb + ib)
    _compare(tq, A, nb, ib)


def test_lu_uniform_entries(tq):
    A = inputs.uniform_matrix(448, 448, seed=31)
    _compare(tq, A, 64, 16)


@pytest.mark.parametrize("n,nb,ib", [(384, 64, 16), (520, 128, 32)])
def test_lu_solve_matches_oracle(tq, n, nb, ib):
    A = inputs.normal_matrix(n, n, seed=41)
    B = inputs.normal_matrix(n, 40, seed=42)   # two column chunks, the second ragged
    f = tq.tileqr_lu(tq.to_device_colmajor(A), nb, ib).check()
    X = f.solve(tq.to_device_colmajor(B)).cpu().numpy()
    o = oracle.tiled_lu(_padded(A, nb), nb, ib)
    Bp = np.zeros((o.n, B.shape[1]))
    Bp[:n] = B
    Xo = o.solve(Bp)[:n]
    assert np.abs(X - Xo).max() <= 1e-9 * np.abs(Xo).max()
    inf = lambda M: np.abs(M).sum(axis=1).max()
    assert inf(B - A @ X) / (inf(A) * inf(X)) <= 10 * n * EPS
    x1 = f.solve(tq.to_device_colmajor(B[:, 0])).cpu().numpy().reshape(-1)
    assert np.abs(x1 - X[:, 0]).max() == 0.0


def test_lu_identity_and_diagonal(tq):
    n = 300
    f = tq.tileqr_lu(tq.to_device_colmajor(np.eye(n)), 64, 16).check()
    F, Lx, piv = (t.cpu().numpy() for t in f.factors())
    assert np.array_equal(F, np.eye(n))
    # every DTSTRF L1 block is the identity (unit diagonal stored), zero for i <= k
    p = 5
    Lexp = np.zeros((p * 16, p * 64))
    for k in range(p):
        for i in range(k + 1, p):
            Lexp[i * 16:(i + 1) * 16, k * 64:(k + 1) * 64] = np.tile(np.eye(16), (1, 4))
    assert np.array_equal(Lx, Lexp[:, :n])
    # no interchange anywhere: DGETRF keeps row c, DTSTRF keeps the U row c
    for col in range(n):
        k, c = divmod(col, 64)
        assert np.all(piv[k:, col] == c) and np.all(piv[:k, col] == 0)
    d = np.diag(np.linspace(1.0, 3.0, n))
    g = tq.tileqr_lu(tq.to_device_colmajor(d), 64, 16).check()
    assert np.array_equal(g.factors()[0].cpu().numpy(), d)


def test_lu_zero_pivot_reported(tq):
    n = 256
    A = inputs.normal_matrix(n, n, seed=12)
    A[:, 100] = 0.0
    f, o = _compare(tq, A, 64, 16)
    assert f.info() == 101 == o.info


def test_lu_singular_solve_reports(tq):
    A = inputs.normal_matrix(128, 128, seed=13)
    A[:, 5] = 0.0
    f = tq.tileqr_lu(tq.to_device_colmajor(A), 64, 16).check()
    with pytest.raises(tq.TileQRError) as e:
        f.solve(tq.to_device_colmajor(np.ones((128, 1))))
    assert e.value.code == tq.TILEQR_ERR_SINGULAR


def test_lu_nonfinite_input(tq):
    A = inputs.normal_matrix(200, 200, seed=14)
    A[17, 33] = np.nan
    f = tq.tileqr_lu(tq.to_device_colmajor(A), 64, 16)
    assert f.status() == tq.TILEQR_ERR_NONFINITE
    B = inputs.normal_matrix(200, 200, seed=15)
    _compare(tq, B, 64, 16)   # the context stays usable


def test_lu_watchdog(tq):
    A = inputs.normal_matrix(256, 256, seed=16)
    f = tq.tileqr_lu(tq.to_device_colmajor(A), 64, 16, flags=tq.TILEQR_FLAG_TEST_WITHHOLD_LAST_TASK)
    assert f.status() == tq.TILEQR_ERR_TIMEOUT
    _compare(tq, A, 64, 16)


def test_lu_argument_errors(tq):
    import ctypes
    lib = tq.load()
    d = tq.tileqr_desc()
    buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    A = tq.to_device_colmajor(np.eye(8))
    vp = ctypes.c_void_p
    assert lib.tileqr_lu(-1, vp(A.data_ptr()), 8, 64, 16, 0, vp(buf.data_ptr()), buf.numel(), None, ctypes.byref(d)) == -1
    assert lib.tileqr_lu(8, vp(A.data_ptr()), 4, 64, 16, 0, vp(buf.data_ptr()), buf.numel(), None, ctypes.byref(d)) == -3
    assert lib.tileqr_lu(8, vp(A.data_ptr()), 8, 64, 24, 0, vp(buf.data_ptr()), buf.numel(), None, ctypes.byref(d)) == -5
    assert lib.tileqr_lu(8, vp(A.data_ptr()), 8, 96, 16, 0, vp(buf.data_ptr()), buf.numel(), None,
                         ctypes.byref(d)) == tq.TILEQR_ERR_UNSUPPORTED
    assert lib.tileqr_lu(8, vp(A.data_ptr()), 8, 64, 16, 0, vp(buf.data_ptr()), 100, None,
                         ctypes.byref(d)) == tq.TILEQR_ERR_WORKSPACE
    assert lib.tileqr_lu(0, None, 1, 64, 16, 0, vp(buf.data_ptr()), buf.numel(), None, ctypes.byref(d)) == 0


def test_lu_full_size_properties(tq):
    # the benchmark's launch: 16384 x 16384 N(0,1), nb 128, ib 16
    n, nb, ib = 16384, 128, 16
    g = torch.Generator(device="cuda").manual_seed(20070709)
    A = torch.randn((n, n), generator=g, dtype=torch.float64, device="cuda").t()
    f = tq.tileqr_lu(A, nb, ib).check()
    assert f.info() == 0
    F, Lx, piv = f.factors()
    p = n // nb
    # every multiplier is bounded by 1 (each pivot is the largest candidate)
    for k in range(0, p, 7):
        blk = F[k * nb:, k * nb:(k + 1) * nb]
        low = torch.tril(blk[:nb], -1)
        assert low.abs().max().item() <= 1.0
        if k + 1 < p:
            assert blk[nb:].abs().max().item() <= 1.0
    assert Lx.abs().max().item() <= 1.0
    # pivots: DGETRF's lie in [c, nb), DTSTRF's in [c, 2 nb) (stacked rows)
    pv = piv.cpu().numpy()
    c = np.arange(n) % nb
    kk = np.arange(n) // nb
    for k in range(0, p, 5):
        cols = kk == k
        assert np.all(pv[k, cols] >= c[cols]) and np.all(pv[k, cols] < nb)
        if k + 1 < p:
            sub = pv[k + 1:, cols]
            assert np.all(sub >= c[cols][None, :]) and np.all(sub < 2 * nb)
    # Sec. 3.2.4: solution backward error at rounding level
    B = torch.randn((n, 4), generator=g, dtype=torch.float64, device="cuda")
    X = f.solve(B)
    inf = lambda M: M.abs().sum(dim=1).max().item()
    be = inf(B - A @ X) / (inf(A) * inf(X))
    assert be <= n * EPS, be
