"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerance: relative Frobenius error 1e-12 in FP64 (R after sign
normalisation; V and T compared directly, since with equal (nb, ib) both
sides compute the same reflectors in the same order).  Integer-exact checks:
the persistent task-graph kernel and the fork-join comparator produce
identical bits (every tile is written by a fixed sequence of deterministic
tasks), and so do repeated runs.
"""
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


def _gpu_factor(tq, A, nb, ib, schedule=0):
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor(Ad, nb, ib, schedule=schedule).check()
    AV, T = f.factors()
    R = f.R()
    torch.cuda.synchronize()
    return f, Ad, AV.cpu().numpy(), T.cpu().numpy(), R.cpu().numpy()


CASES = [
    # (m, n, nb, ib, generator)  -- several tiles each, ragged tails included
    (512, 512, 64, 16, "uniform"),      # the 512 x 512, nb 64, ib 16 workload
    (1000, 700, 128, 32, "normal"),
    (700, 1000, 128, 16, "normal"),
    (640, 200, 64, 32, "uniform"),
    (300, 300, 256, 32, "normal"),
    (777, 333, 256, 16, "normal"),
    (2048, 256, 128, 32, "normal"),     # tall-skinny shape, reduced
    (65, 65, 64, 16, "uniform"),        # one full tile plus a 1-wide ragged edge
    (1, 1, 64, 16, "uniform"),
    (5, 200, 64, 16, "normal"),         # wide, a single partial tile row
]


@pytest.mark.parametrize("m,n,nb,ib,gen", CASES)
def test_factor_matches_oracle(tq, m, n, nb, ib, gen):
    g = inputs.uniform_matrix if gen == "uniform" else inputs.normal_matrix
    A = g(m, n, seed=1000 + m + 7 * n)
    f, _, AV, T, R = _gpu_factor(tq, A, nb, ib)
    ref = oracle.tiled_qr(A, nb, ib)
    assert _rel(oracle.sign_normalize(R), oracle.sign_normalize(ref.R())) <= TOL
    assert _rel(AV, ref.A) <= TOL
    assert _rel(T, ref.T) <= TOL
    assert np.all(np.tril(R, -1) == 0.0)


@pytest.mark.parametrize("m,n,nb,ib", [(1000, 700, 128, 32), (512, 512, 64, 16), (600, 900, 256, 32)])
def test_dag_equals_fork_join_bitwise(tq, m, n, nb, ib):
    A = inputs.normal_matrix(m, n, seed=77)
    _, _, AV0, T0, _ = _gpu_factor(tq, A, nb, ib, schedule=tq.TILEQR_SCHED_DAG)
    _, _, AV1, T1, _ = _gpu_factor(tq, A, nb, ib, schedule=tq.TILEQR_SCHED_BULK)
    _, _, AV2, T2, _ = _gpu_factor(tq, A, nb, ib, schedule=tq.TILEQR_SCHED_DAG)
    assert np.array_equal(AV0, AV1) and np.array_equal(T0, T1)
    assert np.array_equal(AV0, AV2) and np.array_equal(T0, T2)


def test_invariants_512(tq):
    m = n = 512
    A = inputs.uniform_matrix(m, n, seed=20070710)
    f, Ad, AV, T, R = _gpu_factor(tq, A, 64, 16)
    Qt = f.apply_qt(tq.to_device_colmajor(np.eye(m))).cpu().numpy()
    Q = Qt.T
    assert np.linalg.norm(Q.T @ Q - np.eye(m)) <= 20 * n * EPS
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= 20 * n * EPS


@pytest.mark.parametrize("m,n,nb,ib,nrhs", [(1000, 700, 128, 32, 16), (512, 512, 64, 16, 3),
                                            (777, 333, 256, 16, 40)])
def test_apply_qt_and_solve_match_oracle(tq, m, n, nb, ib, nrhs):
    A = inputs.normal_matrix(m, n, seed=5)
    B = inputs.normal_matrix(m, nrhs, seed=6)
    f, _, _, _, _ = _gpu_factor(tq, A, nb, ib)
    ref = oracle.tiled_qr(A, nb, ib)
    QtB = f.apply_qt(tq.to_device_colmajor(B)).cpu().numpy()
    assert _rel(QtB, oracle.apply_qt(ref, B)) <= TOL
    X = f.solve_ls(tq.to_device_colmajor(B)).cpu().numpy()
    Xo = oracle.solve_ls(ref, B)
    assert _rel(X, Xo) <= 1e-10
    r = B - A @ X
    if m > n:   # inconsistent system: the residual is orthogonal to range(A)
        assert np.linalg.norm(A.T @ r) / (np.linalg.norm(A) * np.linalg.norm(r)) <= 20 * n * EPS
    else:       # square: normwise backward error of the solve (Sec. 3.2.4 metric)
        assert np.linalg.norm(r) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 20 * n * EPS


@pytest.mark.parametrize("scale", [1e150, 1e-160])
def test_extreme_magnitudes(tq, scale):
    """Columns whose squared norms over- or underflow take the rescaled-norm
    path of the panel kernels; results must still match the oracle, which
    always accumulates norms with scaling."""
    A = inputs.normal_matrix(300, 200, seed=31) * scale
    f, _, AV, T, R = _gpu_factor(tq, A, 64, 16)
    ref = oracle.tiled_qr(A, 64, 16)
    assert np.all(np.isfinite(AV)) and np.all(np.isfinite(T))
    assert _rel(AV, ref.A) <= TOL
    assert _rel(T, ref.T) <= TOL


def test_tails_whose_squares_underflow(tq):
    """A graded matrix (singular values 1 .. 1e-6) scaled by 2^-530: late
    panel columns have tails of ~1e-166, whose squares underflow to zero;
    the panel must still see a nonzero tail (rescaled norm), as the oracle
    does.  R is compared at unit scale (exact power-of-two rescaling)."""
    A, _, _, _ = inputs.kappa_matrix(384, 1e6, seed=33)
    As = np.ldexp(A, -530)
    f, _, AV, T, R = _gpu_factor(tq, As, 64, 16)
    ref = oracle.tiled_qr(As, 64, 16)
    assert np.all(np.isfinite(AV)) and np.all(np.isfinite(T))
    assert _rel(np.ldexp(np.triu(AV[:384]), 530), np.ldexp(np.triu(ref.A[:384]), 530)) <= TOL
    assert _rel(np.tril(AV, -1), np.tril(ref.A, -1)) <= TOL
    assert _rel(T, ref.T) <= TOL


def test_nonfinite_input_is_reported(tq):
    A = inputs.normal_matrix(300, 200, seed=1)
    A[17, 33] = np.nan
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor(Ad, 64, 16)
    assert f.status() == tq.TILEQR_ERR_NONFINITE


def test_watchdog_reports_timeout_and_context_survives(tq):
    """The scheduler never releases the final task: the persistent kernel's
    bounded waits must expire, record TILEQR_ERR_TIMEOUT and return; the next
    factorization on the same context must succeed."""
    A = inputs.normal_matrix(256, 256, seed=2)
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor(Ad, 64, 16, flags=tq.TILEQR_FLAG_TEST_WITHHOLD_LAST_TASK)
    assert f.status() == tq.TILEQR_ERR_TIMEOUT
    g = tq.tileqr_factor(Ad, 64, 16).check()
    ref = oracle.tiled_qr(A, 64, 16)
    assert _rel(g.factors()[0].cpu().numpy(), ref.A) <= TOL


def test_singular_solve_is_reported(tq):
    A = np.array(inputs.normal_matrix(256, 128, seed=3), order="F")
    A[:, 70] = 0.0       # a zero column stays exactly zero under the reflections: R(70,70) == 0
    f, _, _, _, R = _gpu_factor(tq, A, 64, 16)
    assert R[70, 70] == 0.0
    with pytest.raises(tq.TileQRError) as e:
        f.solve_ls(tq.to_device_colmajor(np.ones((256, 1))))
    assert e.value.code in (tq.TILEQR_ERR_SINGULAR,)


def test_empty_and_degenerate(tq):
    for (m, n) in [(0, 5), (5, 0), (0, 0)]:
        A = torch.zeros((max(n, 1), max(m, 1)), dtype=torch.float64, device="cuda").t()[:m, :n]
        f = tq.tileqr_factor(A, 64, 16)
        assert f.status() == 0
    # a zero matrix: no reflection anywhere, R == 0, T == 0
    A = np.zeros((200, 130), order="F")
    f, _, AV, T, R = _gpu_factor(tq, A, 64, 16)
    assert not np.any(AV) and not np.any(T)


# ---------------------------------------------------------------------------
# full-size workloads, in the launch configuration the benchmark times
@pytest.mark.parametrize("ib", [16, 32])
def test_full_16384_sampled(tq, ib):
    """16384 x 16384 N(0,1), nb 128, ib 16 (the benchmarked launch) and 32,
    persistent kernel.  Sampled
    against the oracle: the first tile column's R_00, V_i0, T_i0 (the oracle
    factors that 16384 x 128 panel) and the first tile row R_0j for sampled
    j (the oracle applies those reflectors to column block j).  Properties at
    full size: Q^T (A x) = R x and ||Q^T y|| = ||y||."""
    m = n = 16384
    nb = 128
    A = inputs.normal_matrix(m, n, seed=20070711)
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor(Ad, nb, ib).check()
    R = f.R()
    AV, T = f.factors()
    panel = oracle.tiled_qr(A[:, :nb], nb, ib)
    AVc = AV[:, :nb].cpu().numpy()
    Tc = T[:, :nb].cpu().numpy()
    assert _rel(AVc[nb:], panel.A[nb:]) <= TOL                     # V_i0, i > 0
    assert _rel(np.tril(AVc[:nb], -1), np.tril(panel.A[:nb], -1)) <= TOL   # V_00
    assert _rel(Tc, panel.T) <= TOL
    assert _rel(np.triu(AVc[:nb]), np.triu(panel.A[:nb])) <= TOL   # R_00
    for j in (1, 57, 127):
        blk = oracle.apply_qt(panel, A[:, j * nb:(j + 1) * nb])
        assert _rel(R[:nb, j * nb:(j + 1) * nb].cpu().numpy(), blk[:nb]) <= TOL
    x = inputs.normal_matrix(n, 2, seed=9)
    xd = tq.to_device_colmajor(x)
    Ax = Ad @ xd
    QtAx = f.apply_qt(tq.as_colmajor(Ax.clone())).cpu().numpy()
    Rx = (R @ xd).cpu().numpy()
    assert _rel(QtAx, Rx) <= 1e-11
    y = inputs.normal_matrix(m, 1, seed=10)
    Qty = f.apply_qt(tq.to_device_colmajor(y)).cpu().numpy()
    assert abs(np.linalg.norm(Qty) / np.linalg.norm(y) - 1.0) <= 1e-12


def test_full_tall_skinny_solve(tq):
    """262144 x 512 N(0,1), nb 128, ib 16 (the benchmarked flat-tree launch),
    with tileqr_solve_ls on 16 RHS.  Sampled: the first tile column against
    the oracle; properties: the least-squares optimality ||A^T r|| / (||A||
    ||r||) at rounding level."""
    m, n, nb, ib = 262144, 512, 128, 16
    A = inputs.normal_matrix(m, n, seed=20070712)
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor(Ad, nb, ib).check()
    AV, T = f.factors()
    panel = oracle.tiled_qr(A[:, :nb], nb, ib)
    assert _rel(AV[:, :nb].cpu().numpy(), panel.A) <= TOL
    assert _rel(T[:, :nb].cpu().numpy(), panel.T) <= TOL
    B = inputs.normal_matrix(m, 16, seed=20070713)
    Bd = tq.to_device_colmajor(B)
    X = f.solve_ls(Bd.clone())
    r = Bd - Ad @ X
    Atr = (Ad.t() @ r)
    nA = torch.linalg.matrix_norm(Ad, ord="fro")
    ratio = (torch.linalg.matrix_norm(Atr) / (nA * torch.linalg.matrix_norm(r))).item()
    assert ratio <= 20 * n * EPS


def test_full_elementwise_4096(tq):
    """4096 x 4096 N(0,1), nb 128 / ib 16, the persistent task-graph kernel
    at two CTAs per SM with 32 steps of queue contention (the benchmarked
    launch configuration): every element of R/V (in place) and of the T
    strips against the oracle's Algorithm 2 at 1e-12 (the oracle run level
    by level on all host cores; identical bits to its sequential order)."""
    import os
    m = n = 4096
    A = inputs.normal_matrix(m, n, seed=20070715)
    f, _, AV, T, R = _gpu_factor(tq, A, 128, 16)
    ref, _ = oracle.tiled_qr_levels(A, 128, 16, len(os.sched_getaffinity(0)))
    assert _rel(AV, ref.A) <= TOL
    assert _rel(T, ref.T) <= TOL
    assert _rel(oracle.sign_normalize(R), oracle.sign_normalize(ref.R())) <= TOL


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_task_delays_keep_the_bits(tq, seed):
    """Schedule stress test: with TILEQR_FLAG_TEST_RANDOM_DELAYS every task
    sleeps a seeded pseudo-random time before it runs and before it releases
    its successors; the factors must equal the fork-join comparator's bit
    for bit (any topological order gives the same bits, Sec. 4)."""
    A = inputs.normal_matrix(1000, 700, seed=77)
    Ad = tq.to_device_colmajor(A)
    flags = tq.TILEQR_FLAG_TEST_RANDOM_DELAYS | (seed << 8)
    f = tq.tileqr_factor(Ad, 128, 32, flags=flags).check()
    AV, T = f.factors()
    _, _, AV1, T1, _ = _gpu_factor(tq, A, 128, 32, schedule=tq.TILEQR_SCHED_BULK)
    assert np.array_equal(AV.cpu().numpy(), AV1) and np.array_equal(T.cpu().numpy(), T1)
