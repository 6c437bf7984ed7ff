"""Mixed precision (TILEQR_TF32): DLARFB/DSSRFB as 3xTF32 products on the
tcgen05 tensor cores with FP32 accumulation, DGEQRT/DTSQRT in FP64.

Bounds (derived from the arithmetic):
- one update task, through tileqr_mixed_update_tile against the oracle's
  FP64 DLARFB / DSSRFB on the same reflectors: every product term carries
  ~2^-21 relative error, so each output column is within BOUND = 32 * 2^-21
  of its norm (tests/mixed_cases.py; test_mixed_bound.py shows on the CPU
  that this bound fails products that drop a cross term, i.e. plain TF32);
- the factorization: each column passes through at most p updates, so the
  backward error ||Q^T A - [R; 0]|| / ||A|| stays a small multiple of that,
  checked at <= BACK_BOUND = 2^-16; R agrees with the FP64 oracle to the
  backward error times cond(A) (checked at <= R_BOUND = 2^-13 on these
  well-conditioned shapes).  Plain TF32 products give ~1e-3 here.
- The reflectors are formed in FP64, so the Q they define is orthogonal to
  FP64 rounding (||Q^T Q - I|| <= 20 n eps).
- Any magnitude of A: the FP32 operands are scaled per column by powers of
  two, so A scaled by 2^500 or 2^-530, or with columns graded over 2^+-400,
  gives the same accuracy and no Inf, NaN or flushed update."""
import numpy as np
import pytest
import torch

import mixed_cases as mc
import oracle
from paper_0709_1272_gb300 import inputs

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
BACK_BOUND = 2.0 ** -16
R_BOUND = 2.0 ** -13


@pytest.fixture(scope="module")
def tq():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    tileqr.load()
    return tileqr


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("m,n,ib", [(1000, 700, 32), (512, 512, 16), (2048, 256, 32), (300, 1000, 16),
                                    (129, 129, 32)])
def test_mixed_factor_accuracy(tq, m, n, ib):
    nb = 128
    A = inputs.normal_matrix(m, n, seed=7 + m + n)
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor(Ad, nb, ib, precision=tq.TILEQR_TF32).check()
    R = f.R().cpu().numpy()
    QtA = f.apply_qt(tq.to_device_colmajor(A)).cpu().numpy()
    k = min(m, n)
    back = np.linalg.norm(QtA[:k] - R) / np.linalg.norm(A)
    back_low = np.linalg.norm(QtA[k:]) / np.linalg.norm(A) if m > n else 0.0
    assert back <= BACK_BOUND and back_low <= BACK_BOUND, (back, back_low)
    ref = oracle.tiled_qr(A, nb, ib)
    assert _rel(oracle.sign_normalize(R), oracle.sign_normalize(ref.R())) <= R_BOUND
    # Q is built from FP64 reflectors: orthogonal to FP64 rounding
    if m <= 1024:
        Qt = f.apply_qt(tq.to_device_colmajor(np.eye(m))).cpu().numpy()
        assert np.linalg.norm(Qt @ Qt.T - np.eye(m)) <= 20 * max(m, n) * EPS


def test_mixed_is_deterministic(tq):
    A = inputs.normal_matrix(900, 640, seed=3)
    Ad = tq.to_device_colmajor(A)
    outs = []
    for _ in range(2):
        f = tq.tileqr_factor(Ad, 128, 32, precision=tq.TILEQR_TF32).check()
        AV, T = f.factors()
        outs.append((AV.cpu().numpy(), T.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_mixed_unsupported_combinations_refused(tq):
    Ad = tq.to_device_colmajor(inputs.normal_matrix(256, 256, seed=1))
    for kw in [dict(nb=64, ib=16, precision=tq.TILEQR_TF32),
               dict(nb=128, ib=32, precision=tq.TILEQR_TF32, schedule=tq.TILEQR_SCHED_BULK),
               dict(nb=128, ib=32, precision=tq.TILEQR_SPLIT_BF16)]:
        with pytest.raises(tq.TileQRError) as e:
            tq.tileqr_factor(Ad, **kw)
        assert e.value.code == tq.TILEQR_ERR_UNSUPPORTED


def _dev(x):
    """A column-major tile as a flat float64 CUDA tensor."""
    return torch.from_numpy(np.asfortranarray(x).ravel(order="F").copy()).cuda()


def _host(t, rows):
    return t.cpu().numpy().reshape((rows, -1), order="F")


@pytest.mark.parametrize("ib", [16, 32])
@pytest.mark.parametrize("scale_exp", [0, 500, -530])
def test_single_larfb_task_within_3xtf32_bound(tq, ib, scale_exp):
    V, T, C, ref = mc.larfb_case(ib, scale_exp)
    Cd = _dev(C)
    tq.tileqr_mixed_update_tile(tq.TILEQR_UPDATE_LARFB, ib, _dev(V), _dev(T), None, Cd)
    out = _host(Cd, 128)
    assert np.all(np.isfinite(out))
    # compared at unit scale (exact power-of-two rescaling), so that the
    # norms of the error do not underflow
    err = mc.column_error(np.ldexp(out, -scale_exp), np.ldexp(ref, -scale_exp), np.ldexp(C, -scale_exp))
    assert err <= mc.BOUND, err


@pytest.mark.parametrize("ib", [16, 32])
@pytest.mark.parametrize("scale_exp", [0, 500, -530])
def test_single_ssrfb_task_within_3xtf32_bound(tq, ib, scale_exp):
    V, T, Bp, C, ref = mc.ssrfb_case(ib, scale_exp)
    Bd, Cd = _dev(Bp), _dev(C)
    tq.tileqr_mixed_update_tile(tq.TILEQR_UPDATE_SSRFB, ib, _dev(V), _dev(T), Bd, Cd)
    out = np.vstack([_host(Bd, 128), _host(Cd, 128)])
    assert np.all(np.isfinite(out))
    sc = lambda x: np.ldexp(x, -scale_exp)
    err = mc.column_error(sc(out), sc(ref), sc(np.vstack([Bp, C])))
    assert err <= mc.BOUND, err


def _column_r_error(R, Rref, A):
    """max over columns of ||R(:,c) - Rref(:,c)|| / ||a_c|| after sign
    normalisation (R(:, c) has the norm of a_c)."""
    D = oracle.sign_normalize(R) - oracle.sign_normalize(Rref)
    return float(np.max(np.linalg.norm(D, axis=0) / np.linalg.norm(A, axis=0)))


@pytest.mark.parametrize("scale_exp", [500, -530])
def test_mixed_factor_extreme_uniform_scaling(tq, scale_exp):
    """A scaled by 2^500 (~3e150) or 2^-530 (~3e-160): the TF32 factors
    are those of A scaled alike, to the unscaled accuracy (no overflow to
    Inf, no flushed update)."""
    A = inputs.normal_matrix(700, 500, seed=9)
    As = np.ldexp(A, scale_exp)
    Ad = tq.to_device_colmajor(As)
    f = tq.tileqr_factor(Ad, 128, 16, precision=tq.TILEQR_TF32).check()
    R = f.R().cpu().numpy()
    assert np.all(np.isfinite(R))
    ref = oracle.tiled_qr(A, 128, 16)
    assert _rel(oracle.sign_normalize(np.ldexp(R, -scale_exp)), oracle.sign_normalize(ref.R())) <= R_BOUND
    QtA = f.apply_qt(tq.to_device_colmajor(As)).cpu().numpy()
    back = np.linalg.norm(np.ldexp(QtA[:500] - R, -scale_exp)) / np.linalg.norm(A)
    assert back <= BACK_BOUND, back


def test_mixed_factor_graded_columns(tq):
    """Columns scaled by 2^e with e from -400 to 400: each column of R is
    within the mixed bound of the FP64 oracle's, relative to that column's
    own norm (the FP32 operands are scaled per column)."""
    A = inputs.normal_matrix(600, 384, seed=10)
    e = np.round(np.linspace(-400, 400, 384)).astype(int)
    As = np.ldexp(A, e[None, :])
    f = tq.tileqr_factor(tq.to_device_colmajor(As), 128, 32, precision=tq.TILEQR_TF32).check()
    R = f.R().cpu().numpy()
    assert np.all(np.isfinite(R))
    ref = oracle.tiled_qr(As, 128, 32)
    err = _column_r_error(R, ref.R(), As)
    assert err <= R_BOUND, err


def test_mixed_random_task_delays_keep_the_bits(tq):
    """The TF32 factorization is deterministic too: seeded random task
    delays change the schedule, not the bits."""
    A = inputs.normal_matrix(900, 640, seed=3)
    Ad = tq.to_device_colmajor(A)
    f0 = tq.tileqr_factor(Ad, 128, 32, precision=tq.TILEQR_TF32).check()
    AV0, T0 = f0.factors()
    AV0, T0 = AV0.cpu().numpy(), T0.cpu().numpy()
    for seed in (5, 6):
        f = tq.tileqr_factor(Ad, 128, 32, precision=tq.TILEQR_TF32,
                             flags=tq.TILEQR_FLAG_TEST_RANDOM_DELAYS | (seed << 8)).check()
        AV, T = f.factors()
        assert np.array_equal(AV.cpu().numpy(), AV0) and np.array_equal(T.cpu().numpy(), T0)
