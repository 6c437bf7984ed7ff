"""Mixed precision (TILEQR_TF32): DLARFB/DSSRFB as 3xTF32 products on the
tcgen05 tensor cores with FP32 accumulation, DGEQRT/DTSQRT in FP64.

Bound used here (derived from the arithmetic): every update product carries
~2^-21 relative error and is accumulated in FP32 (2^-24), so the backward
error ||Q^T A - [R; 0]|| / ||A|| of the factorization is an FP32-level
quantity, checked at <= 32 n 2^-24 for these well-conditioned shapes; R
then agrees with the FP64 oracle to that backward error times cond(A)
(checked at <= 1e-4).  The reflectors are formed in FP64, so the Q they
define is orthogonal to FP64 rounding (||Q^T Q - I|| <= 20 n eps)."""
import numpy as np
import pytest
import torch

import oracle
from paper_0709_1272_gb300 import inputs

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps
U32 = 2.0 ** -24


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
    assert back <= 32 * n * U32 and back_low <= 32 * n * U32
    ref = oracle.tiled_qr(A, nb, ib)
    assert _rel(oracle.sign_normalize(R), oracle.sign_normalize(ref.R())) <= 1e-4
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
