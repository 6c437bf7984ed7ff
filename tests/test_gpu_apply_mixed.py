"""Q^T B and Q B on the tensor cores (tileqr_apply_mixed) for TILEQR_TF32
factorizations, against the oracle applying the same reflectors in FP64.

The oracle side is oracle.apply_qt / oracle.apply_q on the factors the GPU
computed (tileqr_get_factors, tileqr_get_tree_T), so both sides apply the
same V and T in the same order (Sec. 3.2.1, Algorithm 2 and its reverse);
they differ by the 3xTF32 products with FP32 accumulation of the mixed
updates.  Bound: each update task keeps the single-task bound of
test_mixed_bound.py (a few 2^-21 relative to its tiles); a column of B
passes through at most steps x (domain chain + merges) of them, so the
column's error stays below 2^-16 of its norm at these sizes (measured: see
the assertion messages), while FP64 would be 1e-15 and plain TF32 ~1e-3."""
import numpy as np
import pytest
import torch

import oracle
from paper_0709_1272_gb300 import inputs

pytestmark = pytest.mark.gpu

BOUND = 2.0 ** -16


@pytest.fixture(scope="module")
def tq():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    tileqr.load()
    return tileqr


def _col_err(got, exp):
    return float(np.max(np.linalg.norm(got - exp, axis=0) / np.maximum(np.linalg.norm(exp, axis=0), 1e-300)))


def _factor(tq, m, n, ib, h, seed):
    A = inputs.normal_matrix(m, n, seed=seed)
    Ad = tq.to_device_colmajor(A)
    if h:
        f = tq.tileqr_factor_tree(Ad, 128, ib, h, precision=tq.TILEQR_TF32).check()
    else:
        f = tq.tileqr_factor(Ad, 128, ib, precision=tq.TILEQR_TF32).check()
    AV, T = f.factors()
    T2 = f.tree_T().cpu().numpy() if h else None
    ref = oracle.Factored(np.asfortranarray(AV.cpu().numpy()), np.asfortranarray(T.cpu().numpy()), m, n, 128,
                          ib, None if T2 is None else np.asfortranarray(T2), h)
    return f, ref


CASES = [
    # (m, n, ib, domain, nrhs): flat and tree forms, ragged edges, one and
    # several 128-column chunks
    (1000, 700, 16, 0, 5),
    (2000, 384, 32, 3, 130),
    (64 * 23 + 17, 260, 16, 2, 1),
    (384, 1000, 16, 0, 40),
]


@pytest.mark.parametrize("m,n,ib,h,nrhs", CASES)
def test_apply_mixed_matches_oracle(tq, m, n, ib, h, nrhs):
    f, ref = _factor(tq, m, n, ib, h, seed=2100 + m)
    B = inputs.normal_matrix(m, nrhs, seed=2101)
    got = f.apply_mixed(tq.to_device_colmajor(B), trans=True).cpu().numpy()
    e_qt = _col_err(got, oracle.apply_qt(ref, B.copy()))
    got = f.apply_mixed(tq.to_device_colmajor(B), trans=False).cpu().numpy()
    e_q = _col_err(got, oracle.apply_q(ref, B.copy()))
    assert e_qt <= BOUND and e_q <= BOUND, (e_qt, e_q)
    # the FP64 application of the same factors agrees with the oracle to
    # rounding: the mixed error above is the products', not the operands'
    fp = f.apply_qt(tq.to_device_colmajor(B)).cpu().numpy()
    assert _col_err(fp, oracle.apply_qt(ref, B.copy())) <= 1e-12


def test_apply_mixed_column_scaling(tq):
    """Columns of B far outside FP32's range (2^300, 2^-300, 0) keep the
    same relative accuracy: the columns are scaled by powers of two."""
    m, n = 900, 300
    f, ref = _factor(tq, m, n, 16, 0, seed=2200)
    B = inputs.normal_matrix(m, 4, seed=2201)
    B[:, 0] *= 2.0 ** 300
    B[:, 1] *= 2.0 ** -300
    B[:, 2] = 0.0
    for trans, fn in ((True, oracle.apply_qt), (False, oracle.apply_q)):
        got = f.apply_mixed(tq.to_device_colmajor(B), trans=trans).cpu().numpy()
        exp = fn(ref, B.copy())
        assert np.all(np.isfinite(got))
        assert np.all(got[:, 2] == 0.0)
        keep = [0, 1, 3]
        assert _col_err(got[:, keep], exp[:, keep]) <= BOUND


def test_apply_mixed_round_trip_and_errors(tq):
    m, n = 1500, 500
    f, _ = _factor(tq, m, n, 32, 4, seed=2300)
    B = tq.to_device_colmajor(inputs.normal_matrix(m, 7, seed=2301))
    back = f.apply_mixed(f.apply_mixed(B.clone(), trans=True), trans=False)
    assert (torch.linalg.matrix_norm(back - B) / torch.linalg.matrix_norm(B)).item() <= 2 * BOUND
    # no right-hand sides: nothing to do
    f.apply_mixed(tq.colmajor_empty(m, 0), trans=True)
    # an FP64 factorization has no tensor-core operands
    f64 = tq.tileqr_factor(tq.to_device_colmajor(inputs.normal_matrix(300, 200, seed=2302)), 128, 16).check()
    with pytest.raises(tq.TileQRError):
        f64.apply_mixed(tq.to_device_colmajor(inputs.normal_matrix(300, 2, seed=2303)))
