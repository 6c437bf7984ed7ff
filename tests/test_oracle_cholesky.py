"""Pins of the tiled Cholesky oracle (Sec. 3.1, Algorithm 1: DPOTF2, DTRSM,
DGSMM) against what the mathematics fixes: the Cholesky factor of an SPD
matrix is unique, so it must equal LAPACK's (a library routine, the special
case nb >= n included); L L^T reproduces A; a 2 x 2 closed form; a matrix
that is not positive definite is reported at the right column; any order
respecting the dependencies gives the same bits; the flop count is n^3/3 to
leading order; a plausible mistake (transposed triangle in DTRSM) fails."""
import numpy as np
import pytest

import oracle
from paper_0709_1272_gb300 import inputs

EPS = np.finfo(np.float64).eps


@pytest.mark.parametrize("n,nb", [(500, 64), (512, 128), (257, 64), (64, 64), (100, 256), (1, 64)])
def test_factor_equals_lapack_and_reproduces_A(n, nb):
    A = inputs.spd_matrix(n, seed=n + nb)
    L, info = oracle.tiled_cholesky(A, nb)
    assert info == 0
    assert np.array_equal(L, np.tril(L))
    assert np.all(np.diag(L) > 0)
    assert np.abs(L @ L.T - A).max() <= 10 * n * EPS * np.abs(A).max()
    Lref = np.linalg.cholesky(A)
    assert np.abs(L - Lref).max() <= 10 * n * EPS * np.abs(Lref).max()


def test_closed_form_2x2():
    a, b, d = 4.0, 2.0, 5.0
    L, info = oracle.tiled_cholesky(np.array([[a, b], [b, d]], order="F"), 64)
    assert info == 0
    assert L[0, 0] == 2.0 and L[1, 0] == 1.0 and L[1, 1] == 2.0 and L[0, 1] == 0.0


def test_not_positive_definite_reports_the_column():
    n = 300
    A = inputs.spd_matrix(n, seed=5)
    A[170, 170] = -1.0   # a negative diagonal entry: the leading 171 x 171 minor is not PD
    _, info = oracle.tiled_cholesky(A, 64)
    assert 1 <= info <= 171
    # an exactly singular leading minor: a zero row / column
    B = inputs.spd_matrix(n, seed=6)
    B[80, :] = 0.0
    B[:, 80] = 0.0
    _, info = oracle.tiled_cholesky(B, 64)
    assert info == 81


def test_upper_triangle_is_never_referenced():
    A = inputs.spd_matrix(300, seed=8)
    B = A.copy(order="F")
    B[np.triu_indices(300, 1)] = np.nan
    L1, _ = oracle.tiled_cholesky(A, 64)
    L2, info = oracle.tiled_cholesky(B, 64)
    assert info == 0
    assert np.array_equal(L1, L2)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_any_topological_order_same_bits(seed):
    n, nb = 520, 64
    A = inputs.spd_matrix(n, seed=40)
    ref, _ = oracle.tiled_cholesky(A, nb)
    order = oracle.cholesky_random_order(n, nb, np.random.Generator(np.random.Philox(key=seed)))
    L, info = oracle.tiled_cholesky_ordered(A, nb, order)
    assert info == 0
    assert np.array_equal(L, ref)


def test_flop_count():
    n = 640
    oracle.cholesky_reset_flops()
    oracle.tiled_cholesky(inputs.spd_matrix(n, seed=9), 64)
    f = oracle.cholesky_flops()
    assert abs(f - n ** 3 / 3.0) <= 0.02 * n ** 3 / 3.0


def test_planted_transpose_mistake_is_caught():
    A = inputs.spd_matrix(300, seed=11)
    try:
        oracle.cholesky_set_mutation(1)
        L, _ = oracle.tiled_cholesky(A, 64)
    finally:
        oracle.cholesky_set_mutation(0)
    assert np.abs(L @ L.T - A).max() > 1e-6 * np.abs(A).max()
