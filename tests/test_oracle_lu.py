"""Pins of the tiled LU oracle (Sec. 3.2.2, Algorithm 3: DGETRF, DGESSM,
DTSTRF, DSSSSM with tiled pairwise pivoting, inner blocking s) against what
the mathematics fixes: with one tile the method is GEPP (identical pivots and
factors to LAPACK's), N U = A (the reconstruction of Sec. 3.2.4), solves
reach rounding-level backward error, every multiplier is at most 1 in
magnitude (each pivot is the largest of its candidates), any dependency-
respecting order gives the same bits, the flop count is n^2(n - n/3)(1 +
s/(2b)) to leading order, and a plausible pivoting mistake fails."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_0709_1272_gb300 import inputs

EPS = np.finfo(np.float64).eps


def test_one_tile_is_gepp():
    n = 256
    A = inputs.normal_matrix(n, n, seed=1)
    f = oracle.tiled_lu(A, n, 16)
    lu, pv = scipy.linalg.lu_factor(A)
    assert np.array_equal(f.piv[0], pv)
    assert np.abs(np.triu(f.A) - np.triu(lu)).max() <= 50 * n * EPS * np.abs(np.triu(lu)).max()
    assert np.abs(np.tril(f.A, -1) - np.tril(lu, -1)).max() <= 50 * n * EPS


@pytest.mark.parametrize("n,nb,ib", [(256, 64, 16), (256, 32, 8), (384, 128, 32), (192, 64, 64), (64, 16, 4)])
def test_reconstruction_and_solve(n, nb, ib):
    A = inputs.normal_matrix(n, n, seed=n + nb)
    f = oracle.tiled_lu(A, nb, ib)
    assert f.info == 0
    st = oracle.lu_stability(A, f, inputs.normal_matrix(n, 2, seed=5))
    assert st["fact_backward"] <= 1e3 * n * EPS
    assert st["solve_backward"] <= 20 * n * EPS
    xt = inputs.normal_matrix(n, 1, seed=6)
    x = f.solve(A @ xt)
    assert np.abs(x - xt).max() <= 1e-9


@pytest.mark.parametrize("nb,ib", [(64, 16), (32, 32)])
def test_multipliers_bounded_by_one(nb, ib):
    n = 256
    A = inputs.uniform_matrix(n, n, seed=9)
    f = oracle.tiled_lu(A, nb, ib)
    p = n // nb
    for k in range(p):
        Lkk = np.tril(f.A[k * nb:(k + 1) * nb, k * nb:(k + 1) * nb], -1)
        assert np.abs(Lkk).max() <= 1.0
        for i in range(k + 1, p):
            assert np.abs(f.A[i * nb:(i + 1) * nb, k * nb:(k + 1) * nb]).max() <= 1.0
            assert np.abs(f.Lx[i * ib:(i + 1) * ib, k * nb:(k + 1) * nb]).max() <= 1.0


def test_planted_pivoting_mistake_is_caught():
    A = inputs.uniform_matrix(256, 256, seed=10)
    try:
        oracle.lu_set_mutation(1)   # DTSTRF never keeps the pivot row of U
        f = oracle.tiled_lu(A, 64, 16)
    finally:
        oracle.lu_set_mutation(0)
    big = max(np.abs(f.A[64:, :64]).max(), np.abs(f.Lx).max())
    assert big > 1.0


@pytest.mark.parametrize("seed", [1, 2])
def test_any_topological_order_same_bits(seed):
    n, nb, ib = 320, 64, 16
    A = inputs.normal_matrix(n, n, seed=20)
    ref = oracle.tiled_lu(A, nb, ib)
    order = oracle.lu_random_order(n, nb, np.random.Generator(np.random.Philox(key=seed)))
    f = oracle.tiled_lu_ordered(A, nb, ib, order)
    assert np.array_equal(f.A, ref.A) and np.array_equal(f.Lx, ref.Lx) and np.array_equal(f.piv, ref.piv)


def test_flop_count():
    n, nb, ib = 512, 64, 16
    oracle.lu_reset_flops()
    oracle.tiled_lu(inputs.normal_matrix(n, n, seed=11), nb, ib)
    model = n * n * (n - n / 3.0) * (1 + ib / (2.0 * nb))
    assert abs(oracle.lu_flops() - model) <= 0.05 * model


def test_zero_pivot_reported():
    n = 256
    A = inputs.normal_matrix(n, n, seed=12)
    A[:, 100] = 0.0
    f = oracle.tiled_lu(A, 64, 16)
    assert f.info == 101


def test_stability_decreases_with_more_tiles():
    # Sec. 3.2.4: the growth of N increases with the number of tiles
    n = 256
    A = inputs.normal_matrix(n, n, seed=13)
    s1 = oracle.lu_stability(A, oracle.tiled_lu(A, 256, 16))
    s8 = oracle.lu_stability(A, oracle.tiled_lu(A, 32, 16))
    assert s8["norm_N"] > s1["norm_N"]
