"""The seeded input generators (no factorization arithmetic): determinism and
the equivalence of the threaded batch pool with per-matrix generation."""
import numpy as np

from paper_0709_1272_gb300 import inputs


def test_batch_pool_equals_per_matrix_draws():
    shapes = inputs.batch_shapes(9, seed=3)
    pool, offs = inputs.batch_pool(shapes, seed=3, threads=4)
    mats = inputs.batch_matrices(shapes, seed=3)
    for (m, n), o, M in zip(shapes, offs, mats):
        assert np.array_equal(pool[o:o + m * n].reshape(n, m).T, M)


def test_batch_shapes_distribution():
    shapes = inputs.batch_shapes(4096, seed=20070714)
    ms = np.array([s[0] for s in shapes])
    ns = np.array([s[1] for s in shapes])
    assert ms.min() >= 64 and ms.max() <= 2048 and np.all(ns >= 32) and np.all(ns <= ms)
    assert abs(ms.mean() - (64 + 2048) / 2) < 40


def test_generators_are_deterministic():
    assert np.array_equal(inputs.normal_matrix(7, 5, 1), inputs.normal_matrix(7, 5, 1))
    assert not np.array_equal(inputs.normal_matrix(7, 5, 1), inputs.normal_matrix(7, 5, 2))
    a = inputs.uniform_matrix(100, 50, 4)
    assert a.flags.f_contiguous and a.min() >= -1 and a.max() < 1


def test_kappa_columns_and_factors_match_the_full_matrix():
    A, s, u, v = inputs.kappa_matrix(300, 1e6, seed=5)
    s2, u2, v2 = inputs.kappa_factors(300, 1e6, seed=5)
    assert np.array_equal(s, s2) and np.array_equal(u, u2) and np.array_equal(v, v2)
    assert np.allclose(inputs.kappa_columns(300, 1e6, 5, 17, 140), A[:, 17:140], rtol=0, atol=1e-15)
    # singular values exactly s: cond_2 = kappa
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(sv, s, rtol=1e-10, atol=1e-14)
