"""Pins of the oracle's least-squares refinement on the augmented system
(Bjorck's method; an addition to the paper) on the CPU: exact factors give
the FP64 solution at once, and factors of a perturbed matrix (errors of the
size a TF32 factorization leaves) are refined to the FP64 least-squares
solution of an inconsistent system, where refining x alone stalls."""
import numpy as np
import scipy.linalg

import oracle
from paper_0709_1272_gb300 import inputs

EPS = np.finfo(np.float64).eps


def _tall_problem(m, n, kappa, resid, seed):
    """A = U diag(s) V^T with s geometric from 1 to 1/kappa, and b = A x_t + e
    with e orthogonal to range(A), ||e|| = resid ||A x_t||."""
    U = np.linalg.qr(inputs.normal_matrix(m, n, seed=seed))[0]
    V = np.linalg.qr(inputs.normal_matrix(n, n, seed=seed + 1))[0]
    s = kappa ** (-np.arange(n) / (n - 1))
    A = np.asfortranarray((U * s) @ V.T)
    xt = inputs.normal_matrix(n, 1, seed=seed + 2).reshape(-1)
    y = A @ xt
    e = inputs.normal_matrix(m, 1, seed=seed + 3).reshape(-1)
    e -= U @ (U.T @ e)
    e *= resid * np.linalg.norm(y) / np.linalg.norm(e)
    return A, y + e


def _x_only(f, A, b, steps):
    x = oracle.solve_ls(f, b.copy()).reshape(-1)
    for _ in range(steps):
        x = x + oracle.solve_ls(f, (b - A @ x).copy()).reshape(-1)
    return x


def test_exact_factors_give_the_least_squares_solution():
    A, b = _tall_problem(160, 48, 1e3, 1.0, seed=71)
    f = oracle.tiled_qr(A, 16, 4)
    x, r, steps = oracle.refine_ls_augmented(f, A, b)
    xl = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(x - xl) <= 20 * 48 * EPS * 1e3 * np.linalg.norm(xl)
    assert np.linalg.norm(r - (b - A @ x)) <= 1e-13 * np.linalg.norm(b)
    assert steps <= 3


def test_perturbed_factors_are_refined_to_fp64_accuracy():
    m, n, kappa = 200, 64, 1e4
    A, b = _tall_problem(m, n, kappa, 10.0, seed=81)
    # factors of A + E with ||E|| ~ 1e-7 ||A||: the error a TF32 factorization leaves
    E = inputs.normal_matrix(m, n, seed=91) * (1e-7 * np.linalg.norm(A, 2) / np.sqrt(m))
    f = oracle.tiled_qr(np.asfortranarray(A + E), 16, 4)
    xl = np.linalg.lstsq(A, b, rcond=None)[0]
    x, r, steps = oracle.refine_ls_augmented(f, A, b, max_iter=40)
    err = np.linalg.norm(x - xl) / np.linalg.norm(xl)
    assert err <= 1e3 * n * EPS * kappa       # FP64 accuracy for this kappa
    # the normal equations hold to rounding: A^T r ~ 0
    assert np.linalg.norm(A.T @ (b - A @ x)) <= 1e-12 * np.linalg.norm(A, 2) * np.linalg.norm(b)
    # refining x alone stalls well above that on this inconsistent system
    x1 = _x_only(f, A, b, 40)
    assert np.linalg.norm(x1 - xl) / np.linalg.norm(xl) >= 100 * err


def test_consistent_system_matches_the_true_solution():
    A, b = _tall_problem(120, 40, 1e2, 0.0, seed=101)
    f = oracle.tiled_qr(A, 8, 4)
    x, r, _ = oracle.refine_ls_augmented(f, A, b)
    xl = scipy.linalg.lstsq(A, b)[0]
    assert np.linalg.norm(x - xl) <= 1e-12 * np.linalg.norm(xl)
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(b)
