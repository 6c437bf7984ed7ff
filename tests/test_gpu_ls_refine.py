"""Least squares for inconsistent (tall) systems refined to FP64 accuracy on
the augmented system (tileqr_solve_ls_refine, Bjorck's method; the oracle of
the method is oracle.refine_ls_augmented, pinned in test_oracle_refine.py).

Bar: on a TF32 factorization (flat and tree form) the refined X agrees with
the FP64 oracle's least-squares solution (Algorithm 2 + Q^T B + R^{-1}) to
1e-10 relative, and every residual is orthogonal to range(A) to FP64
rounding, ||A^T r|| / (||A|| ||r||) <= 20 n eps -- while the TF32 factors
alone give errors of ~1e-6."""
import numpy as np
import pytest
import torch

import oracle
from paper_0709_1272_gb300 import inputs

pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def tq():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    tileqr.load()
    return tileqr


def _tall_problem(m, n, nrhs, kappa, resid, seed):
    """A = U diag(s) V^T, s geometric 1 .. 1/kappa; B = A X_t + E with the
    columns of E orthogonal to range(A), ||e_k|| = resid ||A x_k||."""
    U = np.linalg.qr(inputs.normal_matrix(m, n, seed=seed))[0]
    V = np.linalg.qr(inputs.normal_matrix(n, n, seed=seed + 1))[0]
    s = kappa ** (-np.arange(n) / max(n - 1, 1))
    A = np.asfortranarray((U * s) @ V.T)
    Xt = inputs.normal_matrix(n, nrhs, seed=seed + 2)
    Y = A @ Xt
    E = inputs.normal_matrix(m, nrhs, seed=seed + 3)
    E -= U @ (U.T @ E)
    E *= resid * np.linalg.norm(Y, axis=0) / np.linalg.norm(E, axis=0)
    return A, np.asfortranarray(Y + E)


def _optimality(A, R):
    return float(np.max(np.linalg.norm(A.T @ R, axis=0) / (np.linalg.norm(A) * np.linalg.norm(R, axis=0))))


@pytest.mark.parametrize("domain", [0, 4])
def test_refined_ls_matches_fp64_oracle(tq, domain):
    m, n, nrhs = 4096, 384, 16
    A, B = _tall_problem(m, n, nrhs, 1e2, 10.0, seed=81)
    Ad, Bd = tq.to_device_colmajor(A), tq.to_device_colmajor(B)
    f = tq.tileqr_factor_tree(Ad, 128, 16, domain, precision=tq.TILEQR_TF32).check()
    X, Rres, info = f.solve_ls_refine(Ad, Bd, max_iter=10, tol=1e-14, residual=True)
    X, Rres = X.cpu().numpy(), Rres.cpu().numpy()
    ref = oracle.tiled_qr(A, 128, 16)
    Xo = oracle.solve_ls(ref, B.copy())
    err = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    assert info.converged == 1 and err <= 1e-10, (info.as_dict(), err)
    # the TF32 factors alone are far from FP64 accuracy: refinement did work
    assert info.initial_rel_residual > 1e-9
    assert _optimality(A, B - A @ X) <= 20 * n * EPS
    # the residual returned is b - A x
    assert np.linalg.norm(Rres - (B - A @ X)) <= 1e-12 * np.linalg.norm(B)


def test_refined_ls_on_fp64_factors_stops_at_once(tq):
    m, n, nrhs = 2000, 300, 3
    A, B = _tall_problem(m, n, nrhs, 1e3, 1.0, seed=91)
    Ad, Bd = tq.to_device_colmajor(A), tq.to_device_colmajor(B)
    f = tq.tileqr_factor(Ad, 64, 16).check()
    X, info = f.solve_ls_refine(Ad, Bd, max_iter=10, tol=1e-14)
    assert info.converged == 1 and info.iterations <= 3
    Xo = oracle.solve_ls(oracle.tiled_qr(A, 64, 16), B.copy())
    # two FP64 least-squares solutions differ by up to ~eps kappa^2 ||r|| /
    # (||A|| ||x||) ~ 1e-10 here (kappa 1e3, residual as large as A x)
    assert np.linalg.norm(X.cpu().numpy() - Xo) / np.linalg.norm(Xo) <= 1e-9


def test_refined_ls_consistent_system(tq):
    """b in range(A): the residual goes to rounding level and x to x_t."""
    m, n = 1500, 260
    A, B = _tall_problem(m, n, 2, 1e2, 0.0, seed=95)
    Ad, Bd = tq.to_device_colmajor(A), tq.to_device_colmajor(B)
    f = tq.tileqr_factor(Ad, 128, 32, precision=tq.TILEQR_TF32).check()
    X, info = f.solve_ls_refine(Ad, Bd, max_iter=10, tol=1e-14)
    X = X.cpu().numpy()
    assert np.linalg.norm(B - A @ X) / np.linalg.norm(B) <= 20 * n * EPS
    assert info.converged == 1


def test_full_tall_skinny_16_rhs(tq):
    """262144 x 512 N(0,1), 16 N(0,1) right-hand sides (inconsistent), TF32
    tree form (domains of 16 tile rows) as the benchmark times it; against
    the FP64 oracle's least-squares solution."""
    m, n, nrhs = 262144, 512, 16
    A = inputs.normal_matrix(m, n, seed=20070709 + 3)
    B = inputs.normal_matrix(m, nrhs, seed=20070709 + 6)
    Ad, Bd = tq.to_device_colmajor(A), tq.to_device_colmajor(B)
    f = tq.tileqr_factor_tree(Ad, 128, 16, 16, precision=tq.TILEQR_TF32).check()
    X, info = f.solve_ls_refine(Ad, Bd, max_iter=10, tol=1e-14)
    X = X.cpu().numpy()
    import os
    threads = len(os.sched_getaffinity(0))
    ref, _ = oracle.tiled_qr_levels(A, 128, 16, threads)
    Xo = oracle.solve_ls(ref, B.copy())
    err = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    assert info.converged == 1 and err <= 1e-10, (info.as_dict(), err)
    assert _optimality(A, B - A @ X) <= 20 * n * EPS


def test_refined_ls_many_rhs(tq):
    """More right-hand sides than one 128-column chunk of the tensor-core
    application (two chunks, the second partial), flat TF32 factors."""
    m, n, nrhs = 2000, 300, 130
    A, B = _tall_problem(m, n, nrhs, 1e2, 1.0, seed=97)
    Ad, Bd = tq.to_device_colmajor(A), tq.to_device_colmajor(B)
    f = tq.tileqr_factor(Ad, 128, 16, precision=tq.TILEQR_TF32).check()
    X, info = f.solve_ls_refine(Ad, Bd, max_iter=10, tol=1e-14)
    X = X.cpu().numpy()
    Xo = oracle.solve_ls(oracle.tiled_qr(A, 128, 16), B.copy())
    err = np.linalg.norm(X - Xo) / np.linalg.norm(Xo)
    assert info.converged == 1 and err <= 1e-10, (info.as_dict(), err)
    assert _optimality(A, B - A @ X) <= 20 * n * EPS
