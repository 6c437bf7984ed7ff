"""Mixed-precision factorization + FP64 iterative refinement of the solve
(tileqr_solve_refine) on the prescribed-singular-value matrices
A = (I - 2uu^T) diag(s) (I - 2vv^T), s geometric from 1 to 1/kappa, with a
consistent right-hand side b = A x_true.

Bar: relative residual ||b - A x|| / ||b|| <= 1e-12, measured here in FP64
on the host, and the solution agrees with the FP64 oracle's tiled-QR solve to
within the forward error the conditioning allows (kappa * 1e-12)."""
import numpy as np
import pytest
import torch

import oracle
from paper_0709_1272_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tq():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    tileqr.load()
    return tileqr


def _solve(tq, A, b, precision):
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor(Ad, 128, 16, precision=precision).check()
    x, info = f.solve_refine(Ad, torch.from_numpy(b).cuda(), max_iter=40, tol=1e-12)
    return x.cpu().numpy(), info


@pytest.mark.parametrize("n,kappa", [(1024, 1e2), (1024, 1e6), (1024, 1e10), (1000, 1e6), (2560, 1e10)])
def test_refined_solve_reaches_fp64_accuracy(tq, n, kappa):
    A, s, u, v = inputs.kappa_matrix(n, kappa, seed=11 + n)
    xt = inputs.normal_matrix(n, 1, seed=12).reshape(-1)
    b = A @ xt
    x, info = _solve(tq, A, b, tq.TILEQR_TF32)
    relres = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert info.converged == 1 and relres <= 1e-12, (info.as_dict(), relres)
    # the factors alone are only FP32-accurate: refinement did real work
    assert info.initial_rel_residual > 1e-9
    if n <= 1024:
        ref = oracle.tiled_qr(A, 128, 16)
        xo = oracle.solve_ls(ref, b).reshape(-1)
        assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= max(kappa * 1e-12, 1e-12)


def test_refine_on_fp64_factors_converges_at_once(tq):
    n = 768
    A, _, _, _ = inputs.kappa_matrix(n, 1e6, seed=3)
    b = A @ inputs.normal_matrix(n, 1, seed=4).reshape(-1)
    x, info = _solve(tq, A, b, tq.TILEQR_FP64)
    assert info.converged == 1 and info.iterations <= 2


def test_refine_full_size_16384(tq):
    """16384 x 16384, kappa 1e6: the conditioning workload at full size."""
    n, kappa = 16384, 1e6
    A, _, _, _ = inputs.kappa_matrix(n, kappa, seed=20070714)
    xt = inputs.normal_matrix(n, 1, seed=20070715).reshape(-1)
    b = A @ xt
    x, info = _solve(tq, A, b, tq.TILEQR_TF32)
    relres = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert info.converged == 1 and relres <= 1e-12, (info.as_dict(), relres)
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= kappa * 1e-12


@pytest.mark.parametrize("m,n,h", [(8192, 512, 4), (16384, 384, 8), (4096, 512, 0)])
def test_refine_tall_tree_mixed(tq, m, n, h):
    """Tall A with TF32 updates, tree form (domain h; 0 = Algorithm 2's flat
    tree) and a consistent right-hand side b = A x_true: the FP32 correction
    solve replays the tree's apply graph (DLARFB, DSSRFB, DTTMQR) and the
    refinement reaches the FP64 bar."""
    A = inputs.normal_matrix(m, n, seed=40 + h)
    xt = inputs.normal_matrix(n, 1, seed=41).reshape(-1)
    b = A @ xt
    Ad = tq.to_device_colmajor(A)
    f = (tq.tileqr_factor_tree(Ad, 128, 16, h, precision=tq.TILEQR_TF32) if h
         else tq.tileqr_factor(Ad, 128, 16, precision=tq.TILEQR_TF32)).check()
    x, info = f.solve_refine(Ad, torch.from_numpy(b).cuda(), max_iter=40, tol=1e-12)
    x = x.cpu().numpy()
    relres = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert info.converged == 1 and relres <= 1e-12, (info.as_dict(), relres)
    assert info.initial_rel_residual > 1e-9
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= 1e-11


@pytest.mark.parametrize("scale_exp", [500, -530])
def test_refined_solve_extreme_magnitudes(tq, scale_exp):
    """A and b scaled by 2^500 (~3e150) or 2^-530 (~3e-160): the FP32
    correction solve works on power-of-two scaled quantities, so the refined
    solve reaches the same accuracy as unscaled (x is scale-free here)."""
    n = 1024
    A, _, _, _ = inputs.kappa_matrix(n, 1e6, seed=21)
    xt = inputs.normal_matrix(n, 1, seed=22).reshape(-1)
    As = np.ldexp(A, scale_exp)
    b = As @ xt
    x, info = _solve(tq, As, b, tq.TILEQR_TF32)
    assert np.all(np.isfinite(x))
    # the residual at unit scale (exact rescaling; the norms of ~1e-160
    # vectors would underflow)
    relres = np.linalg.norm(np.ldexp(b - As @ x, -scale_exp)) / np.linalg.norm(np.ldexp(b, -scale_exp))
    assert info.converged == 1 and relres <= 1e-12, (info.as_dict(), relres)
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= 1e6 * 1e-12
