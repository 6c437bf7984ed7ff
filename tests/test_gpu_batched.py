"""Batched form: many ragged matrices in one persistent launch
(tileqr_batched_prepare / tileqr_factor_batched), FP64 and mixed.

Checks: every matrix of the batch matches the CPU oracle (FP64: 1e-12
relative, R sign-normalised, V and T directly) and is bit-identical to the
single-matrix entry point on the same matrix (same deterministic task
kernels); a CUDA-graph replay of the batched launch reproduces the bits."""
import numpy as np
import pytest
import torch

import oracle
from paper_0709_1272_gb300 import inputs

EPS = np.finfo(np.float64).eps

pytestmark = pytest.mark.gpu
TOL = 1e-12


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


def _batch(count, seed, m_hi=700):
    shapes = inputs.batch_shapes(count, seed, m_lo=64, m_hi=m_hi, n_lo=32)
    shapes += [(64, 32), (1, 1), (129, 129), (5, 200)]     # tiny, one-element, ragged, wide
    pool, offs = inputs.batch_pool(shapes, seed)
    return shapes, pool, offs


def _to_dev(tq, shapes, pool, offs):
    return [tq.to_device_colmajor(pool[o:o + m * n].reshape(n, m).T) for (m, n), o in zip(shapes, offs)]


@pytest.mark.parametrize("nb,ib", [(64, 16), (128, 32), (256, 16)])
def test_batched_fp64_matches_oracle_and_single(tq, nb, ib):
    shapes, pool, offs = _batch(24, seed=900 + nb)
    mats = _to_dev(tq, shapes, pool, offs)
    bt = tq.Batch(mats, nb, ib)
    bt.run()
    assert bt.status() == 0
    for b, ((m, n), o) in enumerate(zip(shapes, offs)):
        A = pool[o:o + m * n].reshape(n, m).T
        AV, T = bt.get(b).factors()
        AV, T = AV.cpu().numpy(), T.cpu().numpy()
        ref = oracle.tiled_qr(A, nb, ib)
        assert _rel(AV, ref.A) <= TOL and _rel(T, ref.T) <= TOL, (b, m, n)
        if b % 5 == 0:
            s = tq.tileqr_factor(mats[b], nb, ib).check()
            AVs, Ts = s.factors()
            assert np.array_equal(AV, AVs.cpu().numpy()) and np.array_equal(T, Ts.cpu().numpy())


def test_batched_mixed_matches_single(tq):
    shapes, pool, offs = _batch(20, seed=77, m_hi=900)
    mats = _to_dev(tq, shapes, pool, offs)
    bt = tq.Batch(mats, 128, 16, precision=tq.TILEQR_TF32)
    bt.run()
    assert bt.status() == 0
    for b in range(0, len(shapes), 3):
        (m, n), o = shapes[b], offs[b]
        AV, T = bt.get(b).factors()
        s = tq.tileqr_factor(mats[b], 128, 16, precision=tq.TILEQR_TF32).check()
        AVs, Ts = s.factors()
        assert np.array_equal(AV.cpu().numpy(), AVs.cpu().numpy())
        A = pool[o:o + m * n].reshape(n, m).T
        R = bt.get(b).R().cpu().numpy()
        ref = oracle.tiled_qr(A, 128, 16)
        assert _rel(oracle.sign_normalize(R), oracle.sign_normalize(ref.R())) <= 1e-4


def test_batched_cuda_graph_replay(tq):
    shapes, pool, offs = _batch(30, seed=5)
    mats = _to_dev(tq, shapes, pool, offs)
    bt = tq.Batch(mats, 128, 16)
    bt.run()                       # first call outside capture (kernel attributes)
    assert bt.status() == 0
    ref = [bt.get(b).factors()[0].cpu().numpy() for b in range(len(shapes))]
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            bt.run(stream=s)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        assert bt.status() == 0
        for b in range(len(shapes)):
            assert np.array_equal(bt.get(b).factors()[0].cpu().numpy(), ref[b])


@pytest.mark.parametrize("prec_name,nb,ib", [("TILEQR_FP64", 64, 16), ("TILEQR_TF32", 128, 16)])
def test_full_batch_4096(tq, prec_name, nb, ib):
    """The benchmarked batch at full size: 4096 matrices, m ~ U[64, 2048],
    n ~ U[32, m], entries U[-1, 1) (the benchmark's seed), with the (nb, ib)
    the autotuner picks for it (FP64 64/16, TF32 128/16).  Every matrix
    finishes; sampled matrices are bit-identical to the single-matrix entry
    point; in FP64 the smallest sampled ones also match the oracle."""
    prec = getattr(tq, prec_name)
    seed = 20070709 + 5
    shapes = inputs.batch_shapes(4096, seed=seed)
    pool, offs = inputs.batch_pool(shapes, seed=seed)
    pool_d = torch.from_numpy(pool).to("cuda")
    mats = [pool_d[o:o + m * n].view(n, m).t() for (m, n), o in zip(shapes, offs)]
    bt = tq.Batch(mats, nb, ib, prec)
    bt.run()
    assert bt.status() == 0
    rng = np.random.Generator(np.random.Philox(key=77))
    sample = sorted(set(rng.integers(0, len(shapes), 10).tolist()) | {int(np.argmin([m * n for m, n in shapes]))})
    for b in sample:
        m, n = shapes[b]
        AV, T = bt.get(b).factors()
        s = tq.tileqr_factor(mats[b], nb, ib, precision=prec).check()
        AVs, Ts = s.factors()
        assert np.array_equal(AV.cpu().numpy(), AVs.cpu().numpy())
        assert np.array_equal(T.cpu().numpy(), Ts.cpu().numpy())
        if prec == tq.TILEQR_FP64 and m * n <= 400 * 400:
            A = pool[offs[b]:offs[b] + m * n].reshape(n, m).T
            ref = oracle.tiled_qr(A, nb, ib)
            assert _rel(AV.cpu().numpy(), ref.A) <= TOL
    del bt, mats, pool_d
    torch.cuda.empty_cache()


def test_batched_solve_matches_oracle_on_ragged_sub_batch(tq):
    """tileqr_batched_solve_ls on a ragged batch (FP64 and TF32 factors,
    inconsistent right-hand sides): each x agrees with the oracle's
    least-squares solution (Algorithm 2 + Q^T b + R^-1) to the accuracy the
    problem's conditioning allows two FP64 solvers, 100 eps kappa (1 + kappa
    ||r|| / (||A|| ||x||)), and each residual is orthogonal to range(A); one
    step on FP64 factors is the plain solve."""
    shapes = [(300, 200), (129, 129), (700, 64), (64, 33), (1000, 999), (513, 260), (257, 256), (90, 90)]
    mats = [inputs.uniform_matrix(m, n, seed=400 + b) for b, (m, n) in enumerate(shapes)]
    rhs = [inputs.normal_matrix(m, 1, seed=500 + b).reshape(-1) for b, (m, n) in enumerate(shapes)]
    dmats = [tq.to_device_colmajor(A) for A in mats]
    drhs = [torch.from_numpy(b).cuda() for b in rhs]
    refs = []
    for A, b in zip(mats, rhs):
        refs.append(oracle.solve_ls(oracle.tiled_qr(A, 128, 16), b.copy()).reshape(-1))
    for prec, steps in ((tq.TILEQR_FP64, 1), (tq.TILEQR_FP64, 8), (tq.TILEQR_TF32, 8)):
        bt = tq.Batch(dmats, 128, 16, prec)
        bt.run()
        assert bt.status() == 0
        xs, info = bt.solve_ls(drhs, max_iter=steps, tol=1e-14)
        assert info.converged == 1 or steps == 1
        for A, b, x, xo in zip(mats, rhs, xs, refs):
            x = x.cpu().numpy()
            r = b - A @ x
            kappa = np.linalg.cond(A)
            tol = 100 * EPS * kappa * (1 + kappa * np.linalg.norm(r) / (np.linalg.norm(A, 2) * np.linalg.norm(x)))
            assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= tol, (prec, steps)
            if A.shape[0] > A.shape[1]:   # inconsistent: the residual is orthogonal to range(A)
                assert np.linalg.norm(A.T @ r) / (np.linalg.norm(A) * np.linalg.norm(r)) <= 20 * A.shape[1] * EPS
            else:                          # square: normwise backward error of the solve
                assert np.linalg.norm(r) / (np.linalg.norm(A) * np.linalg.norm(x)) <= 20 * A.shape[1] * EPS
