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
