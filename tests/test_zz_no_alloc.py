"""tileqr_factor_noalloc, the factorization entry point for callers that
cannot allocate device memory (services that reserve their whole memory
budget at start-up, plug-ins whose host framework owns every allocation).
They pass only the input matrix and the output buffers; the scheduler's
scratch lives in a fixed array inside the library.

Checked here through the C ABI:
- calls in a row on different tile grids, where a later call needs more
  scratch than, or a different layout from, the one the previous call left
  behind (and the same sequence reversed), give the same tiles and T factors
  as tileqr_factor and as the CPU oracle's Algorithm 2, within the 1e-12
  tolerance of the other parity tests;
- the calls allocate no device memory: neither torch's allocator nor the
  device's free memory changes across them;
- a problem too large for the fixed scratch is refused up front.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_0709_1272_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12
GRANULE = 2 << 20   # the device allocator's page: any cudaMalloc takes at least this much


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


def _buffers(Ad, nb, ib):
    m, n = Ad.shape
    p, q = -(-m // nb), -(-n // nb)
    tiles = torch.empty(p * q * nb * nb, dtype=torch.float64, device=Ad.device)
    T = torch.empty(p * q * ib * nb, dtype=torch.float64, device=Ad.device)
    return tiles, T


def _call(tq, Ad, nb, ib, tiles, T):
    """One call of tileqr_factor_noalloc into caller-owned buffers; returns
    the descriptor after the device-side status was read."""
    lib = tq.load()
    m, n = Ad.shape
    d = tq.tileqr_desc()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.tileqr_factor_noalloc(m, n, ctypes.c_void_p(Ad.data_ptr()), Ad.stride(1), nb, ib,
                                   ctypes.c_void_p(tiles.data_ptr()), tiles.numel() * 8,
                                   ctypes.c_void_p(T.data_ptr()), T.numel() * 8, stream, ctypes.byref(d))
    assert rc == 0, tq.strerror(rc)
    assert lib.tileqr_status(ctypes.byref(d), stream) == 0
    return d


def _run_sequence(tq, cases):
    """Calls in the given order with every buffer made beforehand; checks the
    calls themselves allocate nothing, then returns the factors of each."""
    mats = [tq.to_device_colmajor(inputs.normal_matrix(m, n, seed)) for (m, n, _, _, seed) in cases]
    bufs = [_buffers(Ad, nb, ib) for Ad, (_, _, nb, ib, _) in zip(mats, cases)]
    # the first call on a device looks up the scratch address (and may load
    # the library's module): made outside the measured sequence
    Ad0, (_, _, nb0, ib0, _) = mats[0], cases[0]
    _call(tq, Ad0, nb0, ib0, *_buffers(Ad0, nb0, ib0))
    torch.cuda.synchronize()
    stats0 = torch.cuda.memory_stats()
    free0, _ = torch.cuda.mem_get_info()
    descs = [_call(tq, Ad, nb, ib, tiles, T) for Ad, (_, _, nb, ib, _), (tiles, T) in zip(mats, cases, bufs)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert stats1.get("allocation.all.allocated", 0) == stats0.get("allocation.all.allocated", 0)
    assert stats1.get("allocated_bytes.all.current", 0) == stats0.get("allocated_bytes.all.current", 0)
    assert free1 > free0 - GRANULE, (free0, free1)
    out = []
    for d, (tiles, T), Ad in zip(descs, bufs, mats):
        f = tq.Factorization(d, tiles, Ad.device)   # keeps the output buffers alive
        AV, Tcm = f.factors()
        torch.cuda.synchronize()
        out.append((AV.cpu().numpy(), Tcm.cpu().numpy()))
    return mats, out


def _check_against_factor_and_oracle(tq, mats, cases, got):
    for Ad, (m, n, nb, ib, seed), (AV, T) in zip(mats, cases, got):
        ref = tq.tileqr_factor(Ad, nb, ib).check()
        AVr, Tr = ref.factors()
        torch.cuda.synchronize()
        assert _rel(AV, AVr.cpu().numpy()) <= TOL
        assert _rel(T, Tr.cpu().numpy()) <= TOL
        o = oracle.tiled_qr(inputs.normal_matrix(m, n, seed), nb, ib)
        assert _rel(AV, o.A) <= TOL
        assert _rel(T, o.T[:T.shape[0], :]) <= TOL


# (m, n, nb, ib, seed): tile grids 8 x 6 at nb 128, then 8 x 8 at nb 64 (more
# tasks, so more scratch and other queue offsets), then 11 x 8 at nb 128
GROWING = [(1000, 700, 128, 32, 101), (512, 512, 64, 16, 102), (1300, 900, 128, 16, 103)]


def test_noalloc_growing_scratch_matches_factor_and_oracle(tq):
    mats, got = _run_sequence(tq, GROWING)
    _check_against_factor_and_oracle(tq, mats, GROWING, got)


def test_noalloc_shrinking_scratch_matches_factor_and_oracle(tq):
    cases = list(reversed(GROWING))
    mats, got = _run_sequence(tq, cases)
    _check_against_factor_and_oracle(tq, mats, cases, got)


def test_noalloc_refuses_problems_beyond_its_scratch(tq):
    lib = tq.load()
    d = tq.tileqr_desc()
    # 16384 x 16384 at nb 128 needs ~14 MB of scheduler state: refused from the
    # shape alone, before anything is read (the one-element buffer stands in
    # for A and is never touched)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.tileqr_factor_noalloc(16384, 16384, ctypes.c_void_p(dummy.data_ptr()), 16384, 128, 32,
                                   None, 0, None, 0, None, ctypes.byref(d))
    assert rc == tq.TILEQR_ERR_SCRATCH_LIMIT
    assert "noalloc" in tq.strerror(rc)
