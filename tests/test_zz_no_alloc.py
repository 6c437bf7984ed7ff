"""tileqr_factor_noalloc, the factorization entry point for callers that
cannot allocate device memory (services that reserve their whole memory
budget at start-up, plug-ins whose host framework owns every allocation).
They pass only the input matrix and the output buffers; the scheduler's
scratch lives in a fixed array inside the library.

Checked here through the C ABI: two calls in a row on different shapes (the
second reuses the scratch the first left behind) give the same tiles and T
factors as tileqr_factor, within the 1e-12 tolerance of the other parity
tests; a problem too large for the fixed scratch is refused up front.
"""
import ctypes

import numpy as np
import pytest
import torch

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


def _noalloc(tq, Ad, nb, ib):
    """One call of tileqr_factor_noalloc; outputs in torch buffers we own."""
    lib = tq.load()
    m, n = Ad.shape
    p, q = -(-m // nb), -(-n // nb)
    tiles = torch.empty(p * q * nb * nb, dtype=torch.float64, device=Ad.device)
    T = torch.empty(p * q * ib * nb, dtype=torch.float64, device=Ad.device)
    d = tq.tileqr_desc()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.tileqr_factor_noalloc(m, n, ctypes.c_void_p(Ad.data_ptr()), Ad.stride(1), nb, ib,
                                   ctypes.c_void_p(tiles.data_ptr()), tiles.numel() * 8,
                                   ctypes.c_void_p(T.data_ptr()), T.numel() * 8, stream, ctypes.byref(d))
    assert rc == 0, tq.strerror(rc)
    assert lib.tileqr_status(ctypes.byref(d), stream) == 0
    f = tq.Factorization(d, tiles, Ad.device)     # keeps the output buffers alive
    AV, Tcm = f.factors()
    torch.cuda.synchronize()
    return AV.cpu().numpy(), Tcm.cpu().numpy()


def test_noalloc_matches_factor_on_two_calls_in_a_row(tq):
    cases = [(1000, 700, 128, 32, 101), (512, 384, 64, 16, 102)]
    mats = [tq.to_device_colmajor(inputs.normal_matrix(m, n, seed)) for (m, n, _, _, seed) in cases]
    got = [_noalloc(tq, Ad, nb, ib) for Ad, (_, _, nb, ib, _) in zip(mats, cases)]
    for Ad, (m, n, nb, ib, _), (AV, T) in zip(mats, cases, got):
        ref = tq.tileqr_factor(Ad, nb, ib).check()
        AVr, Tr = ref.factors()
        torch.cuda.synchronize()
        assert _rel(AV, AVr.cpu().numpy()) <= TOL
        assert _rel(T, Tr.cpu().numpy()) <= TOL


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
