"""Out-of-bounds writes: every caller-owned buffer is surrounded by canary
bytes and checked after the call.

The workspaces are passed at exactly their queried size inside a larger
allocation whose first and last 64 KB hold a byte pattern; the output
matrices get padding rows (ld > rows) holding a sentinel value.  A kernel
that writes outside what it owns changes one of them.  Covers the FP64 and
TF32 factorizations (flat and tree form, ragged shapes, so the ragged-edge
tile instances run), the mixed application of Q, the least-squares
refinement and the plain solve."""
import ctypes

import numpy as np
import pytest
import torch

from paper_0709_1272_gb300 import inputs

pytestmark = pytest.mark.gpu

CANARY = 1 << 16
PATTERN = 0xA5
SENTINEL = -7.25


@pytest.fixture(scope="module")
def tq():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    tileqr.load()
    return tileqr


def _padded(nbytes):
    buf = torch.full((nbytes + 2 * CANARY,), PATTERN, dtype=torch.uint8, device="cuda")
    return buf, buf[CANARY:CANARY + nbytes]


def _intact(buf, nbytes):
    torch.cuda.synchronize()
    return bool((buf[:CANARY] == PATTERN).all()) and bool((buf[CANARY + nbytes:] == PATTERN).all())


def _padded_matrix(a, extra=8):
    """Column-major copy of a with `extra` sentinel rows below it (ld = rows + extra)."""
    m, n = a.shape
    full = torch.full((n, m + extra), SENTINEL, dtype=torch.float64, device="cuda")
    full[:, :m] = torch.from_numpy(np.ascontiguousarray(a.T)).cuda()
    return full


def _rows_intact(full, m):
    torch.cuda.synchronize()
    return bool((full[:, m:] == SENTINEL).all())


@pytest.mark.parametrize("m,n,nb,ib,h,prec", [
    (1000, 700, 128, 32, 0, "fp64"), (777, 333, 64, 16, 0, "fp64"), (2000, 384, 128, 16, 3, "fp64"),
    (1000, 700, 128, 16, 0, "tf32"), (2000, 384, 128, 16, 4, "tf32"),
])
def test_factorization_stays_in_its_workspace(tq, m, n, nb, ib, h, prec):
    p = tq.TILEQR_TF32 if prec == "tf32" else tq.TILEQR_FP64
    A = inputs.normal_matrix(m, n, seed=3100 + m)
    Ad = _padded_matrix(A)
    Acm = Ad[:, :m].t()   # m x n column-major view with ld m + 8
    need = tq.tileqr_workspace_size_tree(m, n, nb, ib, p, h) if h else tq.tileqr_workspace_size(m, n, nb, ib, p)
    buf, ws = _padded(need)
    if h:
        f = tq.tileqr_factor_tree(Acm, nb, ib, h, precision=p, workspace=ws).check()
    else:
        f = tq.tileqr_factor(Acm, nb, ib, precision=p, workspace=ws).check()
    assert _intact(buf, need)
    assert _rows_intact(Ad, m)            # A is read only
    R = f.R()
    assert torch.isfinite(R).all()
    # the plain solve (its own workspace, from the binding) leaves the
    # factorization's workspace and its canaries as they were
    B = inputs.normal_matrix(m, 3, seed=3101)
    f.solve_ls(tq.to_device_colmajor(B))
    assert _intact(buf, need)


def test_mixed_application_and_refinement_stay_in_their_buffers(tq):
    m, n, nrhs = 1500, 500, 7
    lib = tq.load()
    A = inputs.normal_matrix(m, n, seed=3200)
    Ad = tq.to_device_colmajor(A)
    need = tq.tileqr_workspace_size_tree(m, n, 128, 16, tq.TILEQR_TF32, 4)
    fbuf, fws = _padded(need)
    f = tq.tileqr_factor_tree(Ad, 128, 16, 4, precision=tq.TILEQR_TF32, workspace=fws).check()
    B = inputs.normal_matrix(m, nrhs, seed=3201)
    for trans in (1, 0):
        Bd = _padded_matrix(B)
        sz = ctypes.c_size_t(0)
        assert lib.tileqr_apply_mixed_workspace_size(ctypes.byref(f.desc), nrhs, ctypes.byref(sz)) == 0
        abuf, aws = _padded(sz.value)
        rc = lib.tileqr_apply_mixed(ctypes.byref(f.desc), trans, ctypes.c_void_p(Bd.data_ptr()), m + 8, nrhs,
                                    ctypes.c_void_p(aws.data_ptr()), sz.value, None)
        assert rc == 0
        assert _intact(abuf, sz.value) and _rows_intact(Bd, m)
    # least-squares refinement: workspace, X and the residual output
    sz = ctypes.c_size_t(0)
    assert lib.tileqr_ls_refine_workspace_size(ctypes.byref(f.desc), nrhs, ctypes.byref(sz)) == 0
    rbuf, rws = _padded(sz.value)
    Bd = _padded_matrix(B)
    X = torch.full((nrhs, n + 8), SENTINEL, dtype=torch.float64, device="cuda")
    Rr = torch.full((nrhs, m + 8), SENTINEL, dtype=torch.float64, device="cuda")
    info = tq.tileqr_refine_info()
    rc = lib.tileqr_solve_ls_refine(ctypes.byref(f.desc), ctypes.c_void_p(Ad.data_ptr()), m,
                                    ctypes.c_void_p(Bd.data_ptr()), m + 8, nrhs,
                                    ctypes.c_void_p(X.data_ptr()), n + 8, ctypes.c_void_p(Rr.data_ptr()), m + 8,
                                    10, 1e-14, ctypes.c_void_p(rws.data_ptr()), sz.value, None, ctypes.byref(info))
    assert rc == 0 and info.converged == 1
    assert _intact(rbuf, sz.value)
    assert _rows_intact(Bd, m) and _rows_intact(X, n) and _rows_intact(Rr, m)
    assert _intact(fbuf, need)
