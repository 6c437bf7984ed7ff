"""Tree form of the factorization on the GPU (domains of h tile rows, heads
merged pairwise by DTTQRT / DTTMQR) against the oracle's tree variant,
element by element through the C ABI.

Tolerance: relative Frobenius error 1e-12 in FP64 for R (sign-normalised),
the in-place factors (R, DGEQRT and DTSQRT reflectors, DTTQRT triangles)
and both T arrays: with equal (nb, ib, h) both sides compute the same
reflectors in the same order.  Bit-exact: the tree form with one domain per
step is Algorithm 2's kernel sequence, so it reproduces tileqr_factor's
bits.  Full size (262144 x 512, the benchmarked tall-skinny shape): the
first tile column against the oracle, and properties that hold at any size
(Q^T A = [R; 0], R^T R = A^T A, least-squares optimality)."""
import numpy as np
import pytest
import torch

import oracle
from paper_0709_1272_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12
EPS = np.finfo(np.float64).eps


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


CASES = [
    # (m, n, nb, ib, h): several domains and merge levels, ragged tails
    (700, 300, 64, 16, 1),
    (700, 300, 64, 16, 2),
    (1500, 256, 128, 16, 2),
    (2000, 384, 128, 32, 3),
    (2600, 200, 256, 16, 1),
    (64 * 23 + 17, 64 * 4 + 5, 64, 32, 4),
    (300, 900, 64, 16, 2),       # wide
    (4096, 128, 128, 16, 5),     # one tile column
]


@pytest.mark.parametrize("m,n,nb,ib,h", CASES)
def test_tree_matches_oracle(tq, m, n, nb, ib, h):
    A = inputs.normal_matrix(m, n, seed=700 + h)
    f = tq.tileqr_factor_tree(tq.to_device_colmajor(A), nb, ib, h).check()
    AV, T = f.factors()
    T2 = f.tree_T()
    R = f.R().cpu().numpy()
    ref = oracle.tiled_qr_tree(A, nb, ib, h)
    assert f.desc.domain == h
    assert _rel(oracle.sign_normalize(R), oracle.sign_normalize(ref.R())) <= TOL
    assert _rel(AV.cpu().numpy(), ref.A) <= TOL
    assert _rel(T.cpu().numpy(), ref.T) <= TOL
    assert _rel(T2.cpu().numpy(), ref.T2) <= TOL
    assert np.all(np.tril(R, -1) == 0.0)


@pytest.mark.parametrize("m,n,nb,ib,h", [(700, 300, 64, 16, 2), (2000, 384, 128, 32, 3), (300, 900, 64, 16, 2)])
def test_tree_apply_and_solve(tq, m, n, nb, ib, h):
    A = inputs.normal_matrix(m, n, seed=800 + h)
    B = inputs.normal_matrix(m, 37, seed=801 + h)
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor_tree(Ad, nb, ib, h).check()
    ref = oracle.tiled_qr_tree(A, nb, ib, h)
    QtB = f.apply_qt(tq.to_device_colmajor(B)).cpu().numpy()
    assert _rel(QtB, oracle.apply_qt(ref, B)) <= TOL
    if m >= n:
        X = f.solve_ls(tq.to_device_colmajor(B)).cpu().numpy()
        r = B - A @ X
        ratio = np.linalg.norm(A.T @ r) / (np.linalg.norm(A) * np.linalg.norm(r))
        assert ratio <= 20 * n * EPS
        assert _rel(X, oracle.solve_ls(ref, B)) <= 1e-10


@pytest.mark.parametrize("m,n,nb,ib", [(1000, 700, 128, 32), (640, 200, 64, 32)])
def test_one_domain_is_algorithm2_bitwise(tq, m, n, nb, ib):
    A = inputs.normal_matrix(m, n, seed=31)
    Ad = tq.to_device_colmajor(A)
    f0 = tq.tileqr_factor(Ad, nb, ib).check()
    p = -(-m // nb)
    for h in (p, p + 3):
        f1 = tq.tileqr_factor_tree(Ad, nb, ib, h).check()
        AV0, T0 = f0.factors()
        AV1, T1 = f1.factors()
        assert torch.equal(AV0, AV1) and torch.equal(T0, T1)
        assert f1.desc.T2 is None
    with pytest.raises(tq.TileQRError) as e:
        f0.tree_T()
    assert e.value.code == tq.TILEQR_ERR_UNSUPPORTED


def test_tree_repeatable_bitwise(tq):
    A = inputs.normal_matrix(3000, 512, seed=33)
    Ad = tq.to_device_colmajor(A)
    a = tq.tileqr_factor_tree(Ad, 128, 16, 2).check().factors()[0].clone()
    b = tq.tileqr_factor_tree(Ad, 128, 16, 2).check().factors()[0]
    assert torch.equal(a, b)


@pytest.mark.parametrize("m,n,nb,ib,h", [(2560, 512, 128, 16, 2), (3000, 600, 256, 32, 1), (64 * 23, 256, 64, 16, 3)])
def test_tree_trace_respects_dependencies(tq, m, n, nb, ib, h):
    from paper_0709_1272_gb300 import trace
    A = inputs.normal_matrix(m, n, seed=4343)
    tasks, preds = oracle.dependencies_tree(m, n, nb, h)
    rec = torch.zeros((len(tasks) + 16, 4), dtype=torch.int64, device="cuda")
    tq.tileqr_set_trace(rec)
    try:
        f = tq.tileqr_factor_tree(tq.to_device_colmajor(A), nb, ib, h).check()
        cnt = tq.tileqr_trace_count(f)
    finally:
        tq.tileqr_set_trace(None)
    assert cnt == len(tasks)
    d = trace.decode(rec[:cnt].cpu().numpy(), domain=h)
    seen = {}
    for n_ in range(cnt):
        key = (int(d["kind"][n_]), int(d["i"][n_]), int(d["j"][n_]), int(d["k"][n_]))
        assert key not in seen, f"task {key} ran twice"
        seen[key] = (int(d["t0"][n_]), int(d["t1"][n_]))
    assert set(seen) == set(tasks)
    for t in tasks:
        for pr in preds[t]:
            assert seen[pr][1] <= seen[t][0], f"{t} started before its predecessor {pr} finished"


def test_tree_mixed_precision(tq):
    """TILEQR_TF32 with the tree: the three update kinds (DLARFB, DSSRFB,
    DTTMQR) on the tensor cores; backward error within the FP32-accumulation
    bound of the flat mixed path."""
    m, n, nb, ib, h = 8192, 512, 128, 16, 4
    A = inputs.normal_matrix(m, n, seed=35)
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor_tree(Ad, nb, ib, h, precision=tq.TILEQR_TF32).check()
    R = f.R()
    QtA = f.apply_qt(Ad.clone())
    back = (torch.linalg.matrix_norm(QtA[:n] - R) / torch.linalg.matrix_norm(Ad)).item()
    assert back <= 32 * n * 2.0 ** -24
    assert (torch.linalg.matrix_norm(QtA[n:]) / torch.linalg.matrix_norm(Ad)).item() <= 32 * n * 2.0 ** -24
    ref = oracle.tiled_qr_tree(A, nb, ib, h)
    Rn = oracle.sign_normalize(R.cpu().numpy())
    assert _rel(Rn, oracle.sign_normalize(ref.R())) <= 1e-4


@pytest.mark.parametrize("ib,h", [(16, 8), (32, 16)])
def test_full_tall_skinny_tree(tq, ib, h):
    """262144 x 512 N(0,1), nb 128: ib 16 with domain 8 (the benchmarked FP64
    tree launch) and ib 32 with domain 16, with tileqr_solve_ls on 16
    right-hand sides."""
    m, n, nb = 262144, 512, 128
    A = inputs.normal_matrix(m, n, seed=20070712)
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor_tree(Ad, nb, ib, h).check()
    AV, T = f.factors()
    T2 = f.tree_T()
    # the first tile column is step 0 alone: the oracle's tree on that panel
    panel = oracle.tiled_qr_tree(A[:, :nb], nb, ib, h)
    assert _rel(AV[:, :nb].cpu().numpy(), panel.A) <= TOL
    assert _rel(T[:, :nb].cpu().numpy(), panel.T) <= TOL
    assert _rel(T2[:, :nb].cpu().numpy(), panel.T2) <= TOL
    R = f.R()
    QtA = f.apply_qt(Ad.clone())
    nA = torch.linalg.matrix_norm(Ad)
    assert (torch.linalg.matrix_norm(QtA[:n] - R) / nA).item() <= 20 * n * EPS
    assert (torch.linalg.matrix_norm(QtA[n:]) / nA).item() <= 20 * n * EPS
    # R^T R = A^T A: a backward error dA gives ||R^T R - A^T A|| <= 2 ||A|| ||dA||
    G = Ad.t() @ Ad
    assert (torch.linalg.matrix_norm(R.t() @ R - G) / nA ** 2).item() <= 20 * n * EPS
    B = inputs.normal_matrix(m, 16, seed=20070713)
    Bd = tq.to_device_colmajor(B)
    X = f.solve_ls(Bd.clone())
    r = Bd - Ad @ X
    ratio = (torch.linalg.matrix_norm(Ad.t() @ r) / (nA * torch.linalg.matrix_norm(r))).item()
    assert ratio <= 20 * n * EPS


def test_full_tall_skinny_tree_mixed(tq):
    """262144 x 512 N(0,1), nb 128, ib 16, domain 16 with TILEQR_TF32 (the
    benchmarked mixed tree launch): backward error within the FP32
    accumulation bound, and Q (built from FP64 reflectors) orthogonal to FP64
    rounding on random probes."""
    m, n, nb, ib, h = 262144, 512, 128, 16, 16
    A = inputs.normal_matrix(m, n, seed=20070712)
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor_tree(Ad, nb, ib, h, precision=tq.TILEQR_TF32).check()
    R = f.R()
    QtA = f.apply_qt(Ad.clone())
    nA = torch.linalg.matrix_norm(Ad)
    assert (torch.linalg.matrix_norm(QtA[:n] - R) / nA).item() <= 32 * n * 2.0 ** -24
    assert (torch.linalg.matrix_norm(QtA[n:]) / nA).item() <= 32 * n * 2.0 ** -24
    X = tq.to_device_colmajor(inputs.normal_matrix(m, 4, seed=20070714))
    Y = f.apply_qt(f.apply_q(X.clone()))
    assert (torch.linalg.matrix_norm(Y - X) / torch.linalg.matrix_norm(X)).item() <= 20 * n * EPS


def test_tree_argument_errors(tq):
    import ctypes
    lib = tq.load()
    d = tq.tileqr_desc()
    rc = lib.tileqr_factor_tree(10, 10, ctypes.c_void_p(1), 10, 64, 16, -1, 0, 0, None, 0, None, ctypes.byref(d))
    assert rc == -7
    rc = lib.tileqr_factor_tree(10, 10, ctypes.c_void_p(1), 10, 64, 16, 2, 9, 0, None, 0, None, ctypes.byref(d))
    assert rc == -8
    # refinement needs nb 128 (its FP32 correction solve), any domain size
    A = tq.to_device_colmajor(inputs.normal_matrix(600, 128, seed=1))
    f = tq.tileqr_factor_tree(A, 64, 16, 2).check()
    with pytest.raises(tq.TileQRError) as e:
        f.solve_refine(A, A[:, 0].contiguous())
    assert e.value.code == tq.TILEQR_ERR_UNSUPPORTED


def test_full_elementwise_tree_16384x512(tq):
    """16384 x 512 N(0,1), nb 128 / ib 16, domains of 8 tile rows (the
    benchmarked FP64 tree configuration on a 128 x 4 tile grid): every
    element of R/V, T and the DTTQRT strips T2 against the oracle's tree
    variant at 1e-12."""
    m, n, nb, ib, h = 16384, 512, 128, 16, 8
    A = inputs.normal_matrix(m, n, seed=20070716)
    Ad = tq.to_device_colmajor(A)
    f = tq.tileqr_factor_tree(Ad, nb, ib, h).check()
    AV, T = f.factors()
    T2 = f.tree_T()
    ref = oracle.tiled_qr_tree(A, nb, ib, h)
    assert _rel(AV.cpu().numpy(), ref.A) <= TOL
    assert _rel(T.cpu().numpy(), ref.T) <= TOL
    assert _rel(T2.cpu().numpy(), ref.T2) <= TOL
