"""Pins of the CPU oracle to things other than itself (CPU only).

Closed forms (tests/golden/), LAPACK's own tile kernels (dgeqrt = DGEQRT,
dgemqrt = DLARFB, dtpqrt = DTSQRT, dtpmqrt = DSSRFB, all with inner block ib
and the same compact-WY T layout), LAPACK's dgeqrf R, an independently
written unblocked Householder QR, Cholesky of A^T A, the invariants of the
factorization, bitwise zero-padding and DAG-order independence, and the flop
model of Sec. 3.2.3.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.linalg.lapack as lapack

import oracle
from paper_0709_1272_gb300 import inputs

EPS = np.finfo(np.float64).eps
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _tri_blocks(strip, ib, ncols):
    """Upper triangles of the ib x ib blocks of a T strip (other entries unused)."""
    out = np.zeros_like(strip[:, :ncols])
    for l0 in range(0, ncols, ib):
        sb = min(ib, ncols - l0)
        out[:sb, l0:l0 + sb] = np.triu(strip[:sb, l0:l0 + sb])
    return out


# ---------------------------------------------------------------------------
# closed forms
@pytest.mark.parametrize("nb,ib", [(2, 1), (2, 2), (1, 1), (4, 2)])
def test_2x2_closed_form(nb, ib):
    for case in _golden("qr_2x2_closed_form.json")["cases"]:
        A = np.array(case["A"], dtype=np.float64)
        for R in (oracle.tiled_qr(A, nb, ib).R(), oracle.unblocked_qr(A)):
            assert R[0, 0] == pytest.approx(case["r11"], rel=4 * EPS, abs=0)
            assert R[0, 1] == pytest.approx(case["r12"], rel=8 * EPS, abs=8 * EPS)
            assert abs(R[1, 1]) == pytest.approx(case["abs_r22"], rel=16 * EPS, abs=16 * EPS)
            assert R[1, 0] == 0.0
            if "exact_R" in case:
                assert np.array_equal(R, np.array(case["exact_R"], dtype=np.float64))


@pytest.mark.parametrize("nb,ib", [(3, 1), (3, 3), (1, 1), (2, 1), (2, 2), (8, 4)])
def test_3x3_rational(nb, ib):
    for case in _golden("qr_3x3_rational.json")["cases"]:
        A = np.array(case["A"], dtype=np.float64)
        R0 = np.array(case["R0"], dtype=np.float64)
        f = oracle.tiled_qr(A, nb, ib)
        R = f.R()
        assert np.max(np.abs(oracle.sign_normalize(R) - R0)) <= 64 * EPS
        if "R11" in case and nb >= A.shape[0]:
            # one reflector reduces the whole first column only when it sits in one tile
            assert R[0, 0] == case["R11"]
        if "exact_R" in case:
            assert np.array_equal(R, np.array(case["exact_R"], dtype=np.float64))
            assert not np.any(f.T)  # no reflection anywhere: T == 0
        assert np.max(np.abs(oracle.sign_normalize(oracle.unblocked_qr(A)) - R0)) <= 64 * EPS


# ---------------------------------------------------------------------------
# against LAPACK's tile kernels
@pytest.mark.parametrize("nb,ib", [(16, 4), (12, 12), (32, 8), (20, 5)])
def test_geqrt_larfb_vs_lapack(nb, ib):
    A = inputs.uniform_matrix(nb, 3 * nb, seed=11)
    f = oracle.tiled_qr(A, nb, ib)           # one tile row: GEQRT + 2 LARFB
    a, t, info = lapack.dgeqrt(ib, np.asfortranarray(A[:, :nb]))
    assert info == 0
    assert _rel(f.tile(0, 0), a) <= 16 * nb * EPS
    assert _rel(_tri_blocks(f.tstrip(0, 0), ib, nb), _tri_blocks(t, ib, nb)) <= 16 * nb * EPS
    for j in (1, 2):
        c, info = lapack.dgemqrt(np.asfortranarray(f.tile(0, 0)), np.asfortranarray(f.tstrip(0, 0)),
                                 np.asfortranarray(A[:, j * nb:(j + 1) * nb]), side="L", trans="T")
        assert info == 0
        assert _rel(f.tile(0, j), c) <= 16 * nb * EPS


@pytest.mark.parametrize("nb,ib", [(16, 4), (12, 12), (32, 8)])
def test_tsqrt_ssrfb_vs_lapack(nb, ib):
    A = inputs.normal_matrix(2 * nb, 2 * nb, seed=12)
    # run Algorithm 2 up to (not including) GEQRT of step 1
    tasks = [t for t in oracle.task_list(2 * nb, 2 * nb, nb) if t[3] == 0]
    f = oracle.tiled_qr_ordered(A, nb, ib, tasks)
    top = oracle.tiled_qr(A[:nb, :], nb, ib)   # state after GEQRT(0), LARFB(0,1)
    R00 = np.triu(top.tile(0, 0))
    r, v, t, info = lapack.dtpqrt(0, ib, np.asfortranarray(R00), np.asfortranarray(A[nb:, :nb]))
    assert info == 0
    assert _rel(np.triu(f.tile(0, 0)), np.triu(r)) <= 16 * nb * EPS
    assert _rel(f.tile(1, 0), v) <= 16 * nb * EPS
    assert _rel(_tri_blocks(f.tstrip(1, 0), ib, nb), _tri_blocks(t, ib, nb)) <= 16 * nb * EPS
    b, c, info = lapack.dtpmqrt(0, np.asfortranarray(f.tile(1, 0)), np.asfortranarray(f.tstrip(1, 0)),
                                np.asfortranarray(top.tile(0, 1)), np.asfortranarray(A[nb:, nb:]),
                                side="L", trans="T")
    assert info == 0
    assert _rel(f.tile(0, 1), b) <= 16 * nb * EPS
    assert _rel(f.tile(1, 1), c) <= 16 * nb * EPS


@pytest.mark.parametrize("m,n,nb,ib", [(64, 64, 64, 16), (64, 40, 64, 8), (33, 33, 64, 4)])
def test_single_tile_is_lapack_dgeqrt(m, n, nb, ib):
    """With one tile (b >= m, n) Algorithm 2 is a single DGEQRT: V, R and T
    must equal LAPACK's blocked dgeqrt with block size ib."""
    A = inputs.uniform_matrix(m, n, seed=13)
    f = oracle.tiled_qr(A, nb, ib)
    a, t, info = lapack.dgeqrt(ib, np.asfortranarray(A))
    assert info == 0
    assert _rel(f.A, a) <= 16 * n * EPS
    k = min(m, n)
    assert _rel(_tri_blocks(f.T[:ib, :k], ib, k), _tri_blocks(t, ib, k)) <= 16 * n * EPS


# ---------------------------------------------------------------------------
# R against independent routines
SHAPES = [(50, 37, 8, 4), (37, 50, 8, 2), (64, 64, 16, 16), (70, 30, 16, 4), (31, 31, 5, 5),
          (96, 96, 32, 8), (9, 9, 1, 1), (128, 40, 12, 3)]


@pytest.mark.parametrize("m,n,nb,ib", SHAPES)
def test_tiled_equals_unblocked_and_lapack(m, n, nb, ib):
    A = inputs.normal_matrix(m, n, seed=m * 1000 + n)
    R = oracle.sign_normalize(oracle.tiled_qr(A, nb, ib).R())
    Ru = oracle.sign_normalize(oracle.unblocked_qr(A))
    Rl = oracle.sign_normalize(scipy.linalg.qr(A, mode="r")[0][:min(m, n)])
    tol = 20 * max(m, n) * EPS
    assert _rel(R, Ru) <= tol
    assert _rel(R, Rl) <= tol


def test_diag_r_equals_cholesky_of_gram():
    A = inputs.uniform_matrix(200, 120, seed=5)
    R = oracle.tiled_qr(A, 32, 8).R()
    L = np.linalg.cholesky(A.T @ A)
    assert np.max(np.abs(np.abs(np.diag(R)) - np.diag(L)) / np.diag(L)) <= 1e-12
    # and the whole R up to row signs: A^T A = R^T R = L L^T
    assert _rel(oracle.sign_normalize(R), L.T) <= 1e-12


# ---------------------------------------------------------------------------
# invariants of the factorization
@pytest.mark.parametrize("m,n,nb,ib,seed", [(512, 512, 64, 16, 20070710), (1024, 256, 128, 32, 7),
                                            (300, 200, 64, 16, 8), (200, 300, 64, 16, 9)])
def test_invariants(m, n, nb, ib, seed):
    A = inputs.uniform_matrix(m, n, seed)
    f = oracle.tiled_qr(A, nb, ib)
    orth, back, lower = oracle.invariants(A, f)
    assert lower == 0.0
    assert orth <= 20 * n * EPS
    assert back <= 20 * n * EPS


def test_invariants_tall_skinny_thin():
    """2048 x 512 (a reduced tall-skinny case): Q^T A = [R; 0] and Q^T
    preserves norms of random blocks."""
    m, n, nb, ib = 2048, 512, 128, 32
    A = inputs.normal_matrix(m, n, seed=3)
    f = oracle.tiled_qr(A, nb, ib)
    QtA = oracle.apply_qt(f, A)
    R = f.R()
    assert np.linalg.norm(QtA[:n] - R) / np.linalg.norm(A) <= 20 * n * EPS
    assert np.linalg.norm(QtA[n:]) / np.linalg.norm(A) <= 20 * n * EPS
    X = inputs.normal_matrix(m, 8, seed=4)
    Y = oracle.apply_qt(f, X)
    assert abs(np.linalg.norm(Y.T @ Y - X.T @ X)) / np.linalg.norm(X.T @ X) <= 20 * n * EPS


def test_apply_qt_gives_r():
    m, n, nb, ib = 150, 100, 32, 8
    A = inputs.uniform_matrix(m, n, seed=21)
    f = oracle.tiled_qr(A, nb, ib)
    QtA = oracle.apply_qt(f, A)
    assert _rel(QtA[:n], f.R()) <= 20 * n * EPS
    assert np.linalg.norm(QtA[n:]) <= 20 * n * EPS * np.linalg.norm(A)


# ---------------------------------------------------------------------------
# structure: padding and task order
@pytest.mark.parametrize("m,n,nb,ib", [(50, 37, 16, 4), (37, 50, 16, 8), (65, 65, 32, 8), (17, 3, 8, 2)])
def test_zero_padding_is_bitwise_equivalent(m, n, nb, ib):
    """Ragged edge tiles (our reading of the m = p b, n = q b assumption)
    must give the same bits as zero-padding the matrix to full tiles."""
    A = inputs.normal_matrix(m, n, seed=31)
    p, q = -(-m // nb), -(-n // nb)
    Ap = np.zeros((p * nb, q * nb), order="F")
    Ap[:m, :n] = A
    f = oracle.tiled_qr(A, nb, ib)
    g = oracle.tiled_qr(Ap, nb, ib)
    assert np.array_equal(f.A, g.A[:m, :n])
    assert np.array_equal(f.T[:, :n], g.T[:, :n])
    # the padding itself stays zero
    assert not np.any(g.A[m:, :]) if m < p * nb else True


@pytest.mark.parametrize("m,n,nb", [(40, 40, 8), (48, 24, 8), (24, 40, 8)])
def test_any_topological_order_gives_identical_bits(m, n, nb):
    ib = 4
    A = inputs.normal_matrix(m, n, seed=41)
    ref = oracle.tiled_qr(A, nb, ib)
    rng = np.random.default_rng(0)
    for _ in range(4):
        order = oracle.random_topological_order(m, n, nb, rng)
        f = oracle.tiled_qr_ordered(A, nb, ib, order)
        assert np.array_equal(f.A, ref.A)
        assert np.array_equal(f.T, ref.T)


def test_dependency_table():
    """The predecessors derived from the kernels' reads/writes are exactly the
    table of Sec. 4 as read for the flat elimination of Algorithm 2."""
    m = n = 5 * 4
    tasks, preds = oracle.dependencies(m, n, 4)
    G, T, L, S = oracle.TASK_GEQRT, oracle.TASK_TSQRT, oracle.TASK_LARFB, oracle.TASK_SSRFB
    for (kind, i, j, k) in tasks:
        want = set()
        if kind == G:
            if k > 0:
                want.add((S, k, k, k - 1))
        elif kind == L:
            want.add((G, k, k, k))
            if k > 0:
                want.add((S, k, j, k - 1))
        elif kind == T:
            want.add((T, i - 1, k, k) if i > k + 1 else (G, k, k, k))
            if k > 0:
                want.add((S, i, k, k - 1))
        else:
            want.add((T, i, k, k))
            want.add((S, i - 1, j, k) if i > k + 1 else (L, k, j, k))
            if k > 0:
                want.add((S, i, j, k - 1))
        assert preds[(kind, i, j, k)] == want, (kind, i, j, k)


# ---------------------------------------------------------------------------
# flop model (Sec. 3.2.3)
def test_flop_model():
    """The instrumented flop tally approaches 2n^2(m-n/3)(1+s/(4b)) as the
    tile count grows; the gap is the O(n^2 b) panel terms."""
    gaps = []
    for (m, n, nb, ib) in [(256, 256, 32, 8), (512, 512, 32, 8), (640, 320, 32, 16)]:
        A = inputs.uniform_matrix(m, n, seed=1)
        oracle.reset_flops()
        oracle.tiled_qr(A, nb, ib)
        tally = oracle.flops()
        model = oracle.tiled_flop_model(m, n, nb, ib)
        gap = tally / model - 1.0
        gaps.append(gap)
        assert abs(gap) < 4.0 * nb / n
    assert abs(gaps[1]) < abs(gaps[0])   # shrinks as q grows at fixed b


def test_flop_model_garble_reading():
    """The per-call DSSRFB cost is 4b^3 + s b^2 (the summand of Sec. 3.2.3
    prints 4b^2 + s b^2; only the cubic reading reproduces the printed total)."""
    p = q = 40
    b, s = 64, 16
    total = sum((4 * b**3 + s * b**2) * (p - k) * (q - k) for k in range(1, q + 1))
    n = m = p * b
    assert total / oracle.tiled_flop_model(m, n, b, s) == pytest.approx(1.0, rel=4.0 / q)


# ---------------------------------------------------------------------------
# least squares
def test_solve_ls_consistent_and_inconsistent():
    m, n, nb, ib = 300, 120, 32, 8
    A = inputs.normal_matrix(m, n, seed=51)
    f = oracle.tiled_qr(A, nb, ib)
    xt = inputs.normal_matrix(n, 3, seed=52)
    X = oracle.solve_ls(f, A @ xt)
    assert _rel(X, xt) <= 1e3 * EPS * np.linalg.cond(A)
    B = inputs.normal_matrix(m, 4, seed=53)
    X = oracle.solve_ls(f, B)
    Xl = np.linalg.lstsq(A, B, rcond=None)[0]
    assert _rel(X, Xl) <= 1e-12
    r = B - A @ X
    assert np.linalg.norm(A.T @ r) / (np.linalg.norm(A) * np.linalg.norm(r)) <= 20 * n * EPS


def _cholesky_solve_longdouble(G, c):
    """G x = c for SPD G by Cholesky in np.longdouble (plain loops, small n)."""
    n = G.shape[0]
    L = np.zeros((n, n), dtype=np.longdouble)
    for j in range(n):
        d = G[j, j] - np.sum(L[j, :j] * L[j, :j])
        L[j, j] = np.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (G[i, j] - np.sum(L[i, :j] * L[j, :j])) / L[j, j]
    y = np.zeros((n, c.shape[1]), dtype=np.longdouble)
    for i in range(n):
        y[i] = (c[i] - L[i, :i] @ y[:i]) / L[i, i]
    x = np.zeros_like(y)
    for i in reversed(range(n)):
        x[i] = (y[i] - L[i + 1:, i] @ x[i + 1:]) / L[i, i]
    return x


def test_solve_ls_matches_long_double_normal_equations():
    # the least-squares solution of a well-conditioned inconsistent system is
    # the solution of A^T A x = A^T b; formed and solved in extended precision
    # it is an independent check of solve_ls (Q^T b, then R x = (Q^T b)(0:n))
    m, n = 60, 14
    A = inputs.uniform_matrix(m, n, seed=61)
    B = inputs.normal_matrix(m, 2, seed=62)
    Al, Bl = A.astype(np.longdouble), B.astype(np.longdouble)
    Xl = _cholesky_solve_longdouble(Al.T @ Al, Al.T @ Bl).astype(np.float64)
    f = oracle.tiled_qr(A, 8, 4)
    X = oracle.solve_ls(f, B.copy())
    assert _rel(X, Xl) <= 50 * n * EPS * np.linalg.cond(A)


@pytest.mark.parametrize("e", [-1000, -900, -600, 600, 1000])
def test_extreme_magnitudes_scale_exactly(e):
    # scaling A by 2^e is exact, and so is R(2^e A) = 2^e R(A) in exact
    # arithmetic; at |e| = 900..1000 the squares of the entries under- or
    # overflow, so a plain sum of squares would give a zero or infinite norm
    # (the scaled accumulation of the Householder step must keep R finite and
    # accurate)
    m, n, nb, ib = 70, 45, 16, 4
    A = inputs.uniform_matrix(m, n, seed=63)
    c = np.ldexp(1.0, e)
    R = oracle.tiled_qr(A, nb, ib).R()
    Rc = oracle.tiled_qr(A * c, nb, ib).R()
    assert np.all(np.isfinite(Rc))
    assert _rel(Rc / c, R) <= 20 * n * EPS


def test_solve_ls_singular_reports_zero_pivot():
    A = np.zeros((6, 3), order="F")
    A[:, 0] = 1.0
    A[:, 2] = np.arange(6.0)
    f = oracle.tiled_qr(A, 2, 1)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.solve_ls(f, np.ones((6, 1)))


# ---------------------------------------------------------------------------
# inputs of the ill-conditioned workload
def test_kappa_matrix_singular_values():
    A, s, u, v = inputs.kappa_matrix(64, 1e6, seed=9)
    sv = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(sv, s, rtol=1e-12, atol=1e-15)
    R = oracle.tiled_qr(A, 16, 4).R()
    assert np.allclose(np.linalg.svd(R, compute_uv=False), s, rtol=1e-9, atol=1e-15)


# ---------------------------------------------------------------------------
# the pins catch planted mistakes
def _pins_pass():
    try:
        test_geqrt_larfb_vs_lapack(16, 4)
        test_tsqrt_ssrfb_vs_lapack(16, 4)
        test_tiled_equals_unblocked_and_lapack(50, 37, 8, 4)
        test_apply_qt_gives_r()
        test_2x2_closed_form(2, 1)
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mutation", [1, 2, 3, 4])
def test_planted_mistakes_are_caught(mutation):
    assert _pins_pass()
    oracle.set_mutation(mutation)
    try:
        assert not _pins_pass(), f"mutation {mutation} went unnoticed"
    finally:
        oracle.set_mutation(0)
    assert _pins_pass()
