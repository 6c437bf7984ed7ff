"""Pins of the oracle's tree variant (domains of h tile rows whose heads are
merged pairwise by triangle-on-triangle kernels DTTQRT / DTTSSRFB), checked
against what the mathematics fixes: the R factor of a full-rank matrix is
unique up to row signs (so it must equal the unblocked textbook QR's), Q is
orthogonal and reproduces A, the variant with one domain per step is
Algorithm 2 itself (bit for bit), any order respecting the dependencies gives
the same bits, and a plausible off-by-one in the triangular kernels fails."""
import numpy as np
import pytest

import oracle
from paper_0709_1272_gb300 import inputs

EPS = np.finfo(np.float64).eps

SHAPES = [
    (700, 300, 64, 16),    # ragged: last tile row 60 rows, last tile column 44
    (512, 256, 64, 16),    # exact tiles
    (640, 192, 64, 32),
    (200, 250, 64, 16),    # wide (m < n)
    (1100, 64, 64, 16),    # tall-skinny: 18 x 1 tiles, one step
]


def _rel_R_err(A, f):
    Rt = oracle.sign_normalize(f.R())
    Ru = oracle.sign_normalize(oracle.unblocked_qr(A))
    return np.abs(Rt - Ru).max() / max(np.abs(Ru).max(), 1e-300)


@pytest.mark.parametrize("m,n,nb,ib", SHAPES)
@pytest.mark.parametrize("h", [1, 2, 3, 5])
def test_tree_R_equals_unblocked(m, n, nb, ib, h):
    A = inputs.uniform_matrix(m, n, 11 + h)
    f = oracle.tiled_qr_tree(A, nb, ib, h)
    assert _rel_R_err(A, f) <= 20 * max(m, n) * EPS


@pytest.mark.parametrize("m,n,nb,ib", SHAPES[:3])
@pytest.mark.parametrize("h", [1, 3])
def test_tree_invariants(m, n, nb, ib, h):
    A = inputs.normal_matrix(m, n, 29 + h)
    f = oracle.tiled_qr_tree(A, nb, ib, h)
    orth, back, lower = oracle.invariants(A, f)
    assert orth <= 20 * max(m, n) * EPS
    assert back <= 20 * max(m, n) * EPS
    assert lower == 0.0


@pytest.mark.parametrize("h", [0, 11, 12, 1000])
def test_one_domain_is_algorithm2_bitwise(h):
    # 700 rows in tiles of 64: p = 11; h >= p (or h <= 0) leaves one domain per step
    A = inputs.uniform_matrix(700, 300, 3)
    flat = oracle.tiled_qr(A, 64, 16)
    tree = oracle.tiled_qr_tree(A, 64, 16, h)
    assert np.array_equal(flat.A, tree.A)
    assert np.array_equal(flat.T, tree.T)
    assert not np.any(tree.T2)
    assert oracle.task_list_tree(700, 300, 64, h) == oracle.task_list(700, 300, 64)


def test_ttqrt_merges_two_triangles():
    # two tiles of 64 rows, h = 1: DGEQRT on each, then one DTTQRT merge
    A = inputs.uniform_matrix(128, 64, 5)
    f = oracle.tiled_qr_tree(A, 64, 16, 1)
    assert _rel_R_err(A, f) <= 100 * EPS
    # the bottom tile's strict lower part still holds its own DGEQRT
    # reflectors, bit for bit: DTTQRT reads and writes only the triangle
    alone = oracle.tiled_qr(A[64:, :], 64, 16)
    assert np.array_equal(np.tril(f.A[64:, :], -1), np.tril(alone.A, -1))
    assert np.array_equal(f.tstrip(1, 0), alone.tstrip(0, 0))
    # the merged R of [R1; R2] is the QR of the two stacked triangles
    R1 = np.triu(oracle.tiled_qr(A[:64, :], 64, 16).A)
    R2 = np.triu(alone.A)
    Ru = oracle.sign_normalize(oracle.unblocked_qr(np.vstack([R1, R2])))
    assert np.abs(oracle.sign_normalize(f.R()) - Ru).max() <= 100 * EPS * np.abs(Ru).max()
    # the DTTQRT reflectors are upper triangular; T2 holds upper-triangular blocks
    V2 = np.triu(f.A[64:, :])
    assert np.any(V2)
    for l0 in range(0, 64, 16):
        blk = f.tstrip2(1, 0)[:, l0:l0 + 16]
        assert np.array_equal(blk, np.triu(blk))


def test_tt_reflectors_reproduce_R_via_apply():
    A = inputs.normal_matrix(900, 200, 8)
    f = oracle.tiled_qr_tree(A, 64, 16, 2)
    QtA = oracle.apply_qt(f, A)
    R = f.R()
    assert np.abs(QtA[:200, :] - R).max() <= 50 * 900 * EPS * np.abs(A).max()
    assert np.abs(QtA[200:, :]).max() <= 50 * 900 * EPS * np.abs(A).max()


@pytest.mark.parametrize("h", [1, 2, 3])
def test_tree_any_topological_order_same_bits(h):
    m, n, nb, ib = 520, 200, 64, 16
    A = inputs.uniform_matrix(m, n, 41)
    ref = oracle.tiled_qr_tree(A, nb, ib, h)
    rng = np.random.Generator(np.random.Philox(key=77 + h))
    for _ in range(3):
        order = oracle.random_topological_order(m, n, nb, rng, h=h)
        f = oracle.tiled_qr_tree_ordered(A, nb, ib, h, order)
        assert np.array_equal(f.A, ref.A)
        assert np.array_equal(f.T, ref.T)
        assert np.array_equal(f.T2, ref.T2)


def test_tree_dependencies_reduce_to_flat():
    tasks_f, preds_f = oracle.dependencies(520, 200, 64)
    tasks_t, preds_t = oracle.dependencies_tree(520, 200, 64, 100)
    assert tasks_f == tasks_t
    assert preds_f == preds_t


def test_tree_structure_counts():
    # every non-diagonal domain head is merged exactly once per step, into a
    # head above it; the merge levels are ceil(log2(#domains)) deep
    m, n, nb = 64 * 23, 64 * 4, 64
    for h in (1, 2, 3, 4, 7):
        tasks = oracle.task_list_tree(m, n, nb, h)
        for k in range(4):
            ndom = -(-(23 - k) // h)
            heads = [t[1] for t in tasks if t[0] == oracle.TASK_TTQRT and t[3] == k]
            assert sorted(heads) == [k + d * h for d in range(1, ndom)]
            for e in heads:
                pt = oracle.tt_partner(k, h, e)
                assert k <= pt < e and (pt - k) % h == 0
            assert sum(1 for t in tasks if t[0] == oracle.TASK_GEQRT and t[3] == k) == ndom


def test_tree_least_squares():
    m, n = 800, 150
    A = inputs.normal_matrix(m, n, 17)
    b = inputs.normal_matrix(m, 2, 18)
    f = oracle.tiled_qr_tree(A, 64, 16, 2)
    x = oracle.solve_ls(f, b)
    r = b - A @ x
    # optimality: A^T r = 0 to rounding
    assert np.abs(A.T @ r).max() / (np.linalg.norm(A) * np.linalg.norm(r)) <= 100 * EPS
    # consistent right-hand side: the exact solution is recovered
    xt = inputs.normal_matrix(n, 1, 19)
    y = oracle.solve_ls(f, A @ xt)
    assert np.abs(y - xt).max() <= 1e-11


def test_planted_tree_mistake_is_caught():
    A = inputs.uniform_matrix(512, 128, 23)
    try:
        oracle.set_mutation(5)   # triangular reflectors one row short
        f = oracle.tiled_qr_tree(A, 64, 16, 1)
        err = _rel_R_err(A, f)
    finally:
        oracle.set_mutation(0)
    assert err > 1e-3


# ---------------------------------------------------------------------------
# Q itself (not Q^T): the reverse replay, pinned by orthogonality identities
@pytest.mark.parametrize("m,n,nb,ib,h", [(700, 300, 64, 16, 0), (700, 300, 64, 16, 2), (512, 256, 64, 32, 1),
                                         (200, 450, 64, 16, 0), (1100, 64, 64, 16, 3)])
def test_apply_q_inverts_apply_qt(m, n, nb, ib, h):
    A = inputs.normal_matrix(m, n, 51 + h)
    f = oracle.tiled_qr_tree(A, nb, ib, h) if h else oracle.tiled_qr(A, nb, ib)
    B = inputs.normal_matrix(m, 9, 52)
    # Q (Q^T B) = B and Q^T (Q B) = B, to rounding
    assert np.abs(oracle.apply_q(f, oracle.apply_qt(f, B)) - B).max() <= 50 * m * EPS
    assert np.abs(oracle.apply_qt(f, oracle.apply_q(f, B)) - B).max() <= 50 * m * EPS
    # Q [R; 0] = A: the factorization is reproduced
    k = min(m, n)
    RZ = np.zeros((m, n), order="F")
    RZ[:k, :] = f.R()
    assert np.abs(oracle.apply_q(f, RZ) - A).max() <= 50 * m * EPS * np.abs(A).max()


@pytest.mark.parametrize("h", [0, 2])
def test_form_q_is_thin_orthonormal_factor(h):
    m, n = 600, 250
    A = inputs.uniform_matrix(m, n, 61)
    f = oracle.tiled_qr_tree(A, 64, 16, h) if h else oracle.tiled_qr(A, 64, 16)
    Q = oracle.form_q(f)
    assert Q.shape == (m, n)
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 20 * m * EPS
    assert np.linalg.norm(A - Q @ f.R()) / np.linalg.norm(A) <= 20 * m * EPS
    # Q^T applied to the identity is the transpose of the full Q
    Qfull = oracle.apply_q(f, np.eye(m))
    assert np.abs(Qfull - oracle.explicit_qt(f).T).max() <= 50 * m * EPS


def test_planted_block_order_mistake_in_apply_q_is_caught():
    A = inputs.normal_matrix(300, 200, 71)
    f = oracle.tiled_qr(A, 64, 16)
    B = inputs.normal_matrix(300, 3, 72)
    try:
        oracle.set_mutation(6)   # Q's inner blocks applied in forward order
        err = np.abs(oracle.apply_q(f, oracle.apply_qt(f, B)) - B).max()
    finally:
        oracle.set_mutation(0)
    assert err > 1e-6
