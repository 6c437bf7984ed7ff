"""The task graph the persistent kernels execute (exported by the library's
host-only tileqr_task_graph, built from the same functions the kernels call)
against the dependencies the oracle derives mechanically from the tiles each
task reads and writes, for Algorithm 2 and the tree form.

Checked: the same task set; every task is released by exactly ndeps
signals; the graph is acyclic and runs to completion; every mechanically
required ordering is enforced (a path in the library graph); and every
library edge is a real dependency (implied by the mechanical ones).  A wrong
edge here would hang or corrupt the GPU run, so this is checked on the CPU
first.  No GPU is needed."""
import pytest

import oracle

CASES = [
    (520, 200, 64, 0),      # Algorithm 2, ragged edges
    (520, 200, 64, 100),    # domain >= p: flat
    (520, 200, 64, 1),      # binary tree over every tile row
    (520, 200, 64, 2),
    (700, 300, 64, 3),
    (64 * 23, 64 * 4, 64, 4),
    (64 * 23, 64 * 4, 64, 5),
    (200, 450, 64, 2),      # wide: p < q
    (1100, 64, 64, 2),      # one tile column
    (64 * 9, 64 * 9, 64, 2),
]


@pytest.fixture(scope="module")
def tq():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    tileqr.load()
    return tileqr


def _graph(tq, m, n, nb, h, what):
    tasks, ndeps, ptr, succ = tq.tileqr_task_graph(m, n, nb, h, what)
    keys = [tuple(int(x) for x in t) for t in tasks]
    edges = [(a, int(b)) for a in range(len(keys)) for b in succ[ptr[a]:ptr[a + 1]]]
    return keys, [int(x) for x in ndeps], edges


def _ancestors(n, edges):
    """Bit set of the ancestors of every node (Kahn order); also checks that
    the graph is acyclic."""
    preds = [[] for _ in range(n)]
    succ = [[] for _ in range(n)]
    indeg = [0] * n
    for a, b in edges:
        preds[b].append(a)
        succ[a].append(b)
        indeg[b] += 1
    order = [v for v in range(n) if indeg[v] == 0]
    head = 0
    while head < len(order):
        v = order[head]
        head += 1
        for w in succ[v]:
            indeg[w] -= 1
            if indeg[w] == 0:
                order.append(w)
    assert len(order) == n, "cycle or unreachable task"
    anc = [0] * n
    for v in order:
        acc = 0
        for u in preds[v]:
            acc |= anc[u] | (1 << u)
        anc[v] = acc
    return anc


def _compare(keys, ndeps, edges, otasks, opreds):
    n = len(keys)
    assert sorted(keys) == sorted(otasks)
    assert len(set(keys)) == n
    indeg = [0] * n
    for _, b in edges:
        indeg[b] += 1
    assert indeg == ndeps
    pos = {k: i for i, k in enumerate(keys)}
    anc_lib = _ancestors(n, edges)
    oedges = [(pos[p], pos[t]) for t, ps in opreds.items() for p in ps]
    anc_or = _ancestors(n, oedges)
    for a, b in oedges:     # every required order is enforced
        assert (anc_lib[b] >> a) & 1, (keys[a], keys[b])
    for a, b in edges:      # no edge without a real dependency behind it
        assert (anc_or[b] >> a) & 1, (keys[a], keys[b])


@pytest.mark.parametrize("m,n,nb,h", CASES)
def test_factorization_graph(tq, m, n, nb, h):
    keys, ndeps, edges = _graph(tq, m, n, nb, h, 0)
    if h <= 0:
        otasks, opreds = oracle.dependencies(m, n, nb)
    else:
        otasks, opreds = oracle.dependencies_tree(m, n, nb, h)
    _compare(keys, ndeps, edges, otasks, opreds)


@pytest.mark.parametrize("m,n,nb,h", CASES)
def test_apply_graph(tq, m, n, nb, h):
    keys, ndeps, edges = _graph(tq, m, n, nb, h, 1)
    keys = [(k[0], k[1], k[3]) for k in keys]   # {kind, i, -1, k} -> (kind, i, k)
    otasks, opreds = oracle.apply_dependencies_tree(m, n, nb, h)
    _compare(keys, ndeps, edges, otasks, opreds)


@pytest.mark.parametrize("m,n,nb,h", CASES)
def test_apply_q_graph(tq, m, n, nb, h):
    # Q (not Q^T): the same tasks in the reverse graph
    keys, ndeps, edges = _graph(tq, m, n, nb, h, 2)
    keys = [(k[0], k[1], k[3]) for k in keys]
    otasks, opreds = oracle.apply_dependencies_tree(m, n, nb, h, reverse=True)
    _compare(keys, ndeps, edges, otasks, opreds)


@pytest.mark.parametrize("n,nb", [(520, 64), (64 * 9, 64), (100, 64), (64, 64), (1000, 128)])
def test_cholesky_graph(tq, n, nb):
    keys, ndeps, edges = _graph(tq, n, n, nb, 0, 3)
    otasks, opreds = oracle.cholesky_dependencies(n, nb)
    _compare(keys, ndeps, edges, otasks, opreds)


@pytest.mark.parametrize("n,nb", [(320, 64), (64 * 9, 64), (100, 64), (64, 64), (1024, 128)])
def test_lu_graph(tq, n, nb):
    # Algorithm 3's graph, executed with the flat-tree graph functions
    keys, ndeps, edges = _graph(tq, n, n, nb, 0, 4)
    npad = -(-n // nb) * nb
    otasks, opreds = oracle.lu_dependencies(npad, nb)
    _compare(keys, ndeps, edges, otasks, opreds)


def test_task_counts_match_the_workspace_queues(tq):
    # the write-once ready queues are sized from closed-form counts; they must
    # equal the enumerated graph
    import numpy as np
    for (m, n, nb, h) in CASES:
        tasks, _, _, _ = tq.tileqr_task_graph(m, n, nb, h, 0)
        kinds = np.bincount(tasks[:, 0], minlength=6)
        p, q = -(-m // nb), -(-n // nb)
        H = p if (h <= 0 or h > p) else h
        exp = [0] * 6
        for k in range(min(p, q)):
            P, nd, nq = p - k, -(-(p - k) // H), q - k - 1
            exp[0] += nd
            exp[1] += P - nd
            exp[4] += nd - 1
            exp[2] += nd * nq
            exp[3] += (P - nd) * nq
            exp[5] += (nd - 1) * nq
        assert list(kinds) == exp


def _level(kind, k, j):
    """Ready-queue level of a task: the kind's level (tree merge with the
    panels, tree update with the row updates), one level up for an update of
    column k+1, which feeds the next step's panel."""
    base = kind if kind < 4 else (1 if kind == 4 else 2)
    return base - 1 if (kind in (2, 3, 5) and j == k + 1) else base


def _level_counts_closed_form(p, q, h):
    # the closed form the library sizes its write-once queues with
    H = p if (h <= 0 or h > p) else h
    caps = [0] * 4
    for k in range(min(p, q)):
        P, nq = p - k, q - k - 1
        nd = -(-P // H)
        c1, rest = (1, nq - 1) if nq > 0 else (0, 0)
        caps[0] += nd
        caps[1] += (P - nd) + (nd - 1) + nd * c1 + (nd - 1) * c1
        caps[2] += nd * rest + (nd - 1) * rest + (P - nd) * c1
        caps[3] += (P - nd) * rest
    return caps


@pytest.mark.parametrize("m,n,nb,h", CASES + [(128 * 40, 128 * 40, 128, 0), (128 * 40, 128 * 40, 128, 8)])
def test_queue_levels_match_the_enumerated_graph(tq, m, n, nb, h):
    tasks, _, _, _ = tq.tileqr_task_graph(m, n, nb, h, 0)
    cnt = [0] * 4
    for kind, i, j, k in tasks:
        cnt[_level(int(kind), int(k), int(j))] += 1
    assert cnt == _level_counts_closed_form(-(-m // nb), -(-n // nb), h)
