"""Host-side trace analysis (paper_0709_1272_gb300/trace.py) on synthetic
traces of the QR task graph: a list schedule simulated here on the CPU, so
every start, end and readiness time is known."""
import heapq

import numpy as np
import pytest

from paper_0709_1272_gb300 import trace

DUR_NS = {0: 5000, 1: 4000, 2: 2000, 3: 3000, 4: 2500, 5: 1500}   # per kind


@pytest.fixture(scope="module")
def tq():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    tileqr.load()
    return tileqr


def _simulate(graph, nsm, per_sm, claim_ns):
    """Greedy FIFO list schedule of the graph on nsm x per_sm workers; a
    worker spends claim_ns between two tasks.  Returns the trace records and
    the readiness time of every task."""
    tasks, ndeps, ptr, succ = graph
    nt = len(tasks)
    left = ndeps.astype(np.int64).copy()
    ready_t = np.zeros(nt, np.int64)
    queue = [g for g in range(nt) if left[g] == 0]
    free = [(0, w) for w in range(nsm * per_sm)]   # (time the worker is free, worker)
    heapq.heapify(free)
    running = []                                  # (end, task, worker)
    rec = np.zeros((nt, 4), np.int64)
    n = 0
    while n < nt:
        if queue and free:
            t_free, w = heapq.heappop(free)
            g = queue.pop(0)
            t0 = max(t_free + claim_ns, ready_t[g])
            t1 = t0 + DUR_NS[int(tasks[g, 0])]
            kind, i, j, k = (int(x) for x in tasks[g])
            code = (np.uint64(1 if kind >= 4 else 0) << np.uint64(63)) | (np.uint64(k) << np.uint64(42)) | \
                (np.uint64(i) << np.uint64(21)) | np.uint64(j)
            rec[n] = [np.int64(code.astype(np.int64)), t0, t1, w // per_sm]
            n += 1
            heapq.heappush(running, (t1, g, w))
            continue
        t1, g, w = heapq.heappop(running)
        heapq.heappush(free, (t1, w))
        for v in succ[ptr[g]:ptr[g + 1]]:
            left[v] -= 1
            ready_t[v] = max(ready_t[v], t1)
            if left[v] == 0:
                queue.append(int(v))
    return rec, ready_t


@pytest.mark.parametrize("m,n,nb,domain,per_sm", [(1280, 1280, 128, 0, 2), (2560, 512, 128, 4, 1),
                                                  (640, 900, 64, 0, 1)])
def test_summary_and_ready_waits(tq, m, n, nb, domain, per_sm):
    graph = tq.tileqr_task_graph(m, n, nb, domain)
    rec, ready_t = _simulate(graph, nsm=3, per_sm=per_sm, claim_ns=700)
    s = trace.summary(rec, domain)
    assert s["tasks"] == len(graph[0])
    d = trace.decode(rec, domain)
    # the kinds decoded from the codes are the graph's own
    tasks = graph[0]
    lookup = {(int(t[3]), int(t[1]), int(t[2])): int(t[0]) for t in tasks if t[0] < 4}
    for n_ in range(len(rec)):
        if d["kind"][n_] < 4:
            assert lookup[(int(d["k"][n_]), int(d["i"][n_]), int(d["j"][n_]))] == d["kind"][n_]
    # slots: the simulated workers (every SM ran per_sm tasks at once at some time)
    assert s["slots"] == 3 * per_sm
    wall = (rec[:, 2].max() - rec[:, 1].min()) * 1e-9
    busy = ((rec[:, 2] - rec[:, 1]) * 1e-9).sum()
    assert s["busy_fraction"] == pytest.approx(busy / (wall * 3 * per_sm))
    assert 0 < s["busy_fraction"] <= 1
    # ready waits against the simulator's own readiness times
    w = trace.ready_waits(rec, graph, domain)
    start = {}
    for n_ in range(len(rec)):
        start[(int(d["kind"][n_]) >= 4, int(d["k"][n_]), int(d["i"][n_]), int(d["j"][n_]))] = rec[n_, 1]
    t_first = rec[:, 1].min()
    for kd, name in enumerate(trace.KINDS):
        sel = [g for g in range(len(tasks)) if tasks[g, 0] == kd]
        if not sel:
            assert name not in w
            continue
        ref = [(start[(kd >= 4, int(tasks[g, 3]), int(tasks[g, 1]), int(tasks[g, 2]))] -
                max(ready_t[g], t_first)) * 1e-3 for g in sel]
        assert w[name]["count"] == len(sel)
        assert w[name]["mean_us"] == pytest.approx(np.mean(ref))
        assert w[name]["min_us"] >= 0


def test_ready_waits_rejects_an_incomplete_trace(tq):
    graph = tq.tileqr_task_graph(512, 512, 128)
    rec, _ = _simulate(graph, nsm=2, per_sm=1, claim_ns=0)
    with pytest.raises(ValueError):
        trace.ready_waits(rec[:-1], graph)


def test_span_bounds_closed_forms(tq):
    # one tile column: DGEQRT then the chain of p - 1 DTSQRTs (Algorithm 2's
    # flat tree), nothing else
    p, nb = 9, 64
    graph = tq.tileqr_task_graph(p * nb, nb, nb)
    dur = {0: 5.0, 1: 3.0, 2: 1.0, 3: 2.0, 4: 1.0, 5: 1.0}
    b = trace.span_bounds(graph, dur, slots=4)
    assert b["critical_path_s"] == pytest.approx(5.0 + (p - 1) * 3.0)
    assert b["work_s"] == pytest.approx(5.0 + (p - 1) * 3.0)
    # square flat graph with updates of zero duration: the longest chain of
    # panel tasks, against a brute-force longest path over the same edges
    q = 6
    graph = tq.tileqr_task_graph(q * nb, q * nb, nb)
    dur0 = {0: 5.0, 1: 3.0, 2: 0.0, 3: 0.0, 4: 0.0, 5: 0.0}
    b = trace.span_bounds(graph, dur0, slots=4)
    # brute force over the dependency table (longest path by recursion)
    tasks, ndeps, ptr, succ = graph
    preds = {g: [] for g in range(len(tasks))}
    for u in range(len(tasks)):
        for v in succ[ptr[u]:ptr[u + 1]]:
            preds[int(v)].append(u)
    memo = {}

    def fin(g):
        if g not in memo:
            memo[g] = max((fin(u) for u in preds[g]), default=0.0) + dur0[int(tasks[g, 0])]
        return memo[g]

    assert b["critical_path_s"] == pytest.approx(max(fin(g) for g in range(len(tasks))))
    # the simulated list schedule is never shorter than either bound
    rec, _ = _simulate(graph, nsm=2, per_sm=2, claim_ns=0)
    durs = {k: v * 1e-9 for k, v in DUR_NS.items()}
    b = trace.span_bounds(graph, durs, slots=4)
    span = (rec[:, 2].max() - rec[:, 1].min()) * 1e-9
    assert span >= b["critical_path_s"] - 1e-12
    assert span >= b["work_per_slot_s"] - 1e-12


def _ticks_schedule(graph, dur, slots):
    """The kernel's policy stepped one integer tick at a time (a second,
    independent form of trace.priority_schedule for integer durations)."""
    tasks, ndeps, ptr, succ = graph
    nt = len(tasks)
    lvl = [trace.ready_level(int(kd), int(k), int(j)) for kd, _, j, k in tasks]
    left = [int(x) for x in ndeps]
    fifo = [[] for _ in range(4)]
    for g in range(nt):
        if left[g] == 0:
            fifo[lvl[g]].append(g)
    running = {}          # task -> end tick
    started = []          # start order
    t, done = 0, 0
    while done < nt:
        for g in [g for g in started if running.get(g) == t]:
            del running[g]
            done += 1
            for v in succ[ptr[g]:ptr[g + 1]]:
                left[int(v)] -= 1
                if left[int(v)] == 0:
                    fifo[lvl[int(v)]].append(int(v))
        while len(running) < slots and any(fifo):
            g = next(f for f in fifo if f).pop(0)
            running[g] = t + dur[int(tasks[g, 0])]
            started.append(g)
        if done < nt:
            t += 1
    return t


def test_priority_schedule(tq):
    nb = 64
    # one tile column: the DGEQRT then p - 1 DTSQRTs in a chain, whatever the slots
    p = 9
    graph = tq.tileqr_task_graph(p * nb, nb, nb)
    dur = {0: 5.0, 1: 3.0, 2: 1.0, 3: 2.0, 4: 1.0, 5: 1.0}
    for slots in (1, 4):
        assert trace.priority_schedule(graph, dur, slots)["span_s"] == pytest.approx(5.0 + (p - 1) * 3.0)
    # one worker runs the whole work back to back, claims included
    graph = tq.tileqr_task_graph(5 * nb, 4 * nb, nb)
    b = trace.span_bounds(graph, dur, slots=1)
    r = trace.priority_schedule(graph, dur, 1, claim_s=0.5)
    assert r["span_s"] == pytest.approx(b["work_s"] + 0.5 * len(graph[0]))
    assert r["busy_fraction"] == pytest.approx(1.0)
    # as many workers as tasks: the critical path
    r = trace.priority_schedule(graph, dur, len(graph[0]))
    assert r["span_s"] == pytest.approx(trace.span_bounds(graph, dur, 1)["critical_path_s"])
    # in between: never below either bound, and equal to the tick-by-tick
    # form of the same policy (flat and tree graphs, integer durations)
    idur = {0: 7, 1: 5, 2: 2, 3: 3, 4: 4, 5: 2}
    for (m, n, h) in ((6 * nb, 6 * nb, 0), (10 * nb, 3 * nb, 3), (4 * nb, 7 * nb, 0)):
        graph = tq.tileqr_task_graph(m, n, nb, h)
        for slots in (2, 3, 5):
            r = trace.priority_schedule(graph, idur, slots)
            b = trace.span_bounds(graph, idur, slots)
            assert r["span_s"] >= max(b["critical_path_s"], b["work_per_slot_s"]) - 1e-9
            assert r["span_s"] == _ticks_schedule(graph, idur, slots)


def test_ready_levels():
    # DGEQRT > DTSQRT > DLARFB > DSSRFB; the tree's merge joins the panel
    # level, its update the row-update level; column k + 1 one level up
    assert [trace.ready_level(kd, 0, 5) for kd in range(6)] == [0, 1, 2, 3, 1, 2]
    assert [trace.ready_level(kd, 0, 1) for kd in (2, 3, 5)] == [1, 2, 1]
