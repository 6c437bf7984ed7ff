"""Task traces of the persistent scheduler: decoding, a per-kind summary and
export to the Chrome trace-event format (one row per SM, like the execution
flow of Sec. 4, Fig. 6)."""
from __future__ import annotations

import json

import numpy as np

KINDS = ("DGEQRT", "DTSQRT", "DLARFB", "DSSRFB", "DTTQRT", "DTTMQR")


def decode(records: np.ndarray, domain: int = 0):
    """records: (N, 4) int64 {code, t0, t1, sm} -> dict of arrays.  `domain`:
    the tree form's domain size (0 for Algorithm 2), which decides the kinds."""
    r = np.asarray(records, dtype=np.uint64)
    code = r[:, 0]
    tt = (code >> np.uint64(63)).astype(np.int64)
    k = ((code >> np.uint64(42)) & np.uint64(0x1FFFFF)).astype(np.int64)
    i = ((code >> np.uint64(21)) & np.uint64(0x1FFFFF)).astype(np.int64)
    j = (code & np.uint64(0x1FFFFF)).astype(np.int64)
    head = (i == k) if domain <= 0 else ((i - k) % domain == 0)
    kind = np.where(tt == 1, np.where(j == k, 4, 5),
                    np.where(head, np.where(j == k, 0, 2), np.where(j == k, 1, 3)))
    t0 = r[:, 1].astype(np.int64)
    t1 = r[:, 2].astype(np.int64)
    return {"k": k, "i": i, "j": j, "kind": kind, "t0": t0, "t1": t1, "sm": r[:, 3].astype(np.int64)}


def slots_per_sm(d) -> np.ndarray:
    """Most tasks in flight at once on each SM (the worker CTAs it held)."""
    nsm = int(d["sm"].max()) + 1
    out = np.zeros(nsm, dtype=np.int64)
    for sm in np.unique(d["sm"]):
        sel = d["sm"] == sm
        t = np.concatenate([d["t0"][sel], d["t1"][sel]])
        step = np.concatenate([np.ones(int(sel.sum()), np.int64), -np.ones(int(sel.sum()), np.int64)])
        order = np.lexsort((step, t))   # at equal times an end before a start
        out[sm] = int(np.cumsum(step[order]).max())
    return out


def summary(records: np.ndarray, domain: int = 0) -> dict:
    """Per-kind task counts and mean durations, and the occupancy of the
    worker slots: busy_fraction = task time / (wall x slots), slots = the
    tasks in flight at once summed over the SMs (one or two CTAs per SM)."""
    d = decode(records, domain)
    t_begin, t_end = int(d["t0"].min()), int(d["t1"].max())
    wall = (t_end - t_begin) * 1e-9
    dur = (d["t1"] - d["t0"]) * 1e-9
    slots = int(slots_per_sm(d).sum())
    out = {"tasks": int(len(dur)), "wall_s": wall, "slots": slots,
           "busy_fraction": float(dur.sum() / (wall * slots)) if wall > 0 else 1.0,
           "idle_per_task_us": float((wall * slots - dur.sum()) / len(dur) * 1e6), "per_kind": {}}
    for kd, name in enumerate(KINDS):
        sel = d["kind"] == kd
        if sel.any():
            out["per_kind"][name] = {"count": int(sel.sum()), "mean_us": float(dur[sel].mean() * 1e6),
                                     "total_sm_s": float(dur[sel].sum())}
    return out


def ready_waits(records: np.ndarray, graph, domain: int = 0) -> dict:
    """Time from a task's readiness (the end of its last predecessor; the
    first task's start for tasks without one) to its start, per kind.
    `graph` = (tasks, ndeps, succ_ptr, succ) of tileqr_task_graph (what = 0,
    the QR factorization) for the same shape, nb and domain.  Long waits with idle slots point at the scheduler;
    long waits with busy slots at a shortage of workers."""
    d = decode(records, domain)
    tasks, _, ptr, succ = graph
    index = {}
    for g in range(len(tasks)):
        kind, i, j, k = (int(x) for x in tasks[g])
        index[(1 if kind >= 4 else 0, k, i, j)] = g
    tt = np.where(d["kind"] >= 4, 1, 0)
    gid = np.array([index[(int(tt[n]), int(d["k"][n]), int(d["i"][n]), int(d["j"][n]))]
                    for n in range(len(d["t0"]))], dtype=np.int64)
    if len(set(gid.tolist())) != len(tasks) or len(gid) != len(tasks):
        raise ValueError("the trace does not hold every task of the graph exactly once")
    start = np.empty(len(tasks), np.int64)
    end = np.empty(len(tasks), np.int64)
    start[gid] = d["t0"]
    end[gid] = d["t1"]
    ready = np.full(len(tasks), int(d["t0"].min()), np.int64)
    src = np.repeat(np.arange(len(tasks)), np.diff(ptr))
    np.maximum.at(ready, np.asarray(succ, dtype=np.int64), end[src])
    wait = (start - ready) * 1e-3   # us
    kind_of = tasks[:, 0]
    out = {}
    for kd, name in enumerate(KINDS):
        sel = kind_of == kd
        if sel.any():
            w = wait[sel]
            out[name] = {"count": int(sel.sum()), "mean_us": float(w.mean()),
                         "median_us": float(np.median(w)), "p90_us": float(np.percentile(w, 90)),
                         "min_us": float(w.min())}
    return out


def span_bounds(graph, dur_by_kind: dict, slots: int) -> dict:
    """Lower bounds on the span of the task graph `graph` (tileqr_task_graph
    output) with a duration per task kind (seconds, keyed by the kind codes
    0..5) on `slots` workers: the critical path (longest chain of dependent
    tasks) and the work divided by the slots.  A list schedule never beats the
    larger of the two; comparing a trace's span with them tells whether the
    run was bound by the graph, by the work or by the scheduler."""
    tasks, ndeps, ptr, succ = graph
    nt = len(tasks)
    dur = np.array([dur_by_kind[int(k)] for k in tasks[:, 0]], dtype=np.float64)
    # longest path by Kahn's order over the successor lists
    left = ndeps.astype(np.int64).copy()
    finish = np.zeros(nt)
    start = np.zeros(nt)
    order = [g for g in range(nt) if left[g] == 0]
    head = 0
    while head < len(order):
        u = order[head]
        head += 1
        finish[u] = start[u] + dur[u]
        for v in succ[ptr[u]:ptr[u + 1]]:
            start[v] = max(start[v], finish[u])
            left[v] -= 1
            if left[v] == 0:
                order.append(int(v))
    if len(order) != nt:
        raise ValueError("the graph has a cycle or a task that is never released")
    return {"critical_path_s": float(finish.max()) if nt else 0.0, "work_s": float(dur.sum()),
            "work_per_slot_s": float(dur.sum() / slots)}


def ready_level(kind: int, k: int, j: int) -> int:
    """Ready-queue level of a task (0 = served first), as the persistent
    kernel assigns it: DGEQRT 0, DTSQRT and DTTQRT 1, DLARFB and DTTMQR 2,
    DSSRFB 3, and an update of column k + 1 one level up (it feeds the next
    step's panel)."""
    base = kind if kind < 4 else (1 if kind == 4 else 2)
    return base - 1 if (kind in (2, 3, 5) and j == k + 1) else base


def priority_schedule(graph, dur_by_kind: dict, slots: int, claim_s: float = 0.0) -> dict:
    """Simulated span of the persistent kernel's policy on `graph`
    (tileqr_task_graph output, QR kinds): `slots` workers; a released task
    joins the FIFO of its ready level; a free worker takes the oldest task of
    the lowest non-empty level and holds it for claim_s + its kind's duration
    (seconds, keyed by the kind codes 0..5).  With the per-kind mean times of
    a trace it predicts the trace's span, and with other times it answers
    what-if questions (a faster update, a faster panel, more workers).
    Returns the span and the busy fraction of the workers."""
    import heapq
    from collections import deque
    tasks, ndeps, ptr, succ = graph
    nt = len(tasks)
    dur = np.array([dur_by_kind[int(k)] for k in tasks[:, 0]], dtype=np.float64)
    lvl = [ready_level(int(kd), int(k), int(j)) for kd, _, j, k in tasks]
    left = ndeps.astype(np.int64).copy()
    queues = [deque() for _ in range(4)]
    for g in range(nt):
        if left[g] == 0:
            queues[lvl[g]].append(g)
    events = []
    now, free, done, seq, busy = 0.0, slots, 0, 0, 0.0
    while done < nt:
        while free > 0:
            q = next((q for q in queues if q), None)
            if q is None:
                break
            g = q.popleft()
            free -= 1
            busy += claim_s + dur[g]
            heapq.heappush(events, (now + claim_s + dur[g], seq, g))
            seq += 1
        if not events:
            raise ValueError("the graph has a cycle or a task that is never released")
        # every task ending now completes (in start order) before the
        # freed workers claim
        now = events[0][0]
        while events and events[0][0] == now:
            _, _, g = heapq.heappop(events)
            free += 1
            done += 1
            for v in succ[ptr[g]:ptr[g + 1]]:
                left[v] -= 1
                if left[v] == 0:
                    queues[lvl[v]].append(int(v))
    return {"span_s": float(now), "busy_fraction": float(busy / (slots * now)) if now > 0 else 1.0}


def to_chrome(records: np.ndarray, path: str, domain: int = 0) -> None:
    d = decode(records, domain)
    base = int(d["t0"].min())
    ev = []
    for n in range(len(d["t0"])):
        ev.append({"name": KINDS[d["kind"][n]], "ph": "X", "pid": 0, "tid": int(d["sm"][n]),
                   "ts": (int(d["t0"][n]) - base) / 1e3, "dur": (int(d["t1"][n]) - int(d["t0"][n])) / 1e3,
                   "args": {"k": int(d["k"][n]), "i": int(d["i"][n]), "j": int(d["j"][n])}})
    with open(path, "w") as fh:
        json.dump({"traceEvents": ev}, fh)
