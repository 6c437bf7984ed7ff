"""Host replay of the persistent kernel's scheduling protocol (csrc/sched.cuh)
under random delays: worker threads stand in for the CTAs, a lock makes each
of the device's atomic operations atomic, and random sleeps between the
operations and inside the tasks create interleavings the GPU's natural
timing rarely shows.  The graph is the library's own (tileqr_task_graph, the
graph the kernel executes, Sec. 4).

The protocol replayed step by step: per-task counters released by
atomicAdd, the call that completes a counter pushes the task onto its
priority level (atomicAdd on the tail, then a release store of code + 1 into
the write-once slot); a pop takes the highest non-empty level by CAS on the
head, except on the bulk level while more than TICKET_MARGIN tasks are
queued, where an atomicAdd on the head claims a slot that may still be
empty -- the worker's ticket, redeemed on a later pop.

Checked: every task runs exactly once, never before all of its
predecessors have finished, and every run ends (no stranded ticket, no lost
push); and a planted mistake in the protocol (a push at ndeps - 1, or a
ticket dropped when its slot is still empty) is caught."""
import random
import threading
import time

import numpy as np
import pytest

NKIND = 4
TICKET_MARGIN = 8


@pytest.fixture(scope="module")
def tq():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    tileqr.load()
    return tileqr


def _level(kind, k, j):
    base = kind if kind < 4 else (1 if kind == 4 else 2)
    return base - 1 if (kind in (2, 3, 5) and j == k + 1) else base


class Replay:
    def __init__(self, tasks, ndeps, ptr, succ, seed, mistake=None, push_lag=2e-5):
        self.n = len(tasks)
        self.ndeps = [int(x) for x in ndeps]
        self.succ = [[int(s) for s in succ[ptr[t]:ptr[t + 1]]] for t in range(self.n)]
        self.level = [_level(int(kd), int(k), int(j)) for kd, i, j, k in tasks]
        self.cap = [0] * NKIND
        for lv in self.level:
            self.cap[lv] += 1
        self.slot = [[0] * c for c in self.cap]
        self.head = [0] * NKIND
        self.tail = [0] * NKIND
        self.cnt = [0] * self.n
        self.completed = 0
        self.lock = threading.Lock()
        self.rng_seed = seed
        self.mistake = mistake
        self.push_lag = push_lag
        self.runs = [0] * self.n
        self.done_at = [None] * self.n
        self.start_at = [None] * self.n
        self.clock = 0
        self.errors = []

    # atomic operations of the device, made atomic by the lock
    def atomic_add(self, arr, idx, v):
        with self.lock:
            old = arr[idx]
            arr[idx] = old + v
            return old

    def cas(self, arr, idx, expect, new):
        with self.lock:
            old = arr[idx]
            if old == expect:
                arr[idx] = new
            return old

    def load(self, arr, idx):
        with self.lock:
            return arr[idx]

    def store(self, arr, idx, v):
        with self.lock:
            arr[idx] = v

    def tick(self):
        with self.lock:
            self.clock += 1
            return self.clock

    def push(self, t, rng):
        lv = self.level[t]
        s = self.atomic_add(self.tail, lv, 1)
        time.sleep(rng.random() * self.push_lag)   # the slot store lags the tail increment
        if s >= self.cap[lv]:
            self.errors.append("queue overflow")
            return
        self.store(self.slot[lv], s, t + 1)

    def signal(self, t, rng):
        old = self.atomic_add(self.cnt, t, 1)
        need = self.ndeps[t] - (1 if self.mistake == "early_push" else 0)
        if old + 1 == need:
            self.push(t, rng)

    def try_pop(self, w, rng):
        hd = [self.load(self.head, lv) for lv in range(NKIND)]
        tl = [self.load(self.tail, lv) for lv in range(NKIND)]
        for lv in range(NKIND):
            if lv == NKIND - 1 and w["ticket"] is not None:
                v = self.load(self.slot[lv], w["ticket"])
                if v == 0:
                    if self.mistake == "drop_ticket":
                        w["ticket"] = None
                    return None
                w["ticket"] = None
                return v - 1
            if hd[lv] >= self.cap[lv] or hd[lv] >= tl[lv]:
                continue
            if lv == NKIND - 1 and tl[lv] - hd[lv] > TICKET_MARGIN:
                t = self.atomic_add(self.head, lv, 1)
                if t >= self.cap[lv]:
                    return None
                for _ in range(4):
                    v = self.load(self.slot[lv], t)
                    if v:
                        return v - 1
                w["ticket"] = t
                return None
            while True:
                h = self.load(self.head, lv)
                if h >= self.cap[lv]:
                    break
                v = self.load(self.slot[lv], h)
                if v == 0:
                    break
                if self.cas(self.head, lv, h, h + 1) == h:
                    return v - 1
        return None

    def worker(self, wid, deadline):
        rng = random.Random(self.rng_seed * 1000 + wid)
        w = {"ticket": None}
        while time.monotonic() < deadline:
            t = self.try_pop(w, rng)
            if t is None:
                if self.load([self.completed], 0) >= self.n:
                    return
                time.sleep(rng.random() * 1e-5)
                continue
            self.start_at[t] = self.tick()
            self.runs[t] += 1
            time.sleep(rng.random() * 3e-5)      # the task itself
            self.done_at[t] = self.tick()
            for s in self.succ[t]:
                time.sleep(rng.random() * 5e-6)
                self.signal(s, rng)
            with self.lock:
                self.completed += 1

    def run(self, workers, timeout=30.0):
        rng = random.Random(self.rng_seed)
        for t in range(self.n):
            if self.ndeps[t] == 0:
                self.push(t, rng)
        deadline = time.monotonic() + timeout
        th = [threading.Thread(target=self.worker, args=(w, deadline)) for w in range(workers)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        return self


def _check(r, ptr, succ):
    assert not r.errors, r.errors
    assert r.completed == r.n and all(c == 1 for c in r.runs)
    for t in range(r.n):
        for s in succ[ptr[t]:ptr[t + 1]]:
            assert r.done_at[t] < r.start_at[int(s)]


@pytest.mark.parametrize("m,n,nb,h", [(640, 640, 64, 0), (1024, 384, 64, 0), (1280, 256, 64, 3),
                                      (768, 768, 128, 0)])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_protocol_runs_every_task_once_in_order(tq, m, n, nb, h, seed):
    tasks, ndeps, ptr, succ = tq.tileqr_task_graph(m, n, nb, h, 0)
    r = Replay(tasks, ndeps, ptr, succ, seed).run(workers=6)
    _check(r, ptr, succ)


def test_ticket_path_is_exercised(tq):
    """A wide graph keeps more than TICKET_MARGIN bulk tasks queued, so the
    atomicAdd claims (and their tickets) are really taken."""
    tasks, ndeps, ptr, succ = tq.tileqr_task_graph(512, 2048, 64, 0, 0)
    r = Replay(tasks, ndeps, ptr, succ, seed=7)
    orig = r.try_pop
    claims = {"n": 0}

    def counting(w, rng):
        before = r.load(r.head, NKIND - 1)
        out = orig(w, rng)
        if w["ticket"] is not None or r.load(r.head, NKIND - 1) > before:
            claims["n"] += 1
        return out
    r.try_pop = counting
    r.run(workers=8)
    _check(r, ptr, succ)
    assert claims["n"] > 0


@pytest.mark.parametrize("mistake", ["early_push", "drop_ticket"])
def test_planted_protocol_mistakes_are_caught(tq, mistake):
    tasks, ndeps, ptr, succ = tq.tileqr_task_graph(512, 2048, 64, 0, 0)
    caught = False
    for seed in range(1, 6):
        # slow pushes leave claimed bulk slots empty, so tickets are taken
        r = Replay(tasks, ndeps, ptr, succ, seed, mistake=mistake, push_lag=2e-3).run(workers=8, timeout=8.0)
        try:
            _check(r, ptr, succ)
        except AssertionError:
            caught = True
            break
    assert caught
