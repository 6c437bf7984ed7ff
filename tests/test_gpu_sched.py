"""The device scheduler (Sec. 4 task graph) checked from its own trace: every
task of Algorithm 2 runs exactly once, and no task starts before all of its
predecessors (the dependency table of Sec. 4, derived independently by the
oracle's read/write analysis) have finished."""
import numpy as np
import pytest
import torch

import oracle
from paper_0709_1272_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tq():
    from paper_0709_1272_gb300 import build
    build.build()
    from paper_0709_1272_gb300 import tileqr
    tileqr.load()
    return tileqr


@pytest.mark.parametrize("m,n,nb,ib", [(1280, 1024, 128, 16), (640, 1500, 64, 16), (3000, 600, 256, 32)])
def test_trace_respects_dependencies(tq, m, n, nb, ib):
    from paper_0709_1272_gb300 import trace
    A = inputs.normal_matrix(m, n, seed=4242)
    Ad = tq.to_device_colmajor(A)
    tasks, preds = oracle.dependencies(m, n, nb)
    rec = torch.zeros((len(tasks) + 16, 4), dtype=torch.int64, device="cuda")
    tq.tileqr_set_trace(rec)
    try:
        f = tq.tileqr_factor(Ad, nb, ib).check()
        cnt = tq.tileqr_trace_count(f)
    finally:
        tq.tileqr_set_trace(None)
    assert cnt == len(tasks)
    d = trace.decode(rec[:cnt].cpu().numpy())
    kinds = {0: oracle.TASK_GEQRT, 1: oracle.TASK_TSQRT, 2: oracle.TASK_LARFB, 3: oracle.TASK_SSRFB}
    seen = {}
    for n_ in range(cnt):
        key = (kinds[int(d["kind"][n_])], int(d["i"][n_]), int(d["j"][n_]), int(d["k"][n_]))
        assert key not in seen, f"task {key} ran twice"
        seen[key] = (int(d["t0"][n_]), int(d["t1"][n_]))
    assert set(seen) == set(tasks)
    for t in tasks:
        for pr in preds[t]:
            assert seen[pr][1] <= seen[t][0], f"{t} started before its predecessor {pr} finished"
    s = trace.summary(rec[:cnt].cpu().numpy())
    assert s["tasks"] == cnt and 0 < s["busy_fraction"] <= 1.0
