"""Autotuner for the tile size nb and inner block size ib.

The paper tunes b (~200) and s (20-40) by hand for its Opterons (Sec. 5) and
notes the trade-off: small s keeps the s/(4b) extra flops low, too small s
hurts the kernels' efficiency (Sec. 3.2.3).  On GB300 the answer depends on
the precision and on the shapes, so the choice is measured: every built
(nb, ib) for the precision is timed on an evenly spaced sample of the batch
(or on the matrix itself), and the fastest is cached in a JSON file keyed by
GPU name, precision and a coarse shape signature.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import tileqr

CANDIDATES = {
    tileqr.TILEQR_FP64: [(64, 16), (128, 16), (128, 32), (256, 16)],
    tileqr.TILEQR_TF32: [(128, 16), (128, 32)],
}


def _cache_path() -> str:
    p = os.environ.get("TILEQR_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "tileqr", "autotune.json")


def _load_cache():
    try:
        with open(_cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store_cache(cache):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def signature(shapes) -> str:
    """Coarse description of a set of shapes: count (log2 bucket) and the
    quartiles of m and n rounded to powers of two."""
    ms = np.array([s[0] for s in shapes], dtype=np.float64)
    ns = np.array([s[1] for s in shapes], dtype=np.float64)

    def q(v):
        return [int(2 ** round(np.log2(max(x, 1.0)))) for x in np.percentile(v, [25, 50, 75])]

    return f"c{int(2 ** round(np.log2(max(len(shapes), 1))))}_m{q(ms)}_n{q(ns)}"


def _time_batch(mats, nb, ib, precision, reps=2):
    bt = tileqr.Batch(mats, nb, ib, precision)
    bt.run()
    if bt.status() != 0:
        return float("inf")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        bt.run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def sample_indices(count: int, sample: int):
    """An evenly spaced sample of a batch (indices into it, increasing)."""
    if count == 0:
        return []
    idx = np.linspace(0, count - 1, num=min(sample, count)).round().astype(int)
    return sorted(set(idx.tolist()))


def tune_batched(mats, precision=tileqr.TILEQR_FP64, sample: int = 256, use_cache: bool = True, timer=None,
                 device_name: str | None = None):
    """(nb, ib, {candidate: ms on the sample}) for a batch of column-major
    CUDA tensors (or anything with a .shape, with a custom timer).

    Every built (nb, ib) of the precision is timed on an evenly spaced sample
    of the batch by timer(sub, nb, ib, precision) -> ms (default: one
    batched launch on the GPU); the fastest wins and is cached under
    (device name, precision, shape signature), so a later call with the same
    kind of batch times nothing.  The update task's tile shape is nb x nb
    (Algorithm 2's square tiles), so nb fixes it: there is no separate
    tile-shape dimension to search."""
    timer = timer or _time_batch
    shapes = [tuple(a.shape) for a in mats]
    name = device_name if device_name is not None else torch.cuda.get_device_name()
    key = f"{name}|p{precision}|batched|{signature(shapes)}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        c = cache[key]
        return c["nb"], c["ib"], c.get("ms", {})
    sub = [mats[i] for i in sample_indices(len(mats), sample)]
    timings = {}
    for nb, ib in CANDIDATES[precision]:
        timings[f"{nb}/{ib}"] = timer(sub, nb, ib, precision)
    best = min(timings, key=timings.get)
    nb, ib = (int(x) for x in best.split("/"))
    if use_cache:
        cache[key] = {"nb": nb, "ib": ib, "ms": timings}
        _store_cache(cache)
    return nb, ib, timings


def split_by_size(shapes, bound: int):
    """Indices of the matrices with max(m, n) <= bound, and of the rest."""
    small = [i for i, (m, n) in enumerate(shapes) if max(m, n) <= bound]
    large = [i for i, (m, n) in enumerate(shapes) if max(m, n) > bound]
    return small, large


def plan_batched(mats, precision=tileqr.TILEQR_FP64, bounds=(0, 256, 512, 1024), sample: int = 256,
                 use_cache: bool = True, timer=None, device_name: str | None = None):
    """A per-size-class choice of (nb, ib): for each split bound, the small
    and the large matrices are tuned separately (tune_batched on each class)
    and the plan's time is the sum of the two classes' sample times scaled to
    the classes' shares of the batch (two persistent launches, one after the
    other); bound 0 is the single launch.  Returns the fastest plan as a list
    of (indices, nb, ib) and the table of estimated times."""
    shapes = [tuple(a.shape) for a in mats]
    est, plans = {}, {}
    for bound in bounds:
        parts = [list(range(len(mats)))] if bound == 0 else [p for p in split_by_size(shapes, bound) if p]
        total, plan = 0.0, []
        for part in parts:
            sub = [mats[i] for i in part]
            nb, ib, ms = tune_batched(sub, precision, sample, use_cache, timer, device_name)
            share = len(part) / max(len(sample_indices(len(part), sample)), 1)
            total += ms[f"{nb}/{ib}"] * share
            plan.append((part, nb, ib))
        est[bound] = total
        plans[bound] = plan
    best = min(est, key=est.get)
    return plans[best], est
