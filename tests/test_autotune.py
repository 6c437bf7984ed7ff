"""The autotuner's host logic (no GPU): shape signature, sampling, selection
of the fastest candidate, the cache (a hit times nothing; keys separate
devices, precisions and shape signatures) and the per-size-class plan,
all against a fake timer."""
import json

import pytest

from paper_0709_1272_gb300 import autotune, tileqr


class Shape:
    def __init__(self, m, n):
        self.shape = (m, n)


def _fake_timer(costs, calls):
    def timer(sub, nb, ib, precision):
        calls.append((len(sub), nb, ib, precision))
        return sum(costs(m, n, nb, ib) for m, n in (a.shape for a in sub))
    return timer


def test_signature_is_coarse_and_stable():
    a = [(1000, 700), (900, 650), (1100, 720), (64, 32)]
    b = [(1010, 690), (905, 640), (1090, 730), (66, 33)]
    assert autotune.signature(a) == autotune.signature(b)
    assert autotune.signature(a) != autotune.signature([(4000, 4000)] * 4)


def test_sampling_is_even_and_bounded():
    idx = autotune.sample_indices(4096, 256)
    assert len(idx) == 256 and idx[0] == 0 and idx[-1] == 4095
    gaps = {b - a for a, b in zip(idx, idx[1:])}
    assert max(gaps) - min(gaps) <= 1
    assert autotune.sample_indices(10, 256) == list(range(10))
    assert autotune.sample_indices(0, 256) == []


def test_selects_the_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("TILEQR_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    mats = [Shape(500 + 3 * i, 300 + i) for i in range(600)]
    calls = []
    # nb 128 / ib 32 is cheapest in this fake cost model
    cost = lambda m, n, nb, ib: m * n * (1.0 + abs(nb - 128) / 64 + (0.1 if ib == 16 else 0.0))
    nb, ib, ms = autotune.tune_batched(mats, tileqr.TILEQR_FP64, sample=64, timer=_fake_timer(cost, calls),
                                       device_name="fake-gpu")
    assert (nb, ib) == (128, 32)
    assert sorted(ms) == sorted(f"{a}/{b}" for a, b in autotune.CANDIDATES[tileqr.TILEQR_FP64])
    assert len(calls) == len(autotune.CANDIDATES[tileqr.TILEQR_FP64]) and all(c[0] == 64 for c in calls)
    # a second call with the same kind of batch is a cache hit: nothing timed
    calls.clear()
    assert autotune.tune_batched(mats, tileqr.TILEQR_FP64, sample=64, timer=_fake_timer(cost, calls),
                                 device_name="fake-gpu")[:2] == (128, 32)
    assert calls == []
    # another precision, device or shape signature is a miss
    autotune.tune_batched(mats, tileqr.TILEQR_TF32, sample=64, timer=_fake_timer(cost, calls),
                          device_name="fake-gpu")
    autotune.tune_batched(mats, tileqr.TILEQR_FP64, sample=64, timer=_fake_timer(cost, calls),
                          device_name="other-gpu")
    assert len(calls) == len(autotune.CANDIDATES[tileqr.TILEQR_TF32]) + len(autotune.CANDIDATES[tileqr.TILEQR_FP64])
    data = json.load(open(tmp_path / "tune.json"))
    assert len(data) == 3


def test_plan_splits_by_size_when_classes_prefer_different_nb(tmp_path, monkeypatch):
    monkeypatch.setenv("TILEQR_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    mats = [Shape(100, 80)] * 300 + [Shape(1500, 1400)] * 300
    # small matrices favour nb 64, large ones nb 128
    def cost(m, n, nb, ib):
        small = max(m, n) <= 512
        good = 64 if small else 128
        return m * n * (1.0 if nb == good else 2.0) * (1.0 if ib == 16 else 1.05)
    plan, est = autotune.plan_batched(mats, tileqr.TILEQR_FP64, sample=32, timer=_fake_timer(cost, []),
                                      device_name="fake-gpu")
    assert min(est, key=est.get) != 0
    got = {(len(idx), nb, ib) for idx, nb, ib in plan}
    assert got == {(300, 64, 16), (300, 128, 16)}
    # with one class preferring the same nb everywhere, the single launch wins
    cost1 = lambda m, n, nb, ib: m * n * (1.0 if nb == 128 else 2.0)
    plan1, est1 = autotune.plan_batched(mats, tileqr.TILEQR_FP64, sample=32, timer=_fake_timer(cost1, []),
                                        device_name="fake-gpu-2")
    assert len(plan1) == 1 or est1[0] <= min(est1.values()) + 1e-9
