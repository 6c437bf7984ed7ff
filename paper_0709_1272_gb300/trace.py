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


def summary(records: np.ndarray, domain: int = 0) -> dict:
    d = decode(records, domain)
    t_begin, t_end = int(d["t0"].min()), int(d["t1"].max())
    wall = (t_end - t_begin) * 1e-9
    dur = (d["t1"] - d["t0"]) * 1e-9
    nsm = int(d["sm"].max()) + 1
    out = {"tasks": int(len(dur)), "wall_s": wall, "busy_fraction": float(dur.sum() / (wall * nsm)),
           "per_kind": {}}
    for kd, name in enumerate(KINDS):
        sel = d["kind"] == kd
        if sel.any():
            out["per_kind"][name] = {"count": int(sel.sum()), "mean_us": float(dur[sel].mean() * 1e6),
                                     "total_sm_s": float(dur[sel].sum())}
    return out


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
