"""Benchmark: plain FP64 tiled QR of a 16384 x 16384 N(0,1) matrix (nb 128,
ib 16) on one GB300 through libtileqr's C ABI, reported as Gflop/s with the
LAPACK operation count 2 n^2 (m - n/3) (the paper's rate convention, Sec. 5)
and as a fraction of the FP64 peak.

One step = one tileqr_factor call (layout conversion + the persistent task-
graph kernel) on an input resident in HBM.  The input (2.1 GB) is larger than
L2 (129 MB), so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank factors its own replica on its own GPU
(the factorization does not shard; weak scaling) and rank 0 prints one JSON
line with the max-over-ranks time.  --impl reference times the CPU oracle
(Algorithm 2 in plain C, one thread) on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tile-QR Gflop/s & % FP64 peak; mixed/batched speedup at ≤1e-12 LS error"
UNIT = "Gflop/s"
NSM = 152
FP64_FLOP_PER_CLK_PER_SM = 4   # 2 DFMA lanes per clock per SM (1.25 TFLOP/s nominal at 2.07 GHz)


def lapack_opcount(m, n):
    return 2.0 * n * n * (m - n / 3.0)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def tf32_peak_gflops():
    """Dense TF32 tensor peak of this GPU: the measured dense bf16 peak (burst)
    times the nominal tf32 / bf16 ratio (1.1 / 2.25 PFLOP/s)."""
    bf16 = float(measured_peaks().get("bf16_tflops", 1900.0))
    return bf16 * 1e3 * (1.1 / 2.25), f"measured bf16 dense {bf16:.1f} TFLOP/s x nominal tf32/bf16 1.1/2.25"


QR_SOURCES = ("common.cuh", "sched.cuh", "tile_f64.cuh", "dag.cuh", "release.cuh", "factor.cu")
LU_SOURCES = ("common.cuh", "sched.cuh", "graph.cuh", "release.cuh", "lu.cuh", "lu.cu")
CHOL_SOURCES = ("common.cuh", "sched.cuh", "graph.cuh", "chol.cuh", "cholesky.cu")


def kernel_source_hash(files=QR_SOURCES):
    h = hashlib.sha256()
    for rel in files:
        with open(os.path.join(ROOT, "paper_0709_1272_gb300", "csrc", rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def profiled_traffic(workload_key, profile="k_factor_dag_fp64.md", files=QR_SOURCES):
    """DRAM bytes per launch of a task-graph kernel from its committed ncu
    summary, if that was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", profile)
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"source_hash:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != kernel_source_hash(files):
        return None
    m = re.search(rf"traffic_bytes_per_launch\[{re.escape(workload_key)}\]:\s*([0-9.eE+]+)", txt)
    return float(m.group(1)) if m else None


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


CPU_SAMPLE_N = 4096


def _oracle_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(nb, ib, n_sample=CPU_SAMPLE_N):
    """The oracle as it stands on a bounded sample of the workload: Algorithm
    2's tasks run level by level of the task graph, each level spread over
    all host cores with OpenMP (oracle.tiled_qr_levels, identical bits to the
    sequential oracle)."""
    import oracle
    from paper_0709_1272_gb300 import inputs
    threads = _oracle_threads()
    A = inputs.normal_matrix(n_sample, n_sample, seed=20070709 + 2)
    t0 = time.perf_counter()
    _, nlev = oracle.tiled_qr_levels(A, nb, ib, threads)
    dt = time.perf_counter() - t0
    return {"value": lapack_opcount(n_sample, n_sample) / dt / 1e9, "unit": UNIT, "cores": threads,
            "kind": "oracle",
            "sample": f"oracle tiled QR (Algorithm 2, plain C -O2, the {nlev} levels of its task graph in turn, "
                      f"tasks of a level on {threads} OpenMP threads) of one {n_sample}x{n_sample} N(0,1) "
                      f"matrix, nb={nb}, ib={ib}: {dt:.1f} s"}


def run_reference(args, rank):
    """The reference arm: the oracle (there is no other implementation of
    this paper) on the host cores, one CPU_SAMPLE_N^2 sample per step --
    the same sample and build as the cpu_baseline of our arm."""
    if rank != 0:
        return 0
    import oracle
    from paper_0709_1272_gb300 import inputs
    n = args.ref_n
    threads = _oracle_threads()
    A = inputs.normal_matrix(n, n, seed=20070709 + 2)
    for _ in range(args.warmup):
        oracle.tiled_qr_levels(A, args.nb, args.ib, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, nlev = oracle.tiled_qr_levels(A, args.nb, args.ib, threads)
    dt = time.perf_counter() - t0
    value = args.steps * lapack_opcount(n, n) / dt / 1e9
    sample = (f"oracle tiled QR (Algorithm 2, plain C -O2, the {nlev} levels of its task graph in turn, tasks "
              f"of a level on {threads} OpenMP threads) of a {n}x{n} N(0,1) matrix per step, nb={args.nb}, "
              f"ib={args.ib} (bounded sample of the {args.n}x{args.n} workload)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": f"plain FP64 tile QR, {n}x{n} N(0,1), nb={args.nb}, ib={args.ib} "
                                  f"(sample of {args.n}x{args.n})", "parallelism": f"{threads} host threads"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_e2e(args, A_host, m, n, nb, ib, sched, ws, stream, dev, barrier, dist, world, ops):
    """The headline metric end to end through the C ABI with host buffers:
    per step, pinned host A -> device (cudaMemcpyAsync), tileqr_factor,
    tileqr_get_R, R -> pinned host.  Copies run on their own streams and
    overlap the previous / next step's factorization; the timed region spans
    the first input copy to the last result copy.  Also reports the copy
    rates measured alone."""
    import numpy as np
    import torch
    from paper_0709_1272_gb300 import replicas, tileqr
    k = min(m, n)
    A_pin = torch.from_numpy(np.ascontiguousarray(A_host.T)).pin_memory()   # (n, m) row-major == A col-major
    R_pin = [torch.empty((n, k), dtype=torch.float64).pin_memory() for _ in range(2)]
    A_dev = [torch.empty((n, m), dtype=torch.float64, device=dev) for _ in range(2)]
    R_dev = [torch.empty((n, k), dtype=torch.float64, device=dev) for _ in range(2)]
    h2d, d2h = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def copy_rate(dst, src, s):
        e0, e1 = ev(), ev()
        torch.cuda.synchronize()
        e0.record(s)
        with torch.cuda.stream(s):
            dst.copy_(src, non_blocking=True)
        e1.record(s)
        torch.cuda.synchronize()
        return src.numel() * 8 / (e0.elapsed_time(e1) / 1e3) / 1e9

    h2d_gbs = copy_rate(A_dev[0], A_pin, h2d)
    d2h_gbs = copy_rate(R_pin[0], R_dev[0], d2h)
    lib = tileqr.load()
    in_ready = [ev() for _ in range(2)]
    a_free = [ev() for _ in range(2)]
    r_ready = [ev() for _ in range(2)]
    r_free = [ev() for _ in range(2)]
    e0, e1 = ev(), ev()
    barrier()
    torch.cuda.synchronize()
    e0.record(h2d)
    for st in range(args.e2e_steps):
        b = st % 2
        if st >= 2:
            h2d.wait_event(a_free[b])        # step st-2 has read A_dev[b]
        with torch.cuda.stream(h2d):
            A_dev[b].copy_(A_pin, non_blocking=True)
        in_ready[b].record(h2d)
        stream.wait_event(in_ready[b])
        if st >= 2:
            stream.wait_event(r_free[b])     # R_dev[b] of step st-2 is on the host
        g = tileqr.tileqr_factor(A_dev[b].t(), nb, ib, schedule=sched, workspace=ws)
        a_free[b].record(stream)
        rc = lib.tileqr_get_R(tileqr.ctypes.byref(g.desc), tileqr.ctypes.c_void_p(R_dev[b].data_ptr()),
                              max(k, 1), tileqr.ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        r_ready[b].record(stream)
        d2h.wait_event(r_ready[b])
        with torch.cuda.stream(d2h):
            R_pin[b].copy_(R_dev[b], non_blocking=True)
        r_free[b].record(d2h)
    stream.wait_event(r_free[(args.e2e_steps - 1) % 2])
    if args.e2e_steps >= 2:
        stream.wait_event(r_free[(args.e2e_steps - 2) % 2])
    e1.record(stream)
    torch.cuda.synchronize()
    et = replicas.max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
    assert g.status() == 0
    return {"value": world * args.e2e_steps * ops / et / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": m * n * 8, "d2h_bytes_per_step": k * n * 8, "steps": args.e2e_steps,
            "h2d_gbs_alone": round(h2d_gbs, 1), "d2h_gbs_alone": round(d2h_gbs, 1),
            "path": "pinned host A -> cudaMemcpyAsync (copy stream) -> tileqr_factor -> tileqr_get_R -> "
                    "pinned host R (second copy stream); copies overlap the neighbouring steps' factorizations"}


def run_batched(args, dev, rank, world, barrier, dist):
    import numpy as np
    import torch

    from paper_0709_1272_gb300 import autotune, inputs, replicas, tileqr
    shapes = inputs.batch_shapes(args.batch_count, seed=20070709 + 5 + 1000 * rank)
    pool, offs = inputs.batch_pool(shapes, seed=20070709 + 5 + 1000 * rank)
    pool_d = torch.from_numpy(pool).to(dev)
    del pool
    mats = [pool_d[o:o + m * n].view(n, m).t() for (m, n), o in zip(shapes, offs)]
    flops = sum(2.0 * n * n * (m - n / 3.0) for (m, n) in shapes)

    def graph_time(bt, reps=2):
        bt.run()                                  # first call outside capture
        assert bt.status() == 0
        s = torch.cuda.Stream(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=s):
                bt.run(stream=s)
        g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        assert bt.status() == 0
        return replicas.max_over_ranks(e0.elapsed_time(e1) / 1e3 / reps, dist, dev)

    def loop_time(sub, nb, ib, precision):
        ws = torch.empty(max(tileqr.tileqr_workspace_size(a.shape[0], a.shape[1], nb, ib, precision)
                             for a in sub), dtype=torch.uint8, device=dev)
        for a in sub[:4]:
            tileqr.tileqr_factor(a, nb, ib, precision=precision, workspace=ws)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for a in sub:
            f = tileqr.tileqr_factor(a, nb, ib, precision=precision, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        assert f.status() == 0
        return e0.elapsed_time(e1) / 1e3

    # consistent right-hand sides b_k = A_k x_k (x_k N(0,1)), so that the
    # relative residual ||b - A x|| / ||b|| measures the solve's accuracy
    xpool = torch.from_numpy(inputs.normal_matrix(sum(n for _, n in shapes), 1,
                                                  seed=20070709 + 9 + 1000 * rank).reshape(-1)).to(dev)
    bs, xo = [], 0
    for (m, n), A in zip(shapes, mats):
        bs.append(A @ xpool[xo:xo + n])
        xo += n

    def solve_time(bt, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record()
        xs, info = bt.solve_ls(bs, max_iter=steps, tol=1e-14)
        e1.record()
        torch.cuda.synchronize()
        rel = max((torch.linalg.vector_norm(b - A @ x) / torch.linalg.vector_norm(b)).item()
                  for A, b, x in zip(mats, bs, xs))
        return replicas.max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev), rel, info

    out = {"workload": f"{len(shapes)} independent matrices, m ~ U[64,2048], n ~ U[32,m], entries U[-1,1)",
           "count": len(shapes), "flops": flops, "unit": UNIT, "timing": "CUDA-graph replay, events"}
    for label, prec in (("fp64", tileqr.TILEQR_FP64), ("tf32", tileqr.TILEQR_TF32)):
        nb, ib, tune_ms = autotune.tune_batched(mats, prec, sample=256)
        bt = tileqr.Batch(mats, nb, ib, prec)
        t = graph_time(bt)
        out[label] = {"value": world * flops / t / 1e9, "ms": t * 1e3, "nb": nb, "ib": ib,
                      "autotune_ms_on_sample": tune_ms}
        # FP64 factors: the plain solve (one step); TF32 factors: refined
        ts, rel, info = solve_time(bt, 1 if prec == tileqr.TILEQR_FP64 else 8)
        out[label]["solve"] = {"ms": ts * 1e3, "steps": info.iterations, "max_rel_residual": rel,
                               "method": "plain (Q^T b, R^-1)" if prec == tileqr.TILEQR_FP64 else
                               "augmented-system FP64 refinement"}
        del bt
        torch.cuda.empty_cache()
        k = min(args.loop_subset, len(mats))
        sub = mats[:k]
        sflops = sum(2.0 * n * n * (m - n / 3.0) for (m, n) in shapes[:k])
        tl = loop_time(sub, nb, ib, prec)
        tb = graph_time(tileqr.Batch(sub, nb, ib, prec))
        out[label]["loop_subset"] = {"count": k, "per_matrix_loop_ms": tl * 1e3, "batched_ms": tb * 1e3,
                                     "speedup": tl / tb, "loop_value": sflops / tl / 1e9,
                                     "batched_value": sflops / tb / 1e9}
        torch.cuda.empty_cache()
    out["tf32_speedup_vs_fp64"] = out["fp64"]["ms"] / out["tf32"]["ms"]
    # factor + solve, both at relative residual <= 1e-12
    f64 = out["fp64"]["ms"] + out["fp64"]["solve"]["ms"]
    f32 = out["tf32"]["ms"] + out["tf32"]["solve"]["ms"]
    out["solve_speedup_tf32_vs_fp64"] = {
        "value": f64 / f32, "fp64_ms": f64, "tf32_ms": f32,
        "both_at_rel_residual_1e-12": max(out["fp64"]["solve"]["max_rel_residual"],
                                          out["tf32"]["solve"]["max_rel_residual"]) <= 1e-12}
    tpk, tsrc = tf32_peak_gflops()
    out["tf32"]["pct_of_tf32_dense_peak"] = 100.0 * out["tf32"]["value"] / world / tpk
    out["tf32"]["tf32_peak_source"] = tsrc
    return out


def run_tall(args, dev, rank, world, barrier, dist):
    """Tall-skinny workload: 262144 x 512 N(0,1), nb 128, least squares with
    16 N(0,1) right-hand sides.  Algorithm 2's flat tree (a chain of p - 1
    DTSQRT per step) against the tree form (domains of 8 tile rows, heads
    merged pairwise), FP64 and with tensor-core updates."""
    import torch
    from paper_0709_1272_gb300 import inputs, replicas, tileqr
    m, n, nb = args.tall_m, 512, 128
    ops = lapack_opcount(m, n)
    A = tileqr.to_device_colmajor(inputs.normal_matrix(m, n, seed=20070709 + 3 + 1000 * rank), dev)
    B = tileqr.to_device_colmajor(inputs.normal_matrix(m, 16, seed=20070709 + 6 + 1000 * rank), dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        out = None
        best = float("inf")
        for _ in range(reps):
            barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            out = fn()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return replicas.max_over_ranks(best, dist, dev), out

    res = {"workload": f"tall-skinny tile QR, {m}x{n} N(0,1), nb={nb}; least squares with 16 N(0,1) "
                       f"right-hand sides", "unit": UNIT, "timing": "CUDA events, best of the timed runs, "
                       "max over ranks"}
    variants = [("fp64_flat", tileqr.TILEQR_FP64, 16, 0, 1), ("fp64_tree", tileqr.TILEQR_FP64, 16, 8, 3),
                ("tf32_tree", tileqr.TILEQR_TF32, 16, 16, 3)]
    facs = {}
    for label, prec, ib, h, reps in variants:
        ws = torch.empty(tileqr.tileqr_workspace_size_tree(m, n, nb, ib, prec, h), dtype=torch.uint8, device=dev)
        tileqr.tileqr_factor_tree(A, nb, ib, h, precision=prec, workspace=ws).check()   # warm-up
        t, f = timed(lambda: tileqr.tileqr_factor_tree(A, nb, ib, h, precision=prec, workspace=ws), reps)
        f.check()
        res[label] = {"ms": t * 1e3, "value": world * ops / t / 1e9, "ib": ib,
                      "domain": h if h > 0 else "flat (Algorithm 2)"}
        facs[label] = (f, ws)
    res["tree_speedup_fp64"] = res["fp64_flat"]["ms"] / res["fp64_tree"]["ms"]
    res["value"] = res["fp64_tree"]["value"]
    f = facs["fp64_tree"][0]
    t, X = timed(lambda: f.solve_ls(B.clone()), 3)
    r = B - A @ X
    ratio = (torch.linalg.matrix_norm(A.t() @ r) /
             (torch.linalg.matrix_norm(A) * torch.linalg.matrix_norm(r))).item()
    res["solve_ls_ms"] = t * 1e3
    res["ls_optimality"] = ratio   # ||A^T r|| / (||A|| ||r||)
    # TF32 tree factors + FP64 refinement on the augmented system: the
    # least-squares solution to FP64 accuracy
    ft = facs["tf32_tree"][0]
    t_r, (Xr, info) = timed(lambda: ft.solve_ls_refine(A, B, max_iter=10, tol=1e-14), 2)
    rr = B - A @ Xr
    opt_r = (torch.linalg.matrix_norm(A.t() @ rr) /
             (torch.linalg.matrix_norm(A) * torch.linalg.matrix_norm(rr))).item()
    res["tf32_tree_refined_ls"] = {
        "factor_ms": res["tf32_tree"]["ms"], "refine_ms": t_r * 1e3, "steps": info.iterations,
        "ls_optimality": opt_r,
        "x_vs_fp64_tree_solve": (torch.linalg.matrix_norm(Xr - X) / torch.linalg.matrix_norm(X)).item(),
        "speedup_vs_fp64_tree_factor_solve": (res["fp64_tree"]["ms"] + res["solve_ls_ms"]) /
                                             (res["tf32_tree"]["ms"] + t_r * 1e3)}
    del facs, A, B
    return res


def run_cholesky(args, dev, rank, world, barrier, dist):
    """Tiled Cholesky (Sec. 3.1, Algorithm 1): n x n SPD, (G + G^T)/2 + n I
    with G uniform[-1, 1), nb 128, FP64 task graph; rate with the n^3/3
    operation count."""
    import torch
    from paper_0709_1272_gb300 import inputs, replicas, tileqr
    n, nb = args.n, 128
    A = tileqr.to_device_colmajor(inputs.spd_matrix(n, seed=20070709 + 7 + 1000 * rank), dev)
    ws = torch.empty(tileqr.tileqr_cholesky_workspace_size(n, nb), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    tileqr.tileqr_cholesky(A, nb, workspace=ws).check()   # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(2, min(args.steps, 3))
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        f = tileqr.tileqr_cholesky(A, nb, workspace=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    f.check()
    t = replicas.max_over_ranks(e0.elapsed_time(e1) / 1e3 / reps, dist, dev)
    ops = n ** 3 / 3.0
    peaks = measured_peaks()
    fp64_peak = NSM * FP64_FLOP_PER_CLK_PER_SM * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e9
    del A, ws
    roof = {"bound": "alu", "achieved": ops / t / 1e9, "peak": fp64_peak, "unit": "GFLOP/s",
            "frac": ops / t / 1e9 / fp64_peak,
            "traffic": profiled_traffic(f"{n}x{n}/nb{nb}", "k_chol_dag_fp64.md", CHOL_SOURCES),
            "kernel": f"k_chol_dag<{nb}>",
            "achieved_flops": "n^3/3 per factorization (the algorithm's own count) / its CUDA-event time"}
    return {"workload": f"tiled Cholesky (Algorithm 1), {n}x{n} SPD (G+G^T)/2 + nI, G uniform[-1,1), nb={nb}, "
                        f"FP64 task graph", "value": world * ops / t / 1e9, "unit": UNIT, "ms_per_step": t * 1e3,
            "steps": reps, "pct_fp64_peak": 100.0 * (ops / t / 1e9) / fp64_peak, "roofline": roof,
            "timing": "CUDA events around the factorizations (layout conversion included), max over ranks"}


def run_lu(args, dev, rank, world, barrier, dist):
    """Tiled LU with tiled pairwise pivoting (Sec. 3.2.2, Algorithm 3): n x n
    N(0,1), nb 128, ib 16, FP64 task graph; rate with LU's 2n^3/3 operation
    count (the algorithm performs (1 + ib/(2nb)) times that, Sec. 3.2.3).
    Accuracy as in Sec. 3.2.4: the solve's backward error ||b - A x||_inf /
    (||A||_inf ||x||_inf) and the growth ||U||_inf / ||A||_inf, at this size
    and at n = 2048 for the tile counts the library builds (p = 16, 32)."""
    import torch
    from paper_0709_1272_gb300 import replicas, tileqr
    n, nb, ib = args.n, 128, 16
    g = torch.Generator(device=dev).manual_seed(20070709 + 8 + 1000 * rank)
    A = torch.randn((n, n), generator=g, dtype=torch.float64, device=dev).t()
    ws = torch.empty(tileqr.tileqr_lu_workspace_size(n, nb, ib), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    tileqr.tileqr_lu(A, nb, ib, workspace=ws).check()   # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(2, min(args.steps, 3))
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        f = tileqr.tileqr_lu(A, nb, ib, workspace=ws)
    e1.record(stream)
    torch.cuda.synchronize()
    f.check()
    info = f.info()
    t = replicas.max_over_ranks(e0.elapsed_time(e1) / 1e3 / reps, dist, dev)
    ops = 2.0 * n ** 3 / 3.0
    peaks = measured_peaks()
    fp64_peak = NSM * FP64_FLOP_PER_CLK_PER_SM * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e9
    inf = lambda M: M.abs().sum(dim=1).max().item()

    def accuracy(Am, fm):
        B = torch.randn((Am.shape[0], 4), generator=g, dtype=torch.float64, device=dev)
        X = fm.solve(B)
        U = torch.triu(fm.factors()[0])
        nA = inf(Am)
        return inf(B - Am @ X) / (nA * inf(X)), inf(U) / nA

    be, growth = accuracy(A, f)
    del ws
    sweep = {}
    for nbs in (128, 64):
        n2 = 2048
        bes, grs = [], []
        for smp in range(5):
            A2 = torch.randn((n2, n2), generator=g, dtype=torch.float64, device=dev).t()
            f2 = tileqr.tileqr_lu(A2, nbs, 16).check()
            b2, g2 = accuracy(A2, f2)
            bes.append(b2)
            grs.append(g2)
        sweep[f"p={n2 // nbs}"] = {"n": n2, "nb": nbs, "ib": 16, "samples": 5,
                                   "solve_backward_mean": sum(bes) / len(bes), "solve_backward_max": max(bes),
                                   "growth_U_mean": sum(grs) / len(grs)}
    del A, f
    alg = ops * (1.0 + ib / (2.0 * nb))
    roof = {"bound": "alu", "achieved": alg / t / 1e9, "peak": fp64_peak, "unit": "GFLOP/s",
            "frac": alg / t / 1e9 / fp64_peak,
            "traffic": profiled_traffic(f"{n}x{n}/nb{nb}/ib{ib}", "k_lu_dag_fp64.md", LU_SOURCES),
            "kernel": f"k_lu_dag<{nb},{ib}>",
            "achieved_flops": "(2n^3/3)(1+ib/(2nb)) per factorization / its CUDA-event time"}
    return {"workload": f"tiled LU with tiled pairwise pivoting (Algorithm 3), {n}x{n} N(0,1), nb={nb}, ib={ib}, "
                        f"FP64 task graph", "value": world * ops / t / 1e9, "unit": UNIT, "ms_per_step": t * 1e3,
            "steps": reps, "pct_fp64_peak": 100.0 * (ops / t / 1e9) / fp64_peak,
            "algorithmic_gflops": (ops * (1.0 + ib / (2.0 * nb))) / t / 1e9,
            "zero_pivot_info": info, "solve_backward_error": be, "growth_U": growth,
            "stability_n2048": sweep, "roofline": roof,
            "timing": "CUDA events around the factorizations (layout conversion included), max over ranks"}


def run_fp64_peak(args, dev, rank, world, barrier, dist):
    """The FP64 rates behind the roofline denominator: the library's DFMA and
    FP64 mma.sync microbenchmarks (tileqr_measure_fp64_rates), five runs
    each, with the SM clock sampled while they run; the nominal DFMA peak
    152 SMs x 4 flop/clk x clock follows from the clock."""
    import torch
    from paper_0709_1272_gb300 import tileqr
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = "0"
    clocks = ClockSampler(gpu_id)
    clocks.start()
    time.sleep(0.3)
    runs = [tileqr.tileqr_measure_fp64_rates() for _ in range(5)]
    clk = clocks.stop()
    dfma = max(r[0] for r in runs)
    dmma = max(r[1] for r in runs)
    mhz = clk.get("sm_mhz") or float(measured_peaks().get("sm_max_mhz", 2070.0))
    return {"dfma_gflops": dfma, "dmma_gflops": dmma, "runs": runs, "clocks": clk,
            "dfma_flop_per_clk_per_sm": dfma * 1e9 / (NSM * mhz * 1e6),
            "dfma_at_2070_mhz": dfma * 2070.0 / mhz}


def run_config2_sweep(args, dev, rank, world, barrier, dist):
    """16384^2 N(0,1) factorization rate for nb in {128, 256} x ib in {16, 32}
    with the persistent task-graph kernel, and the fork-join comparator (one
    launch per step and task kind) at nb 128 / ib 16; one timed run each after
    a warm-up (opt-in: about a minute)."""
    import torch
    from paper_0709_1272_gb300 import inputs, replicas, tileqr
    m = n = args.n
    A = tileqr.to_device_colmajor(inputs.normal_matrix(m, n, seed=20070709 + 1 + 1000 * rank), dev)
    ops = lapack_opcount(m, n)
    out = {}
    for nb, ib, sched in [(128, 16, "dag"), (128, 32, "dag"), (256, 16, "dag"), (256, 32, "dag"),
                          (128, 16, "bulk")]:
        sc = tileqr.TILEQR_SCHED_DAG if sched == "dag" else tileqr.TILEQR_SCHED_BULK
        ws = torch.empty(tileqr.tileqr_workspace_size(m, n, nb, ib), dtype=torch.uint8, device=dev)
        tileqr.tileqr_factor(A, nb, ib, schedule=sc, workspace=ws).check()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record()
        f = tileqr.tileqr_factor(A, nb, ib, schedule=sc, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        f.check()
        t = replicas.max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
        out[f"{sched}_nb{nb}_ib{ib}"] = {"value": world * ops / t / 1e9, "ms": t * 1e3}
        del ws, f
    return {"workload": f"plain FP64 tile QR, {m}x{n} N(0,1): task graph vs fork-join, nb x ib sweep",
            "unit": UNIT, "runs": out}


def kappa_device_matrix(n, kappa, seed, dev):
    """inputs.kappa_matrix formed on the device from the same (s, u, v):
    A = (I-2uu^T) diag(s) (I-2vv^T) = D - 2 u (Du)^T - 2 (Dv) v^T + 4 c u v^T
    with c = u^T D v, built as its transpose in row-major memory, which is A
    in column-major order (the layout the library reads)."""
    import torch
    from paper_0709_1272_gb300 import inputs
    s, u, v = inputs.kappa_factors(n, kappa, seed)
    c = float(u @ (s * v))
    st, ut, vt = (torch.from_numpy(x).to(dev) for x in (s, u, v))
    At = torch.diag(st)
    At.addr_(st * ut, ut, alpha=-2.0)
    At.addr_(vt, st * vt, alpha=-2.0)
    At.addr_(vt, ut, alpha=4.0 * c)
    return At.t()


def run_kappa_sweep(args, dev, rank, world, barrier, dist, fp64_factor_ms=None):
    """The mixed-precision solve of A x = b (TF32 tensor-core updates + FP64
    refinement) for cond(A) in {1e2, 1e6, 1e10}, A = (I-2uu^T) diag(s)
    (I-2vv^T) at --n, against the plain FP64 factorization + solve of the
    same system.  Per kappa: factorization and refinement time, steps,
    method, the solve's relative residual and forward error, the
    factorization's backward error ||Q^T a_j - r_j|| / ||A|| over 64 sampled
    columns, and R's first two tile columns against the CPU oracle (FP64
    Algorithm 2 of A's first 256 columns)."""
    import numpy as np
    import torch
    import oracle
    from paper_0709_1272_gb300 import inputs, replicas, tileqr
    n = args.n
    nb, ib = 128, 16
    g = torch.Generator(device=dev).manual_seed(20070709 + 5)
    cols = torch.randperm(n, generator=g, device=dev)[:64].sort().values
    xt = torch.from_numpy(inputs.normal_matrix(n, 1, seed=20070709 + 6)).to(dev).reshape(-1)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return replicas.max_over_ranks(e0.elapsed_time(e1), dist, dev), out

    wsm = torch.empty(tileqr.tileqr_workspace_size(n, n, nb, ib, tileqr.TILEQR_TF32), dtype=torch.uint8,
                      device=dev)
    per, fp64 = [], {}
    for kappa in (1e2, 1e6, 1e10):
        seed = 20070709 + 4 + 1000 * rank
        A = kappa_device_matrix(n, kappa, seed, dev)
        b = A @ xt
        if not per:
            tileqr.tileqr_factor(A, nb, ib, precision=tileqr.TILEQR_TF32, workspace=wsm).check()   # warm-up
        t_f, fm = timed(lambda: tileqr.tileqr_factor(A, nb, ib, precision=tileqr.TILEQR_TF32, workspace=wsm))
        fm.check()
        t_r, (x, info) = timed(lambda: fm.solve_refine(A, b, max_iter=40, tol=1e-12))
        d = info.as_dict()
        nA = torch.linalg.matrix_norm(A).item()
        QtA = fm.apply_qt(A[:, cols].contiguous().t().contiguous().t())
        R = fm.R()
        back = torch.linalg.matrix_norm(QtA - R[:, cols]).item() / nA * np.sqrt(n / 64.0)
        fwd = (torch.linalg.vector_norm(x - xt) / torch.linalg.vector_norm(xt)).item()
        r_gpu = R[:256, :256].cpu().numpy()
        ref = oracle.tiled_qr(inputs.kappa_columns(n, kappa, seed, 0, 256), nb, ib)
        r_err = float(np.linalg.norm(oracle.sign_normalize(r_gpu) - oracle.sign_normalize(ref.R())) /
                      np.linalg.norm(ref.R()))
        per.append({"kappa": f"{kappa:.0e}", "factor_ms": round(t_f, 2), "refine_ms": round(t_r, 2),
                    "steps": d["iterations"], "method": {1: "classical", 2: "fgmres"}.get(d["method"], "none"),
                    "rel_res": d["rel_residual"], "fwd_err": fwd, "back_err": back, "r256_vs_oracle": r_err})
        if kappa == 1e10:
            # the plain FP64 path on the hardest system: factorization + solve
            del fm, wsm, QtA
            torch.cuda.empty_cache()
            ws64 = torch.empty(tileqr.tileqr_workspace_size(n, n, nb, ib), dtype=torch.uint8, device=dev)
            t64, f64 = timed(lambda: tileqr.tileqr_factor(A, nb, ib, workspace=ws64))
            f64.check()
            ts, X = timed(lambda: f64.solve_ls(b.reshape(-1, 1).clone()))
            rr = (torch.linalg.vector_norm(b - A @ X[:n, 0]) / torch.linalg.vector_norm(b)).item()
            fp64 = {"factor_ms": round(t64, 1), "solve_ms": round(ts, 2), "rel_res": rr}
            del f64, ws64, X
        del A, b, x, R
        torch.cuda.empty_cache()
    t64_total = fp64["factor_ms"] + fp64["solve_ms"]
    for e in per:
        e["speedup_vs_fp64"] = round(t64_total / (e["factor_ms"] + e["refine_ms"]), 2)
    return {"workload": f"A x = b, {n}x{n}, A = (I-2uu^T)diag(s)(I-2vv^T), s geometric 1..1/kappa; "
                        f"TF32 updates + FP64 refinement to 1e-12 vs FP64 factor + solve",
            "fp64_kappa1e10": fp64, "per_kappa": per}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=16384)
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--nb", type=int, default=128)
    ap.add_argument("--ib", type=int, default=16)
    ap.add_argument("--schedule", default="dag", choices=["dag", "bulk"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--ref-n", type=int, default=CPU_SAMPLE_N)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision + FP64 refinement measurement")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched (4096 ragged matrices) measurement")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--no-cholesky", action="store_true",
                    help="skip the tiled Cholesky (Algorithm 1) measurement")
    ap.add_argument("--only", choices=["lu", "cholesky", "batched", "tall", "config2-sweep", "kappa-sweep",
                                       "fp64-peak"],
                    default=None,
                    help="run only this secondary measurement (at --n) and print its JSON object")
    ap.add_argument("--no-lu", action="store_true",
                    help="skip the tiled LU (Algorithm 3) measurement")
    ap.add_argument("--no-tall", action="store_true",
                    help="skip the tall-skinny (262144 x 512, flat vs tree) measurement")
    ap.add_argument("--tall-m", type=int, default=262144)
    ap.add_argument("--loop-subset", type=int, default=512)
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import numpy as np
    import torch

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    from paper_0709_1272_gb300 import build, inputs, replicas, tileqr
    build.build()
    tileqr.load()
    sched = tileqr.TILEQR_SCHED_DAG if args.schedule == "dag" else tileqr.TILEQR_SCHED_BULK
    m, n, nb, ib = args.m, args.n, args.nb, args.ib

    if args.only:
        # one secondary measurement alone (its JSON object on one line), e.g.
        # for a profiler run of that path
        def barrier():
            if dist is not None:
                dist.barrier()
        section = {"lu": run_lu, "cholesky": run_cholesky, "batched": run_batched, "tall": run_tall,
                   "fp64-peak": run_fp64_peak,
                   "config2-sweep": run_config2_sweep,
                   "kappa-sweep": run_kappa_sweep}[args.only](args, dev, rank, world, barrier, dist)
        if rank == 0:
            print(json.dumps({"section": args.only, **section}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return 0

    A_host = inputs.normal_matrix(m, n, seed=20070709 + 1 + 1000 * rank)
    A = tileqr.to_device_colmajor(A_host, dev)
    ws = torch.empty(tileqr.tileqr_workspace_size(m, n, nb, ib), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    for w in range(max(args.warmup, 1)):
        f = tileqr.tileqr_factor(A, nb, ib, schedule=sched, workspace=ws)
        if w == 0:
            f.check()
    torch.cuda.synchronize()

    # ---- device-resident timed region
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for e in ev_b + ev_a:
        e.record(stream)    # creates the CUDA events before the timed region
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local)
    clocks = ClockSampler(gpu_id)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    tileqr.tileqr_reset_launch_count()
    t_start.record(stream)
    for s in range(args.steps):
        tileqr.tileqr_set_profile_events(ev_b[s], ev_a[s])
        f = tileqr.tileqr_factor(A, nb, ib, schedule=sched, workspace=ws)
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = tileqr.tileqr_launch_count()
    tileqr.tileqr_set_profile_events(None, None)
    clk = clocks.stop()
    barrier()
    status = f.status()
    if status != 0:
        raise SystemExit(f"factorization failed: {tileqr.strerror(status)}")
    elapsed = t_start.elapsed_time(t_end) / 1e3
    dag_times = [ev_b[s].elapsed_time(ev_a[s]) / 1e3 for s in range(args.steps)]
    elapsed = replicas.max_over_ranks(elapsed, dist, dev)
    ops = lapack_opcount(m, n)
    value = world * args.steps * ops / elapsed / 1e9

    # ---- end to end through the public API: pinned host A in, R out.  Two
    # device buffers each for A and R and two copy streams, so the copy of
    # step k+1's input and of step k-1's R run while step k factors.
    e2e = None
    if args.e2e_steps > 0:
        e2e = run_e2e(args, A_host, m, n, nb, ib, sched, ws, stream, dev, barrier, dist, world, ops)

    # ---- mixed precision (tcgen05 updates) + FP64 iterative refinement of the
    # solve A x = b for cond(A) 1e2 / 1e6 / 1e10 at the same order, against
    # the plain FP64 factorization + solve of the same system
    mixed = None
    if not args.no_mixed and m == n and nb == 128:
        del ws
        torch.cuda.empty_cache()
        mixed = run_kappa_sweep(args, dev, rank, world, barrier, dist)

    # ---- batched: 4096 independent matrices, m ~ U[64, 2048], n ~ U[32, m],
    # entries U[-1, 1), one persistent launch replayed from a CUDA graph
    batched = None
    if not args.no_batched:
        torch.cuda.empty_cache()
        batched = run_batched(args, dev, rank, world, barrier, dist)

    # ---- tiled Cholesky (Algorithm 1) on an SPD matrix of the same order
    chol = None
    if not args.no_cholesky and m == n:
        torch.cuda.empty_cache()
        chol = run_cholesky(args, dev, rank, world, barrier, dist)

    # ---- tiled LU with tiled pairwise pivoting (Algorithm 3), same order
    lu = None
    if not args.no_lu and m == n:
        torch.cuda.empty_cache()
        lu = run_lu(args, dev, rank, world, barrier, dist)

    # ---- tall-skinny 262144 x 512: flat tree vs tree form
    tall = None
    if not args.no_tall:
        torch.cuda.empty_cache()
        tall = run_tall(args, dev, rank, world, barrier, dist)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp64_peak = NSM * FP64_FLOP_PER_CLK_PER_SM * sm_max * 1e6 / 1e9   # GFLOP/s
    alg_flops = ops * (1.0 + ib / (4.0 * nb))   # work the algorithm performs (Sec. 3.2.3)
    dag_mean = statistics.mean(dag_times)
    achieved = alg_flops / dag_mean / 1e9
    wl_key = f"{m}x{n}/nb{nb}/ib{ib}"
    traffic = profiled_traffic(wl_key)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"plain FP64 tile QR, {m}x{n} N(0,1), nb={nb}, ib={ib}, "
                               f"{'persistent task-graph kernel' if sched == 0 else 'fork-join per-step launches'}",
                   "m": m, "n": n, "nb": nb, "ib": ib, "schedule": args.schedule,
                   "l2": "input (%.1f GB) and tiles larger than L2 (129 MB); no flush" % (m * n * 8 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "pct_fp64_peak": 100.0 * (value / world) / fp64_peak,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "GFLOP/s",
                     "frac": achieved / fp64_peak, "traffic": traffic,
                     "kernel": f"k_factor_dag<{nb},{ib}>",
                     "peak_source": f"FP64 DFMA: {NSM} SMs x {FP64_FLOP_PER_CLK_PER_SM} flop/clk x "
                                    f"{sm_max:.0f} MHz (sm_max_mhz of measured peaks)",
                     "achieved_flops": "2n^2(m-n/3)(1+ib/(4nb)) per launch / mean launch time (CUDA events)"},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if e2e:
        out["e2e"] = e2e
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(nb, ib)
    # the secondary workloads, the mixed-precision sweep last: a reader that
    # keeps only the end of the line still sees it
    if chol:
        out["cholesky"] = chol
    if lu:
        out["lu"] = lu
    if tall:
        out["tall_skinny"] = tall
    if batched:
        out["batched"] = batched
    if mixed:
        out["mixed_ls"] = mixed
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
