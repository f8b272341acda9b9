#!/usr/bin/env python
"""Benchmark of the GB300 column-ID hot path.

Workload (one step = one full ID: sketch -> pivoted QR -> coefficient solve):
A = U diag(sigma) V^T, 20000 x 2000 FP64, sigma_i = i^-2 (seeded orthonormal
U, V); Gaussian Omega of 110 x 20000 rounded to bfloat16; rank k = 100.
The headline form is the matched-error one (d = ||A_hat_M - A_hat_D||_2 /
||A||_2 <= 1e-6 against the plain FP64 GPU ID): A scaled by powers of two and
split into three bfloat16 pieces, sketched on the tensor cores with FP32
accumulation, FP32 pivoted QR of Y, FP64 T solve with one refinement step.
Inputs stay resident in HBM for the timed loop (A is 320 MB, larger than the
129 MB L2, so no flush is needed); `e2e` repeats the measurement with A and
Omega copied from pinned host memory each step (double-buffered: the copy of
the next ID overlaps the current one's compute) and the result read back.

Also reported: the plain FP64 GPU ID on the same matrix and Omega (FP64
sketch by DFMA), the single-piece bfloat16 sketch (faster, not at matched
error), their errors, the roofline of the dominant kernel against peaks
measured in the same run, sampled SM clocks, the other workloads (plain FP64
ID of a 1000 x 500 matrix, the 65536 x 1000 snapshot matrix at tolerance
1e-6, the 512-matrix uneven batch, the differentiable 64 x 2048 x 512 batch)
and the FP64 CPU oracle timed on the host (`cpu_baseline`).  `--impl
reference` times the oracle alone as the reference arm.

Under torchrun (N > 1) every rank runs its own IDs (independent problems, no
collective on the data path); value = all ranks' IDs / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IDs/sec and effective TFLOP/s, mixed vs plain FP64 GPU ID at rel.err ≤1e-6"
M, N, K, P = 20000, 2000, 100, 10
INFLIGHT = 8        # IDs in flight in the timed stream of IDs
INFLIGHT_GROUPS = 2  # graphs the in-flight IDs are issued as, replayed in turn on their own streams
ELL = K + P
WORKLOAD = ("randomized column ID, A 20000x2000 FP64 (sigma_i = i^-2, seeded orthonormal factors), "
            "Gaussian Omega 110x20000, rank k=100")


def id_flops(m, n, ell, k, sketch=True):
    """Algorithmic flops of one ID: sketch 2 ell m n, truncated Householder CPQR on the
    r x n pivoted matrix 4rnk - 2k^2(r+n) + 4k^3/3, triangular solve k^2 (n-k)."""
    r = ell if sketch else m
    f = 4.0 * r * n * k - 2.0 * k * k * (r + n) + 4.0 * k ** 3 / 3.0 + k * k * (n - k)
    if sketch:
        f += 2.0 * ell * m * n
    return f


def sketch_bytes(m, n, ell, a_bytes=8):
    """Algorithmic bytes of the sketch kernel: read A and Omega once, write Y."""
    return a_bytes * m * n + 2 * ell * m + 4 * ell * n


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


def source_hash(files=("sketch.cu", "common.cuh")):
    h = hashlib.sha256()
    for name in files:
        with open(os.path.join(ROOT, "paper_2012_00706_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(profile="sketch_lowp_20000x2000.md", files=("sketch.cu", "common.cuh")):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary, if the summary
    was taken on the current kernel source (its `source_sha` line)."""
    path = os.path.join(ROOT, "profiles", profile)
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            key, _, v = line.strip()[2:].partition(":")
            vals[key.strip()] = v.strip().strip("`")
    if vals.get("source_sha") != source_hash(files):
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def alu_peaks(gid):
    """FP32 (FFMA) and FP64 (DFMA) rates of this GPU in TFLOP/s, measured now by the
    library's probe (independent FMA chains on every SM)."""
    return {"fp32_tflops": gid.probe_fma_peak("fp32"), "fp64_tflops": gid.probe_fma_peak("fp64"),
            "source": "measured in this run: id_probe_fma_peak (8 independent FMA chains per thread, "
                      "2 x 1024-thread CTAs per SM, CUDA-event time of one ~30 ms launch)"}


def cpqr_flops(r, n, k):
    return 4.0 * r * n * k - 2.0 * k * k * (r + n) + 4.0 * k ** 3 / 3.0


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ oracle arm

def oracle_id_timed(cfg, rows=None):
    """Time the FP64 oracle ID on the workload (optionally on a row sample of the
    sketch; the sketch time is then scaled to all rows).  Returns (seconds per full
    ID, result of the last run)."""
    import oracle
    a, om = cfg["A"], cfg["omega"]
    m = a.shape[0]
    rows = m if rows is None else min(rows, m)
    t0 = time.perf_counter()
    y = oracle.sketch_f64(om[:, :rows], a[:rows])
    t_sketch = (time.perf_counter() - t0) * (m / rows)
    t1 = time.perf_counter()
    r = oracle.cpqr(y, k=K, norm_mode="downdate")
    T = oracle.solve_T(r["R"], r["J"], r["k"])
    t_rest = time.perf_counter() - t1
    return t_sketch + t_rest, {"J": r["J"], "T": T, "k": r["k"]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import workloads as wl
    import oracle
    oracle.build()
    cfg = wl.config2()
    # size each step so that warmup + steps take about two minutes of host time
    probe_rows = 2000
    t_probe, _ = oracle_id_timed(cfg, rows=probe_rows)
    budget = 120.0 / max(1, args.steps + args.warmup)
    rows = int(min(M, max(500, M * budget / max(t_probe, 1e-3))))
    for _ in range(args.warmup):
        oracle_id_timed(cfg, rows=rows)
    ts = [oracle_id_timed(cfg, rows=rows)[0] for _ in range(args.steps)]
    sec = statistics.mean(ts)
    value = 1.0 / sec
    sample = (f"each step: FP64 oracle ID (plain C, 1 thread) with the sketch over {rows} of {M} rows "
              f"(time scaled to all rows) plus the full pivoted QR and T solve")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "IDs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M, "n": N, "k": K, "ell": ELL},
        "cpu_baseline": {"value": value, "unit": "IDs/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "IDs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "tflops": id_flops(M, N, ELL, K) / sec / 1e12,
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------- our arm

def batched_leg(gid, wl, dev, stream, count=512, loops=True, lean_steps=0, world=1, rank=0):
    """512 uneven FP64 IDs (exact rank r, sigma_i = 10^(-i/r), m in [256, 4096],
    n in [64, 1024], k = r): the batched mixed path (default and autotuned unit
    shapes, plain launches and a replayed CUDA graph) against the batched FP64
    twin (same call, precision plain_f64) and one id_factor call per matrix,
    mixed and plain FP64, with the errors of a sample of matrices."""
    import tempfile
    import torch
    t_gen = time.perf_counter()
    share = None
    if world > 1:
        # this process's longest-processing-time share (every rank computes the same split)
        all_shapes = wl.config4_shapes(count, 4)
        rank_of, _ = gid.shard_batch([(m, n) for m, n, _ in all_shapes], [r for _, _, r in all_shapes], world)
        share = [i for i, r in enumerate(rank_of) if r == rank]
    shapes, bufs = wl.config4_device(dev, count=count, indices=share)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    views = [v for _, v in bufs]
    ranks = [r for _, _, r in shapes]
    ldas = [b.shape[1] for b, _ in bufs]
    count = len(shapes)
    a_bytes = sum(8 * m * n for m, n, _ in shapes)
    flops = sum(id_flops(m, n, min(r + 10, m), r) for m, n, r in shapes)
    m_pad = (max(m for m, _, _ in shapes) + 7) // 8 * 8
    ell_max = max(min(r + 10, m) for m, _, r in shapes)
    om64, bits = wl.gaussian_omega(ell_max, m_pad, 4004, "bf16")
    omega = torch.from_numpy(bits.view(np.int16)).to(dev).view(torch.bfloat16)
    omega64 = torch.from_numpy(om64).to(dev)
    out = {"workload": f"{count} FP64 matrices, m in [256,4096], n in [64,1024] (n <= m), exact rank r in "
                       f"[8,128], sigma_i = 10^(-i/r), k = r, ell = r + 10; seed 4; drawn on the GPU",
           "a_bytes": a_bytes, "flops_per_batch": flops, "generate_s": t_gen}

    def time_calls(fn, reps, warm=2):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / reps

    if lean_steps:
        # profiling case: default unit shapes, plain launches only
        plan = gid.BatchPlan([(m, n) for m, n, _ in shapes], ranks, precision="mixed_bf16x3", lda=ldas)
        plan.bind(views)
        ms = time_calls(lambda: plan.run(omega), lean_steps)
        out["mixed_bf16x3"] = {"ms_default_shapes": ms, "ids_per_s": count / (ms / 1e3),
                               "shapes": plan.describe()}
        return out
    for prec in ("mixed_bf16x3", "mixed_bf16"):
        plan = gid.BatchPlan([(m, n) for m, n, _ in shapes], ranks, precision=prec, lda=ldas)
        plan.bind(views)
        ms_default = time_calls(lambda: plan.run(omega), 5)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        gid.set_stage_events(evs)
        plan.run(omega)
        gid.set_stage_events(None)
        torch.cuda.synchronize()
        stages = {"sketch": evs[0].elapsed_time(evs[1]), "cpqr": evs[2].elapsed_time(evs[3]),
                  "solve_T": evs[3].elapsed_time(evs[5]), "solve_inverses": evs[3].elapsed_time(evs[4]),
                  "solve_products": evs[4].elapsed_time(evs[5])}
        info = plan.info.cpu()
        with tempfile.TemporaryDirectory() as td:
            best = plan.autotune(omega, reps=3, cache_path=os.path.join(td, "tune.jsonl"))
        ms_tuned = time_calls(lambda: plan.run(omega), 5)
        # one CUDA graph holding the whole launch sequence
        gs = torch.cuda.Stream()
        gs.wait_stream(torch.cuda.current_stream())
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(gs):
            plan.run(omega, stream=gs)
            gs.synchronize()
            with torch.cuda.graph(graph, stream=gs):
                plan.run(omega, stream=gs)
        torch.cuda.synchronize()
        ms_graph = time_calls(graph.replay, 10)
        best_ms = min(ms_tuned, ms_graph)
        out[prec] = {"ms_default_shapes": ms_default, "ms_tuned": ms_tuned, "ms_graph_tuned": ms_graph,
                     "tuner_ms": best, "ids_per_s": count / (best_ms / 1e3),
                     "tflops": flops / (best_ms / 1e3) / 1e12,
                     "hbm_gbs_whole_batch": a_bytes / (best_ms / 1e3) / 1e9,
                     "stages_ms_default": stages, "tuned_shapes": plan.describe(),
                     "info_nonzero": int((info != 0).sum())}
        if prec == "mixed_bf16x3":
            keep = plan
        else:
            del plan

    # ---- the FP64 twin through the same batched call: each matrix's sketched FP64 ID
    plan = gid.BatchPlan([(m, n) for m, n, _ in shapes], ranks, precision="plain_f64", lda=ldas)
    plan.bind(views)
    ms_plain = time_calls(lambda: plan.run(omega64), 3, warm=1)
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(gs):
        plan.run(omega64, stream=gs)
        gs.synchronize()
        with torch.cuda.graph(graph, stream=gs):
            plan.run(omega64, stream=gs)
    torch.cuda.synchronize()
    ms_plain_graph = time_calls(graph.replay, 3, warm=1)
    best_plain = min(ms_plain, ms_plain_graph)
    best_x3 = min(out["mixed_bf16x3"]["ms_tuned"], out["mixed_bf16x3"]["ms_graph_tuned"])
    out["plain_f64"] = {"ms": ms_plain, "ms_graph": ms_plain_graph, "ids_per_s": count / (best_plain / 1e3),
                        "tflops": flops / (best_plain / 1e3) / 1e12,
                        "info_nonzero": int((plan.info != 0).sum().item())}
    out["batched_bf16x3_vs_batched_plain_f64"] = best_plain / best_x3
    del graph, plan
    if not loops:
        return out

    # ---- one id_factor call per matrix (launch-per-matrix baseline), mixed and plain FP64
    def per_matrix(precision, om):
        ws_bytes = max(gid.id_workspace_size(m, n, torch.float64, k=r, precision=precision, sketch=True,
                                             ell=min(r + 10, m), omega=om[: min(r + 10, m), :m])
                       for m, n, r in shapes)
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        outs = []
        for (m, n, r) in shapes:
            outs.append((torch.empty(n, dtype=torch.int32, device=dev),
                         torch.empty((max(n - 1, 1), r), dtype=torch.float64, device=dev).t(),
                         torch.zeros(2, dtype=torch.int32, device=dev),
                         torch.zeros(1, dtype=torch.float64, device=dev)))

        def loop():
            for (m, n, r), v, o in zip(shapes, views, outs):
                gid.id_factor(v, r, precision=precision, omega=om[: min(r + 10, m), :m], workspace=ws, out=o,
                              sync=False)
        ms = time_calls(loop, 1, warm=1)
        return ms, outs

    ms_loop_mixed, _ = per_matrix("mixed_bf16x3", omega)
    ms_loop_plain, outs_plain = per_matrix("plain_f64", omega64)
    out["per_matrix_loop"] = {"mixed_bf16x3_ms": ms_loop_mixed, "plain_f64_ms": ms_loop_plain,
                              "plain_f64_ids_per_s": count / (ms_loop_plain / 1e3),
                              "plain_f64_tflops": flops / (ms_loop_plain / 1e3) / 1e12}
    out["speedup"] = {"batched_bf16x3_vs_plain_f64_loop": ms_loop_plain / best_x3,
                      "batched_bf16x3_vs_mixed_loop": ms_loop_mixed / best_x3,
                      "tuned_vs_default_bf16x3": out["mixed_bf16x3"]["ms_default_shapes"] /
                      out["mixed_bf16x3"]["ms_tuned"]}

    # ---- errors on a sample of the matrices (FP64 on the GPU, 2-norms by power iteration)
    keep.run(omega)
    res = keep.results()

    def norm2(X, iters=50):
        g = torch.Generator(device=dev)
        g.manual_seed(0)
        v = torch.randn(X.shape[1], dtype=torch.float64, device=dev, generator=g)
        v /= v.norm()
        s = 0.0
        for _ in range(iters):
            w = X.T @ (X @ v)
            nw = w.norm()
            if nw == 0:
                return 0.0
            s = float(nw.sqrt())
            v = w / nw
        return s

    def ahat(A, J, T, k):
        n = A.shape[1]
        Jl = J.long()
        P_ = torch.zeros((k, n), dtype=torch.float64, device=dev)
        P_[:, Jl[:k]] = torch.eye(k, dtype=torch.float64, device=dev)
        if k < n:
            P_[:, Jl[k:]] = T[:k, : n - k]
        return A[:, Jl[:k]] @ P_

    sample = list(range(0, count, count // 8))[:8]
    e_m, e_p, d_mp = [], [], []
    for i in sample:
        m, n, r = shapes[i]
        A = views[i]
        na = norm2(A)
        Jp, Tp, sp, _ = outs_plain[i]
        kp = int(sp[0].item())
        hm = ahat(A, res[i].J, res[i].T, res[i].k)
        hp = ahat(A, Jp, Tp, kp)
        e_m.append(norm2(A - hm) / na)
        e_p.append(norm2(A - hp) / na)
        d_mp.append(norm2(hm - hp) / na)
    out["accuracy_sample"] = {"matrices": sample, "e_batched_bf16x3_max": max(e_m), "e_plain_f64_max": max(e_p),
                              "d_batched_bf16x3_vs_plain_max": max(d_mp),
                              "matched_1e-6": max(d_mp) <= 1e-6}
    del keep, bufs, views
    torch.cuda.empty_cache()
    return out


def _time_id(gid, dev, A, k, reps, **kw):
    """Median time of one id_factor call (ms) over `reps` CUDA-graph replays, the stage split
    of one plain launch (stage events), and the result of the last call."""
    import torch
    om = kw.get("omega")
    ws = torch.empty(gid.id_workspace_size(A.shape[0], A.shape[1], A.dtype, k=k, sketch=om is not None,
                                           ell=om.shape[0] if om is not None else 0, **kw),
                     dtype=torch.uint8, device=dev)
    kcap = kw.get("k_max") or k
    n = A.shape[1]
    out = (torch.empty(n, dtype=torch.int32, device=dev),
           torch.empty((max(n - 1, 1), kcap), dtype=torch.float64, device=dev).t(),
           torch.zeros(2, dtype=torch.int32, device=dev), torch.zeros(1, dtype=torch.float64, device=dev))
    kk = None if kw.get("tol") else k

    def one(stream=None):
        gid.id_factor(A, kk, workspace=ws, out=out, sync=False, stream=stream, **kw)

    for _ in range(3):
        one()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(gs):
        with torch.cuda.graph(g, stream=gs):
            one(gs)
    torch.cuda.synchronize()
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    ts = []
    cur = torch.cuda.current_stream()
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        g.replay()
        e1.record(cur)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    gid.set_stage_events(evs)
    one()
    gid.set_stage_events(None)
    torch.cuda.synchronize()
    names = ["sketch_kernel", "sketch_reduce", "cpqr", "solve_T", "tail"]
    stages = {nm: evs[j].elapsed_time(evs[j + 1]) for j, nm in enumerate(names)}
    return statistics.median(ts), stages, out


def config1_leg(gid, wl, dev, peaks, reps=20):
    """Plain FP64 ID of a 1000 x 500 matrix (sigma_i = 10^(-i/25), k = 50, no sketch), and
    the FP32 pivoted QR of the same matrix (the mixed-single ID of Algorithm 2), one ID at
    a time (CUDA-graph replay)."""
    import torch
    c = wl.config1()
    m, n, k = c["m"], c["n"], c["k"]
    A = torch.from_numpy(c["A"]).to(dev)
    flops = id_flops(m, n, 0, k, sketch=False)
    out = {"workload": "A 1000x500 FP64, sigma_i = 10^(-i/25), k = 50, no sketch; seed 1", "flops_per_id": flops}
    for prec, peak in (("plain_f64", peaks["fp64_tflops"]), ("plain_f32", peaks["fp32_tflops"])):
        ms, stages, res = _time_id(gid, dev, A, k, reps, precision=prec)
        kout = int(res[2][0].item())
        cq_flops = cpqr_flops(m, n, k)
        ach = cq_flops / (stages["cpqr"] / 1e3) / 1e12
        err = gid.id_factor(A, k, precision=prec, estimate_error=True).err
        out[prec] = {"ms_per_id": ms, "ids_per_s": 1e3 / ms, "tflops": flops / (ms / 1e3) / 1e12,
                     "stages_ms": stages, "k": kout, "err_fro": err,
                     "cpqr_roofline": {"kernel": "k_cpqr_resident", "bound": "alu", "achieved": ach, "peak": peak,
                                       "unit": "TFLOP/s", "frac": ach / peak,
                                       "algorithmic_flops": cq_flops}}
    return out


def low_id_leg(gid, wl, dev, peaks, reps=20):
    """Algorithm 2 as the paper states it, on its own test matrices (Slow, Fast: 1000 x 1000,
    sigma_i = i^-1, i^-4, k = 20): the whole matrix cast to half / bfloat16 (scaled per
    64-row block and column), FP32 pivoted QR of A_L, FP64 T; against the plain FP64 ID of
    the same matrix.  Errors of both approximations (A_hat_M from A, A_hat_L from A_L)
    against A, relative 2-norms by 60 FP64 power iterations on the GPU."""
    import torch

    def norm2(X, iters=60):
        g = torch.Generator(device=dev)
        g.manual_seed(0)
        v = torch.randn(X.shape[1], dtype=torch.float64, device=dev, generator=g)
        v /= v.norm()
        s_ = 0.0
        for _ in range(iters):
            w = X.T @ (X @ v)
            s_ = float(w.norm().sqrt())
            v = w / w.norm()
        return s_

    out = {"workload": "paper Slow / Fast matrices 1000x1000 (sigma_i = i^-1, i^-4; seed 21), k = 20, no sketch"}
    k = 20
    for kind in ("slow", "fast"):
        A = torch.from_numpy(wl.paper_dataset(kind, seed=21)).to(dev)
        na = norm2(A)
        row = {}
        for prec in ("plain_f64", "low_bf16", "low_f16"):
            ms, stages, res = _time_id(gid, dev, A, k, reps, precision=prec)
            J, T = res[0], res[1][:k, : A.shape[1] - k]
            hm = gid.reconstruct(A, J, T, k)
            item = {"ms_per_id": ms, "ids_per_s": 1e3 / ms, "stages_ms": stages, "e_M": norm2(A - hm) / na}
            if prec != "plain_f64":
                AL = gid.low_cast(A, prec)
                hl = gid.reconstruct(AL, J, T, k).double()
                item["e_L"] = norm2(A - hl) / na
                item["speedup_vs_plain_f64"] = row["plain_f64"]["ms_per_id"] / ms
            row[prec] = item
        out[kind] = row
    return out


def row_id_leg(gid, dev, A, reps=10):
    """Row ID of the 20000 x 2000 benchmark matrix (100 of its 20000 rows): A transposed
    into the workspace, then the three-piece bfloat16 sketched ID of A^T with a Gaussian
    Omega of 110 x 2000, FP32 pivoted QR of the 110 x 20000 sketch, FP64 T."""
    import torch
    import workloads as wl
    m, n = A.shape
    _, bits = wl.gaussian_omega(ELL, n, 2002, "bf16")
    om = torch.from_numpy(bits.view(np.int16)).to(dev).view(torch.bfloat16)
    gid.id_factor_rows(A, K, precision="mixed_bf16x3", omega=om)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = gid.id_factor_rows(A, K, precision="mixed_bf16x3", omega=om, estimate_error=False)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    err = gid.id_factor_rows(A, K, precision="mixed_bf16x3", omega=om, estimate_error=True).err
    ms = statistics.median(ts)
    return {"workload": "row ID of A 20000x2000 FP64 (the benchmark matrix), k = 100, BF16x3 sketch 110 x 2000",
            "ms_per_id": ms, "ids_per_s": 1e3 / ms, "k": res.k, "err_fro": err,
            "note": "includes the transpose of A into the workspace and the host read of k and info"}


def config3_leg(gid, wl, dev, peaks, reps=3):
    """The 65536 x 1000 FP32 snapshot matrix (travelling sinusoids plus 1e-6 noise) at
    tolerance 1e-6: the plain FP64 ID of A itself against sketched mixed IDs (half sketch,
    three-piece bfloat16 sketch) with ell = k_max + 10."""
    import torch
    c = wl.config3()
    m, n, tol = c["m"], c["n"], c["tol"]
    A = torch.from_numpy(c["A"]).to(dev)
    kmax = 150
    ell = kmax + 10
    out = {"workload": "snapshot matrix 65536x1000 FP32 (40 travelling sinusoids, amplitudes 0.8^j, "
                       "1e-6 noise; seed 3), relative Frobenius tolerance 1e-6, k_max 150",
           "a_bytes": 4 * m * n}
    ms, stages, res = _time_id(gid, dev, A, None, reps, tol=tol, k_max=200, precision="plain_f64")
    k = int(res[2][0].item())
    err = gid.id_factor(A, tol=tol, k_max=200, precision="plain_f64", estimate_error=True).err
    cq = cpqr_flops(m, n, k)
    ach = cq / (stages["cpqr"] / 1e3) / 1e12
    out["plain_f64"] = {"ms_per_id": ms, "ids_per_s": 1e3 / ms, "k": k, "err_fro": err,
                        "tflops": id_flops(m, n, 0, k, sketch=False) / (ms / 1e3) / 1e12, "stages_ms": stages,
                        "cpqr_roofline": {"kernel": "k_cpqr_grid", "bound": "alu", "achieved": ach,
                                          "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                                          "frac": ach / peaks["fp64_tflops"], "algorithmic_flops": cq,
                                          "hbm_bytes_per_step_min": 16 * m * n}}
    for prec, fmt in (("mixed_f16", "f16"), ("mixed_bf16x3", "bf16")):
        _, bits = wl.gaussian_omega(ell, m, 3003, fmt)
        om = torch.from_numpy(bits.view(np.int16)).to(dev).view(torch.bfloat16 if fmt == "bf16" else torch.float16)
        ms, stages, res = _time_id(gid, dev, A, None, max(reps, 10), tol=tol, k_max=kmax, precision=prec, omega=om)
        k = int(res[2][0].item())
        err = gid.id_factor(A, tol=tol, k_max=kmax, precision=prec, omega=om, estimate_error=True).err
        sk_bytes = sketch_bytes(m, n, ell, a_bytes=4)
        out[prec] = {"ms_per_id": ms, "ids_per_s": 1e3 / ms, "k": k, "err_fro": err, "ell": ell,
                     "tflops": id_flops(m, n, ell, k) / (ms / 1e3) / 1e12, "stages_ms": stages,
                     "sketch_hbm_frac": sk_bytes / (stages["sketch_kernel"] / 1e3) / 1e9 / measured_peaks()[0],
                     "speedup_vs_plain_f64": out["plain_f64"]["ms_per_id"] / ms}
    # rank-adaptive: sketch rows (and the rank) grow by blocks of 32, up to 256 rows, until
    # the FP64 residual on A itself meets the tolerance (one host synchronisation per block,
    # inside the time)
    ell_a, kmax_a, blk = 256, 240, 32
    _, bits = wl.gaussian_omega(ell_a, m, 3004, "bf16")
    om = torch.from_numpy(bits.view(np.int16)).to(dev).view(torch.bfloat16)
    res, used = gid.id_factor_adaptive(A, tol, kmax_a, om, block=blk)      # warm-up
    ts = []
    for _ in range(max(reps, 5)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res, used = gid.id_factor_adaptive(A, tol, kmax_a, om, block=blk)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    out["mixed_bf16x3_adaptive"] = {"ms_per_id": ms, "ids_per_s": 1e3 / ms, "k": res.k, "err_fro": res.err,
                                    "ell_used": used, "ell_max": ell_a, "block": blk, "meets_tol": res.err <= tol,
                                    "speedup_vs_plain_f64": out["plain_f64"]["ms_per_id"] / ms}
    return out


def config5_leg(gid, wl, dev, peaks, reps=5):
    """Differentiable IDs: 64 FP32 matrices 2048 x 512 of rank 32 (sigma_i = 10^(-i/16)),
    k = 32, loss ||A_hat - B||_F^2 with Gaussian B; forward (pivoted QR, T, reconstruction)
    and backward (the fixed-pivot adjoint) timed separately with CUDA events."""
    import torch
    c = wl.config5()
    k, m, n = c["k"], c["m"], c["n"]
    batch = c["A"].shape[0]
    A = torch.from_numpy(np.ascontiguousarray(c["A"].transpose(0, 2, 1))).to(dev).transpose(1, 2)
    B = torch.from_numpy(c["B"]).to(dev)
    A.requires_grad_(True)

    def fwd():
        Ahat, T, J = gid.IDFunction.apply(A, k)
        return ((Ahat - B) ** 2).sum()

    for _ in range(2):
        loss = fwd()
        loss.backward()
        A.grad = None
    torch.cuda.synchronize()
    tf, tb = [], []
    cur = torch.cuda.current_stream()
    for _ in range(reps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(cur)
        loss = fwd()
        e1.record(cur)
        loss.backward()
        e2.record(cur)
        torch.cuda.synchronize()
        tf.append(e0.elapsed_time(e1))
        tb.append(e1.elapsed_time(e2))
        A.grad = None
    f_fwd = batch * (id_flops(m, n, 0, k, sketch=False) + 2.0 * m * k * (n - k))
    f_bwd = batch * 8.0 * m * n * k
    fms, bms = statistics.median(tf), statistics.median(tb)
    return {"workload": "64 x (2048x512 FP32), exact rank 32, sigma_i = 10^(-i/16), k = 32, loss ||A_hat - B||_F^2; "
                        "seed 5",
            "forward_ms": fms, "backward_ms": bms, "ids_per_s_forward": batch / (fms / 1e3),
            "forward_tflops": f_fwd / (fms / 1e3) / 1e12, "backward_tflops": f_bwd / (bms / 1e3) / 1e12,
            "backward_flops_model": "8 m n k per matrix (thin QR of the skeleton, the projections of the "
                                    "cotangent and their products)",
            "backward_frac_of_fp32": f_bwd / (bms / 1e3) / 1e12 / peaks["fp32_tflops"],
            "forward_path": gid.BatchPlan([(m, n)] * batch, [k] * batch, dtype=torch.float32, precision="plain_f32",
                                          device=dev).describe(),
            "note": "forward: one PLAIN_F32 batch plan per call (grouped pivoted QRs in waves, one batched "
                    "solve), the reconstruction, and the host read of the 64 ranks (one synchronisation)"}


def profile_case(gid, wl, dev, which):
    """`bwd`: one forward and one backward of the differentiable ID on config 5's 64 FP32
    2048 x 512 matrices (k = 32, loss ||A_hat - B||_F^2).

    `cpqr`: one launch of each pivoted-QR kernel, in this order: the cluster kernel (config 2's
    BF16x3 ID: its sketch 110 x 2000), the resident grid kernel (config 1 plain FP64,
    1000 x 500, k = 50), the streaming grid kernel (plain FP64 16384 x 1000, k = 50,
    sigma_i = i^-2: a 131 MB working copy) and the grouped kernel (one wave of 16 FP32
    2048 x 512 matrices of config 5, k = 32)."""
    import torch
    if which == "bwd":
        c = wl.config5()
        A = torch.from_numpy(np.ascontiguousarray(c["A"].transpose(0, 2, 1))).to(dev).transpose(1, 2)
        B = torch.from_numpy(c["B"]).to(dev)
        A.requires_grad_(True)
        Ahat, T, J = gid.IDFunction.apply(A, c["k"])
        ((Ahat - B) ** 2).sum().backward()
        torch.cuda.synchronize()
        ok = bool(torch.isfinite(A.grad).all())
        print(json.dumps({"profile_case": which, "grad_finite": ok}), flush=True)
        return 0 if ok else 1
    cfg = wl.config2()
    A = torch.from_numpy(cfg["A"]).to(dev)
    om = torch.from_numpy(cfg["omega_bits"].view(np.int16)).to(dev).view(torch.bfloat16)
    gid.id_factor(A, cfg["k"], precision="mixed_bf16x3", omega=om)
    del A
    torch.cuda.empty_cache()
    c1 = wl.config1()
    gid.id_factor(torch.from_numpy(c1["A"]).to(dev), c1["k"], precision="plain_f64")
    a3 = wl.lowrank(16384, 1000, np.arange(1, 1001, dtype=np.float64) ** -2.0, 6)
    gid.id_factor(torch.from_numpy(a3).to(dev), 50, precision="plain_f64")
    c5 = wl.config5()
    mats = [torch.from_numpy(np.asfortranarray(c5["A"][i])).to(dev) for i in range(16)]
    plan = gid.BatchPlan([tuple(a.shape) for a in mats], [c5["k"]] * 16, dtype=torch.float32,
                         precision="plain_f32")
    plan.bind(mats)
    plan.run()
    torch.cuda.synchronize()
    bad = [i for i, r in enumerate(plan.results()) if r.info != 0 or r.k != c5["k"]]
    print(json.dumps({"profile_case": which, "grouped_plan": plan.describe(), "bad": bad}), flush=True)
    return 1 if bad else 0


def figures(gid, wl, dev, ks=tuple(range(1, 52, 5)), ns=(50, 100, 200, 300, 500, 700, 1000)):
    """The sweeps of the paper's Figs. 1-6 (Sec. 3): the paper's Slow / Medium / Fast
    matrices (1000 x 1000, sigma_i = i^-1, i^-2, i^-4), target rank k over `ks` with all
    1000 columns, and column count n over `ns` (first n columns) with k = 20.  For each low
    format (FP32: the plain FP32 ID of A; bfloat16 and half: Algorithm 2, low_bf16 /
    low_f16) both approximations, A_hat_M = A(:,J) P and A_hat_L = A_L(:,J) P, against
    the double ID A_hat_D of the same matrix (d_X = ||A_hat_X - A_hat_D||_2 / ||A||_2,
    Figs. 1-4) and against A itself (e_X = ||A - A_hat_X||_2 / ||A||_2, Figs. 5-6).  The
    half column `f16_unscaled` casts A to half without the power-of-two scaling (torch's
    float16 cast) and pivots it in FP32: the configuration of the paper's half precision
    runs, whose breakdown on Fast beyond k = 21 it reports.  2-norms: 80 FP64 power
    iterations on the GPU."""
    import torch

    def norm2(X, iters=80):
        g = torch.Generator(device=dev)
        g.manual_seed(0)
        v = torch.randn(X.shape[1], dtype=torch.float64, device=dev, generator=g)
        v /= v.norm()
        s_ = 0.0
        for _ in range(iters):
            w = X.T @ (X @ v)
            nw = float(w.norm())
            if nw == 0.0:
                return 0.0
            s_ = nw ** 0.5
            v = w / nw
        return s_

    def one(A, k):
        na = norm2(A)
        d = gid.id_factor(A, k, precision="plain_f64")
        hd = gid.reconstruct(A, d.J, d.T, d.k)
        row = {"e_D": norm2(A - hd) / na, "k_D": d.k}
        forms = [("f32", A, "plain_f32", A.float()), ("bf16", A, "low_bf16", None), ("f16", A, "low_f16", None)]
        a16 = A.to(torch.float16).float()                      # unscaled half cast of A
        forms.append(("f16_unscaled", a16, "plain_f32", a16))
        for name, src, prec, al in forms:
            res = gid.id_factor(src, k, precision=prec)
            if res.info != 0 or res.k < 1:
                row[name] = {"info": res.info, "k": res.k}
                continue
            al = al if al is not None else gid.low_cast(A, prec)
            hm = gid.reconstruct(A, res.J, res.T, res.k)
            hl = gid.reconstruct(al, res.J, res.T, res.k).double()
            row[name] = {"k": res.k, "info": res.info, "d_M": norm2(hm - hd) / na, "d_L": norm2(hl - hd) / na,
                         "e_M": norm2(A - hm) / na, "e_L": norm2(A - hl) / na}
        return row

    out = {"workload": "paper Slow / Medium / Fast matrices, 1000 x 1000 (seed 21)", "k_sweep": {}, "n_sweep": {}}
    for kind in ("slow", "medium", "fast"):
        A = torch.from_numpy(wl.paper_dataset(kind, seed=21)).to(dev)
        out["k_sweep"][kind] = {str(k): one(A, k) for k in ks}
        out["n_sweep"][kind] = {str(n): one(A[:, :n].contiguous().t().contiguous().t(), 20) for n in ns}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", default="mixed_bf16x3",
                    help="form of the headline stream (mixed_bf16x3 meets d <= 1e-6 against plain FP64)")
    ap.add_argument("--no-extras", action="store_true", help="skip plain/matched/e2e/cpu legs")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-matrix batched leg")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 1000x500 plain, 65536x1000 snapshot and differentiable-batch legs")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched leg (a profiling case) and print its JSON")
    ap.add_argument("--batch-count", type=int, default=512, help="matrices in the batched leg")
    ap.add_argument("--inflight", type=int, default=INFLIGHT, help="IDs in flight in the timed stream")
    ap.add_argument("--inflight-groups", type=int, default=INFLIGHT_GROUPS,
                    help="CUDA graphs the in-flight IDs are issued as, replayed in turn")
    ap.add_argument("--figures", action="store_true",
                    help="print the k and n sweeps of the paper's Figs. 1-6 as one JSON object and exit")
    ap.add_argument("--profile-case", choices=["cpqr", "bwd"],
                    help="profiling cases: cpqr runs one launch of each pivoted-QR kernel; bwd one forward and "
                         "backward of the 64 x 2048 x 512 differentiable ID")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import paper_2012_00706_gb300 as gid
    import workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    gid.load()
    if args.profile_case:
        return profile_case(gid, wl, dev, args.profile_case)
    if args.figures:
        if rank == 0:
            print(json.dumps(figures(gid, wl, dev)), flush=True)
        return 0
    peaks = alu_peaks(gid)
    if args.batched_only:
        line = {"batched": batched_leg(gid, wl, dev, torch.cuda.current_stream(), count=args.batch_count,
                                       loops=False, lean_steps=args.steps)}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return 0
    cfg = wl.config2()
    a_np, bits = cfg["A"], cfg["omega_bits"]
    A = torch.from_numpy(a_np).to(dev)                       # (m, n), column-major strides
    assert A.stride(0) == 1
    omega = torch.from_numpy(bits.view(np.int16)).to(dev).view(torch.bfloat16)
    omega64 = torch.from_numpy(cfg["omega"]).to(dev)
    stream = torch.cuda.current_stream()

    def make_out(kcap):
        J = torch.empty(N, dtype=torch.int32, device=dev)
        T = torch.empty((N - 1, kcap), dtype=torch.float64, device=dev).t()
        small = torch.zeros(2, dtype=torch.int32, device=dev)
        err = torch.zeros(1, dtype=torch.float64, device=dev)
        return J, T, small, err

    def run_loop(precision, om, steps, warmup, stage=False, a_src=None, host=None, graph=False):
        ws = torch.empty(gid.id_workspace_size(M, N, torch.float64, k=K, precision=precision, sketch=True,
                                               ell=ELL, omega=om), dtype=torch.uint8, device=dev)
        out = make_out(K)
        A_use = A if a_src is None else a_src

        def one():
            if host is not None:
                A_use.copy_(host["A"], non_blocking=True)
                om.copy_(host["omega"], non_blocking=True)
            gid.id_factor(A_use, K, precision=precision, omega=om, workspace=ws, out=out, sync=False)
            if host is not None:
                host["J"].copy_(out[0], non_blocking=True)
                host["T"].copy_(out[1][:, : N - K], non_blocking=True)
                host["small"].copy_(out[2], non_blocking=True)

        for _ in range(warmup):
            one()
        torch.cuda.synchronize()
        g = None
        if graph:
            # the whole ID captured once into a CUDA graph and replayed each step
            g = torch.cuda.CUDAGraph()
            gs = torch.cuda.Stream()
            gs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(gs):
                with torch.cuda.graph(g, stream=gs):
                    one()
            torch.cuda.synchronize()
            for _ in range(warmup):
                g.replay()
            torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(steps)] if stage else None
        barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for i in range(steps):
            if stage:
                gid.set_stage_events(evs[i])
            if g is not None:
                g.replay()
            else:
                one()
        t1.record(stream)
        gid.set_stage_events(None)
        torch.cuda.synchronize()
        barrier()
        total_ms = t0.elapsed_time(t1)
        stages = None
        if stage:
            names = ["sketch_kernel", "sketch_reduce", "cpqr", "solve_T", "tail"]
            stages = {nm: statistics.mean(e[j].elapsed_time(e[j + 1]) for e in evs) for j, nm in enumerate(names)}
        return total_ms, out, stages

    def run_e2e(precision, host, steps, warmup):
        """End to end through the public API, as a streaming caller runs it: every step copies
        its A and Omega from pinned host memory into one of two device buffers on a copy
        stream, runs id_factor on the compute stream once its copy has landed, and copies J,
        T and (k, info) back to pinned host memory.  The copy of step i + 1 overlaps the
        compute of step i (the host-to-device link, about 0.2 TB/s, is the bound)."""
        ws = torch.empty(gid.id_workspace_size(M, N, torch.float64, k=K, precision=precision, sketch=True,
                                               ell=ELL, omega=omega), dtype=torch.uint8, device=dev)
        out = make_out(K)
        a_buf = [torch.empty_like(A) for _ in range(2)]
        o_buf = [torch.empty_like(omega) for _ in range(2)]
        copy_s = torch.cuda.Stream()
        comp_s = torch.cuda.Stream()
        landed = [torch.cuda.Event() for _ in range(2)]
        used = [torch.cuda.Event() for _ in range(2)]
        for e in used:
            e.record(comp_s)

        def step(i):
            b = i % 2
            copy_s.wait_event(used[b])
            with torch.cuda.stream(copy_s):
                a_buf[b].copy_(host["A"], non_blocking=True)
                o_buf[b].copy_(host["omega"], non_blocking=True)
                landed[b].record(copy_s)
            comp_s.wait_event(landed[b])
            gid.id_factor(a_buf[b], K, precision=precision, omega=o_buf[b], workspace=ws, out=out, sync=False,
                          stream=comp_s)
            with torch.cuda.stream(comp_s):
                host["J"].copy_(out[0], non_blocking=True)
                host["T"].copy_(out[1][:, : N - K], non_blocking=True)
                host["small"].copy_(out[2], non_blocking=True)
                used[b].record(comp_s)

        for i in range(warmup):
            step(i)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        cur = torch.cuda.current_stream()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(cur)
        copy_s.wait_stream(cur)
        comp_s.wait_stream(cur)
        for i in range(steps):
            step(i)
        cur.wait_stream(comp_s)
        t1.record(cur)
        torch.cuda.synchronize()
        barrier()
        return t0.elapsed_time(t1)

    def run_inflight(precision, om, steps, warmup, depth):
        """`steps` IDs with `depth` of them in flight, issued as `--inflight-groups` CUDA graphs
        of depth / groups IDs each, replayed in turn on their own streams: a graph holds
        its IDs on forked streams (each with its own copy of A, workspace and outputs, so
        nothing is shared through L2), and while one group's pivoted QRs run on 16-SM
        clusters the next group's sketches fill the other SMs.  A graph of the remaining
        steps % depth IDs covers the rest.  Throughput of a stream of IDs, as a server would
        run them."""
        copies = [A] + [A.clone() for _ in range(depth - 1)]
        wss = [torch.empty(gid.id_workspace_size(M, N, torch.float64, k=K, precision=precision, sketch=True,
                                                 ell=ELL, omega=om), dtype=torch.uint8, device=dev)
               for _ in range(depth)]
        outs = [make_out(K) for _ in range(depth)]
        streams = [torch.cuda.Stream() for _ in range(depth)]

        def capture(ids):
            g = torch.cuda.CUDAGraph()
            cs = torch.cuda.Stream()
            cs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(cs):
                for i in ids:   # warm each branch once outside the capture
                    gid.id_factor(copies[i], K, precision=precision, omega=om, workspace=wss[i], out=outs[i],
                                  sync=False, stream=cs)
                cs.synchronize()
                with torch.cuda.graph(g, stream=cs):
                    for i in ids:
                        streams[i].wait_stream(cs)
                        gid.id_factor(copies[i], K, precision=precision, omega=om, workspace=wss[i],
                                      out=outs[i], sync=False, stream=streams[i])
                    for i in ids:
                        cs.wait_stream(streams[i])
            torch.cuda.synchronize()
            return g

        ngroups = max(1, min(args.inflight_groups, depth))
        per = depth // ngroups
        bounds = [(gi * per, depth if gi == ngroups - 1 else (gi + 1) * per) for gi in range(ngroups)]
        groups = [capture(range(lo, hi)) for lo, hi in bounds]
        gstreams = [torch.cuda.Stream() for _ in groups]
        rest = steps % depth
        g_rest = capture(range(rest)) if rest else None

        def round_():
            for g, s_ in zip(groups, gstreams):
                with torch.cuda.stream(s_):
                    g.replay()

        for _ in range(warmup):
            round_()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        cur = torch.cuda.current_stream()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(cur)
        for s_ in gstreams:
            s_.wait_stream(cur)
        for _ in range(steps // depth):
            round_()
        if g_rest is not None:
            with torch.cuda.stream(gstreams[0]):
                g_rest.replay()
        for s_ in gstreams:
            cur.wait_stream(s_)
        t1.record(cur)
        torch.cuda.synchronize()
        barrier()
        return t0.elapsed_time(t1), outs[0]

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    gpu_uuid = None
    try:
        gpu_uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if gpu_uuid and not gpu_uuid.startswith("GPU-"):
            gpu_uuid = "GPU-" + gpu_uuid
    except Exception:
        gpu_uuid = None
    sampler = ClockSampler(gpu_uuid) if rank == 0 else None

    # ---- main timed region: inputs resident in HBM
    if sampler:
        sampler.start()
    total_ms, out_main = run_inflight(args.precision, omega, args.steps, args.warmup, max(1, args.inflight))
    clocks = sampler.stop() if sampler else None
    # one ID at a time (latency of a single ID, graph replay) and the stage split from plain launches
    seq_ms, _, _ = run_loop(args.precision, omega, args.steps, args.warmup, graph=True)
    _, _, stages = run_loop(args.precision, omega, max(3, min(args.steps, 10)), 2, stage=True)
    total_ms = max_over_ranks(total_ms)
    ms_per_step = total_ms / args.steps
    value = world * args.steps / (total_ms / 1e3)
    kernels_per_step = 4

    hbm_peak, bf16_peak, peak_src = measured_peaks()
    sk_ms = stages["sketch_kernel"]
    alg_bytes = sketch_bytes(M, N, ELL)
    achieved = alg_bytes / (sk_ms / 1e3) / 1e9
    sketch_roof = {"kernel": "k_sketch_lowp", "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                   "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": ncu_traffic(),
                   "algorithmic_bytes": alg_bytes, "kernel_ms": sk_ms,
                   "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                   else peak_src}
    cq_ms = stages["cpqr"]
    cq_flops = cpqr_flops(ELL, N, K)
    cq_ach = cq_flops / (cq_ms / 1e3) / 1e12
    fp32_peak = peaks["fp32_tflops"]
    cpqr_roof = {"kernel": "k_cpqr_cluster", "bound": "alu", "achieved": cq_ach, "peak": fp32_peak,
                 "unit": "TFLOP/s", "frac": cq_ach / fp32_peak,
                 "traffic": ncu_traffic("cpqr_solve_110x2000.md", ("cpqr_cluster.cu", "common.cuh")),
                 "algorithmic_flops": cq_flops, "kernel_ms": cq_ms,
                 "peak_source": "FP32 FFMA rate " + peaks["source"],
                 "note": "latency-bound: k sequential cluster-wide pivot steps"}
    # the roofline object describes the stage that takes the longest
    roofline = cpqr_roof if cq_ms >= sk_ms else sketch_roof

    line = {
        "metric": METRIC, "value": value, "unit": "IDs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M, "n": N, "k": K, "ell": ELL, "precision": args.precision,
                   "launch": f"a stream of IDs, {args.inflight} in flight: {min(args.inflight_groups, args.inflight)} "
                             f"CUDA graphs of {args.inflight // min(args.inflight_groups, args.inflight)} IDs on forked "
                             f"streams (own A copy, workspace, outputs each), replayed in turn on their own "
                             f"streams; single-ID latency in latency_ms_per_id; e2e double-buffers A",
                   "l2": "inputs larger than L2 (A is 320 MB vs 129 MB L2); no flush needed"},
        "tflops": id_flops(M, N, ELL, K) * value / 1e12,
        "latency_ms_per_id": seq_ms / args.steps,
        "stages_ms": stages, "roofline": roofline, "sketch_roofline": sketch_roof, "cpqr_roofline": cpqr_roof,
        "alu_peaks": peaks,
        "gpu_launches": kernels_per_step * args.steps,
        "clocks": clocks,
    }

    if not args.no_extras:
        # ---- e2e: A and Omega from pinned host memory each step, outputs back to the host
        host = {"A": torch.from_numpy(a_np).pin_memory(),
                "omega": omega.cpu().pin_memory(),
                "J": torch.empty(N, dtype=torch.int32).pin_memory(),
                # T's device layout (column-major K x (N - K)), pinned: a device-to-host copy
                # into pageable memory would block the host and serialise the steps
                "T": torch.empty((N - K, K), dtype=torch.float64).pin_memory().t(),
                "small": torch.empty(2, dtype=torch.int32).pin_memory()}
        e2e_steps = max(3, min(args.steps, 10))
        e2e_ms = run_e2e(args.precision, host, e2e_steps, 2)
        e2e_ms = max_over_ranks(e2e_ms)
        h2d = 8 * M * N + 2 * ELL * M
        d2h = 4 * N + 8 * K * (N - K) + 8
        line["e2e"] = {"value": world * e2e_steps / (e2e_ms / 1e3), "unit": "IDs/s",
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

        # ---- plain FP64 GPU ID (same A, same Omega in FP64) and the other mixed form (a single
        # bfloat16 piece: faster, not at matched error), each one ID at a time (latency) and as a
        # stream with the same number of IDs in flight
        other = "mixed_bf16" if args.precision != "mixed_bf16" else "mixed_bf16x3"
        depth = max(1, args.inflight)
        p_steps = max(3, min(args.steps, 5))
        p_ms, out_plain, p_stages = run_loop("plain_f64", omega64, p_steps, 1, stage=True)
        p_flight_ms, _ = run_inflight("plain_f64", omega64, depth, 1, depth)
        o_ms, out_other, _ = run_loop(other, omega, args.steps, 2, graph=True)
        o_flight_ms, _ = run_inflight(other, omega, args.steps, 2, depth)
        plain_ids = depth / (p_flight_ms / 1e3)
        other_ids = args.steps / (o_flight_ms / 1e3)
        line["plain_f64"] = {"ids_per_s": plain_ids, "latency_ms_per_id": p_ms / p_steps, "stages_ms": p_stages,
                             "tflops": id_flops(M, N, ELL, K) * plain_ids / 1e12, "inflight": depth,
                             "sketch_fp64_frac": 2.0 * ELL * M * N / (p_stages["sketch_kernel"] / 1e3) / 1e12
                             / peaks["fp64_tflops"]}
        line[other] = {"ids_per_s": other_ids, "latency_ms_per_id": o_ms / args.steps, "inflight": depth}

        # ---- accuracy (FP64 on the GPU): relative 2-norm errors and distances between IDs
        def ahat(out):
            J, T, small, _ = out
            k = int(small[0].item())
            Jn = J.long()
            P_ = torch.zeros((k, N), dtype=torch.float64, device=dev)
            P_[:, Jn[:k]] = torch.eye(k, dtype=torch.float64, device=dev)
            P_[:, Jn[k:]] = T[:k, : N - k]
            return A[:, Jn[:k]] @ P_

        def norm2(X, iters=60):
            g = torch.Generator(device=dev)
            g.manual_seed(0)
            v = torch.randn(X.shape[1], dtype=torch.float64, device=dev, generator=g)
            v /= v.norm()
            s = 0.0
            for _ in range(iters):
                w = X.T @ (X @ v)
                s = float(w.norm().sqrt())
                v = w / w.norm()
            return s

        na = norm2(A)
        h_m, h_p, h_o = ahat(out_main), ahat(out_plain), ahat(out_other)
        d_main = norm2(h_m - h_p) / na
        line["accuracy"] = {
            "form": args.precision, "e": norm2(A - h_m) / na, "e_plain_f64": norm2(A - h_p) / na,
            f"e_{other}": norm2(A - h_o) / na, "d_vs_plain": d_main, f"d_{other}_vs_plain": norm2(h_o - h_p) / na,
            "same_skeleton_as_plain": bool(torch.equal(out_main[0][:K], out_plain[0][:K])),
            "matched_1e-6": d_main <= 1e-6,
            "how": "2-norms by 60 power iterations in FP64 on the GPU; d = ||A_hat - A_hat_plain||_2 / ||A||_2",
        }
        lat_plain = p_ms / p_steps
        line["speedup_vs_plain_f64"] = {
            f"throughput_{args.precision}": value / world / plain_ids,
            f"throughput_{other}": other_ids / plain_ids,
            f"latency_{args.precision}": lat_plain / (seq_ms / args.steps),
            f"latency_{other}": lat_plain / (o_ms / args.steps),
            "matched_1e-6_form": args.precision if d_main <= 1e-6 else None}
        del h_m, h_p, h_o

        # ---- the other workloads: plain FP64 ID of a 1000 x 500 matrix, the 65536 x 1000
        # snapshot matrix at tolerance 1e-6, the differentiable 64 x 2048 x 512 batch
        if not args.no_configs:
            line["plain_1000x500"] = config1_leg(gid, wl, dev, peaks)
            line["low_id_1000x1000"] = low_id_leg(gid, wl, dev, peaks)
            line["row_id_20000x2000"] = row_id_leg(gid, dev, A)
            line["snapshot_65536x1000"] = config3_leg(gid, wl, dev, peaks)
            line["differentiable_64x2048x512"] = config5_leg(gid, wl, dev, peaks)

        # ---- the uneven batch: 512 FP64 matrices in one launch sequence (graph-captured)
        if not args.no_batched:
            line["batched"] = batched_leg(gid, wl, dev, stream, count=args.batch_count, world=world, rank=rank)

        # ---- the FP64 CPU oracle on the host (rank 0, N = 1 only)
        if rank == 0 and world == 1:
            import oracle
            oracle.build()
            ts = []
            t_start = time.perf_counter()
            while len(ts) < 3 and (time.perf_counter() - t_start) < 20.0:
                ts.append(oracle_id_timed(cfg)[0])
            line["cpu_baseline"] = {"value": 1.0 / statistics.mean(ts), "unit": "IDs/s", "cores": 1,
                                    "kind": "oracle",
                                    "sample": f"{len(ts)} full IDs of this workload (FP64 oracle, plain C, "
                                              f"1 thread: sketch, pivoted QR, T solve)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
