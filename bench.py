#!/usr/bin/env python3
"""Benchmark of the exact variable-length matrix profile on GB300.

One step = the whole hot path over one synthetic workload: mad_profile over
[lmin, lmax] (window statistics, the diagonal-recurrence matrix profile with
top-p candidates, length extension with the Eq. LB bound test, recomputes,
VALMP, per-length discord tables) plus the read-outs (top-k motifs and the
Top-k m-th discords with their FP64 re-checks).

Metric: distance cells per second over all lengths, sum over series of
n^2 * |L|, per step. The default workload is the planted random walk
(n = 65536, l in [256, 512], p = 5). Input series stay resident in HBM
between steps; L2 (129 MB) is flushed between timed steps by writing a
512 MB buffer.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Rank 0 prints one JSON line. Under torchrun every rank profiles its own
replica of the workload (the path has no exchange step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "distance cells/s over all lengths (n^2*|L|)"
UNIT = "cells/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
OPS_PER_CELL = 4            # FFMA, FFMA (recurrence), FMUL (key), FSETP (threshold test)
# Measured peaks of the GB300s (MEASURED_PEAKS.json when the
# driver has written it; else the values it wrote earlier, recorded here)
RECORDED_PEAKS = {"hbm_gbs": 6775.6, "bf16_tflops": 1906.5, "bf16_tflops_sustained": 1723.6}


def measured_peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return {k: float(d[k]) for k in RECORDED_PEAKS if k in d} or dict(RECORDED_PEAKS), "MEASURED_PEAKS.json"
    except (OSError, ValueError, KeyError, TypeError):
        return dict(RECORDED_PEAKS), "recorded copy of the driver's measurement"


PRECISIONS = {"fp32": lambda mad: mad.MAD_FP32, "fp64": lambda mad: mad.MAD_FP64,
              "split_tc": lambda mad: mad.MAD_SPLIT_TC}
DTYPES = {"fp32": "f32", "fp64": "f64", "split_tc": "f32 (direct path: f16 hi+lo on tensor cores)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="planted65k")
    ap.add_argument("--precision", default="fp32", choices=list(PRECISIONS))
    ap.add_argument("--lrange", default=None, metavar="LMIN:LMAX",
                    help="override the workload's length range (every series)")
    ap.add_argument("--fp64-steps", type=int, default=3, help="timed steps of the plain FP64 GPU path")
    ap.add_argument("--fp64-lrange", default=None, metavar="LMIN:LMAX",
                    help="time the plain FP64 path (and the chosen path again, for a like-for-like ratio) on this "
                         "sub-range of lengths only (for workloads whose full FP64 step takes minutes)")
    ap.add_argument("--e2e-steps", type=int, default=3, help="timed end-to-end repetitions (median)")
    ap.add_argument("--graphs", type=int, default=1, choices=[0, 1],
                    help="1: repeated profiles replay a captured CUDA graph (default); 0: launched one by one")
    ap.add_argument("--tc-tma", type=int, default=0, choices=[0, 1],
                    help="split_tc: 0 column tiles built by the kernel's producer warps (default); "
                         "1 loaded by TMA from per-length shifted copies")
    ap.add_argument("--band-form", type=int, default=0, choices=[0, 1],
                    help="0: full rows; 1: symmetric band form when most bands are active")
    ap.add_argument("--no-fp64-path", action="store_true", help="skip timing the plain FP64 GPU path")
    ap.add_argument("--no-motif-path", action="store_true", help="skip timing the motif mode (mode 1)")
    ap.add_argument("--no-discord-path", action="store_true", help="skip timing the discord mode (mode 2)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the CPU oracle sample")
    ap.add_argument("--p-sweep", default=None, metavar="LMIN:LMAX",
                    help="pruning versus p: profile the workload over [LMIN, LMAX] for p in 5..64 and print one "
                         "JSON line (certified / recomputed fractions, time)")
    ap.add_argument("--ncu-case", default=None, metavar="LMIN:LMAX",
                    help="profile the workload once over [LMIN, LMAX] and exit (a small case for ncu captures)")
    ap.add_argument("--mode", type=int, default=0, choices=[0, 1, 2],
                    help="with --ncu-case: 0 exact rows, 1 motif mode, 2 discord mode")
    return ap.parse_args()


def run_p_sweep(args):
    """Pruning versus the number p of stored entries per row (Sec. 7.2): the
    fractions of rows certified and recomputed after lmin, and the time."""
    import time
    import paper_2008_13447_gb300 as mad
    import workloads
    w = workloads.make(args.workload)
    a, b = (int(v) for v in args.p_sweep.split(":"))
    prec = PRECISIONS[args.precision](mad)
    x = w.series[0]
    res = []
    for p in (5, 10, 20, 40, 64):
        ctx = mad.mad_create(x, precision=prec, k_max=w.k, m_max=1, band_form=args.band_form)
        try:
            mad.mad_profile(ctx, a, b, p)          # warm-up
            t = time.perf_counter()
            mad.mad_profile(ctx, a, b, p)
            dt = time.perf_counter() - t
            st = mad.mad_stats(ctx, 0)[1:]
        finally:
            mad.mad_destroy(ctx)
        rows = sum(s["rows"] for s in st)
        res.append({"p": p, "certified_frac": sum(s["certified"] for s in st) / rows,
                    "recomputed_frac": sum(s["recomputed"] for s in st) / rows,
                    "direct_rows": sum(s["direct_rows"] for s in st), "ms": dt * 1e3})
    print(json.dumps({"p_sweep": res, "workload": args.workload, "lengths": [a, b], "precision": args.precision}))
    return 0


def run_ncu_case(args):
    """One mad_profile of the workload over a short length range, for
    profiler captures (the first length runs the threshold pass and the
    first recompute; later lengths are the steady state)."""
    import paper_2008_13447_gb300 as mad
    import workloads
    w = workloads.make(args.workload)
    a, b = (int(v) for v in args.ncu_case.split(":"))
    prec = PRECISIONS[args.precision](mad)
    ctx = mad.mad_create(w.series[0], precision=prec, k_max=w.k, m_max=w.m, band_form=args.band_form,
                         mode=args.mode)
    try:
        mad.mad_profile(ctx, a, b, w.p)
        for s in mad.mad_stats(ctx, 0):
            print(json.dumps({k: s[k] for k in ("len", "rows", "certified", "recomputed", "band_cells", "band_ms",
                                                "inserts", "direct_rows", "direct_ms", "rows_ms")}))
    finally:
        mad.mad_destroy(ctx)
    return 0


def max_over_ranks(ms, pg, device):
    """The slowest rank's time, on every rank (ms itself with one rank)."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank, world, ms_per_step):
    """Whole-job cells/s: every rank processes its own replica of the
    workload in the step time of the slowest rank."""
    return cells_per_rank * world / (ms_per_step / 1e3)


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- helpers

def kernel_source_hash():
    """Hash of the band kernel's source: its own files and the BandArgs
    declaration (the rest of kernels.cuh declares other kernels)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2008_13447_gb300", "csrc")
    for f in ("k_band.cuh", "k_band_f32.cu", "mad_internal.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    decl = open(os.path.join(csrc, "kernels.cuh")).read()
    a = decl.index("template <typename T> struct BandArgs {")
    h.update(decl[a:decl.index("};", a) + 2].encode())
    return h.hexdigest()[:16]


def measured_traffic(cells_per_launch):
    """DRAM bytes per band-kernel launch from the committed ncu summary,
    scaled by cells; None if absent or taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "band_kernel_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_sha") != kernel_source_hash():
        return None
    return d["dram_bytes_per_cell"] * cells_per_launch


def cpu_oracle_sample(w, seconds):
    """Time the CPU oracle (plain definitions, OpenMP over windows) on a
    bounded sample of the workload: full distance profiles of sampled
    windows at sampled lengths of the range (several series of a batch
    workload: the longest and three drawn at random)."""
    import numpy as np
    import oracle
    threads = oracle.num_threads()
    rng = np.random.default_rng(0)
    if len(w.series) == 1:
        picks = [0]
    else:
        longest = int(np.argmax([len(sx) for sx in w.series]))
        picks = [longest] + [int(v) for v in rng.choice(len(w.series), 3, replace=False) if v != longest][:3]
    plan = []
    for si in picks:
        lmin, lmax = w.lmin[si], w.lmax[si]
        for l in sorted(set(int(v) for v in np.linspace(lmin, lmax, 5 if len(picks) == 1 else 2))):
            plan.append((si, l))
    # calibrate on a few rows of the first series, then size the sample to the budget
    x0 = w.series[picks[0]]
    l0 = plan[len(plan) // 2][1] if len(picks) == 1 else plan[0][1]
    rows = rng.integers(0, len(x0) - l0 + 1, threads)
    t = time.perf_counter()
    oracle.rows(x0, l0, rows)
    per_row = (time.perf_counter() - t) / len(rows) * threads * len(x0) ** -1
    cells = 0
    t0 = time.perf_counter()
    desc = []
    for si, l in plan:
        x = w.series[si]
        n = len(x)
        nrows = max(threads, int(seconds / max(per_row * n, 1e-9) * threads / len(plan)))
        rows = rng.integers(0, n - l + 1, nrows)
        oracle.rows(x, l, rows)
        cells += nrows * (n - l + 1)
        desc.append("%d x l=%d of series %d (n=%d)" % (nrows, l, si, n) if len(picks) > 1 else "%d x l=%d" % (nrows, l))
    dt = time.perf_counter() - t0
    return {"value": cells / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%s of %s: full FP64 distance profiles of sampled windows by definition, %.1f s"
                      % ("; ".join(desc), w.name, dt),
            "seconds": dt, "cells": cells}


# ------------------------------------------------------------ reference arm

def workload_config(name, w):
    """The workload fields of the JSON line's config, shared by both arms."""
    base = {"workload": name, "p": w.p, "k": w.k, "m": w.m, "exclusion": "ceil(l/4)", "cells_per_step": w.cells}
    if len(w.series) == 1:
        return {**base, "n": len(w.series[0]), "lmin": w.lmin[0], "lmax": w.lmax[0]}
    ns = [len(sx) for sx in w.series]
    return {**base, "series": len(ns), "n_min": min(ns), "n_max": max(ns), "n_total": sum(ns),
            "lmin": "per series, %d..%d" % (min(w.lmin), max(w.lmin)), "lmax": "2 * lmin",
            "lengths_total": int(sum(b - a + 1 for a, b in zip(w.lmin, w.lmax)))}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = make_workload(args)
    per = max(2.0, min(20.0, 90.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_sample(w, per / 4)
    vals, secs, samp = [], 0.0, None
    for _ in range(args.steps):
        r = cpu_oracle_sample(w, per)
        vals.append(r["value"])
        secs += r["seconds"]
        samp = r
    value = statistics.median(vals)
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(args.workload, w),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": samp["cores"], "kind": "oracle",
                            "sample": samp["sample"]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------------------- our arm

def parse_range(txt):
    a, b = (int(v) for v in txt.split(":"))
    return a, b


# Length ranges used when a workload's full range would take too long for one
# bench step (stated in the JSON line's config as "lengths").
DEFAULT_RANGE = {"seismic2m": (256, 264)}


def make_workload(args):
    import workloads
    w = workloads.make(args.workload)
    rng = parse_range(args.lrange) if args.lrange else DEFAULT_RANGE.get(args.workload)
    if rng is not None:
        w.lmin = [rng[0]] * len(w.series)
        w.lmax = [rng[1]] * len(w.series)
    return w


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.ncu_case:
        return run_ncu_case(args)
    if args.p_sweep:
        return run_p_sweep(args)
    import numpy as np
    import torch
    import paper_2008_13447_gb300 as mad

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    w = make_workload(args)
    mad.mad_set_graphs(args.graphs)
    mad.mad_debug_tc_tma(args.tc_tma)
    batch = len(w.series) > 1
    p, k, m = w.p, w.k, w.m
    prec = PRECISIONS[args.precision](mad)
    cells = w.cells
    ns = len(w.series)
    if batch:
        ctx = mad.mad_create_batch(w.series, precision=prec, k_max=k, m_max=m, stream=stream,
                                   band_form=args.band_form)
    else:
        x = w.series[0]
        xt = torch.tensor(x, device=dev, dtype=torch.float64)
        ctx = mad.mad_create_device(xt, precision=prec, k_max=k, m_max=m, stream=stream, band_form=args.band_form)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def profile(c):
        if batch:
            mad.mad_profile_batch(c, w.lmin, w.lmax, p)
        else:
            mad.mad_profile(c, w.lmin[0], w.lmax[0], p)

    def readouts(c):
        mot = [mad.mad_motifs(c, s, k) for s in range(ns)]
        dis = [mad.mad_discords(c, s, k, m) for s in range(ns)]
        return mot, dis

    def step(c):
        profile(c)
        return readouts(c)

    for _ in range(args.warmup):
        step(ctx)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    acc = dict(band_ms=0.0, direct_ms=0.0, rows_ms=0.0, band_cells=0, launches=0, band_launches=0,
               rows_after=0, recomputed_after=0, direct_rows=0, graph=0, direct_flops=0.0)
    for si in range(args.steps):
        flush.fill_(si & 0xff)
        torch.cuda.synchronize()
        ev[si][0].record(stream)
        step(ctx)
        ev[si][1].record(stream)
        torch.cuda.synchronize()
        for s in range(ns):
            st = mad.mad_stats(ctx, s)
            lmin_s = w.lmin[s]
            for q in st:
                acc["band_ms"] += q["band_ms"]
                acc["direct_ms"] += q["direct_ms"]
                acc["rows_ms"] += q["rows_ms"]
                acc["band_cells"] += q["band_cells"]
                acc["launches"] += q["launches"]
                acc["graph"] = max(acc["graph"], q["graph"])
                if q["band_cells"] > 0:
                    acc["band_launches"] += q["passes"] + (1 if q["len"] == lmin_s else 0)
                if q["len"] > lmin_s:
                    acc["rows_after"] += q["rows"]
                    acc["recomputed_after"] += q["recomputed"]
                    acc["direct_rows"] += q["direct_rows"]
                # direct path: per listed row and column, l multiply-adds per
                # product; the split form takes three products (hi*hi, hi*lo, lo*hi)
                acc["direct_flops"] += q["direct_rows"] * q["rows"] * 2.0 * q["len"]
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), pg, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(cells, world, ms_per_step)
    K = args.steps

    # read-out launches per step (motif rounds, pair re-check, discord re-check)
    launches_per_step = acc["launches"] / K + ns * (2 * k + 1 + 1)

    # roofline of the dominant kernel (band kernel): FP32 ALU instructions
    peak_mhz = (clk or {}).get("sm_max_mhz", 2070.0)
    peak_ops = SM_COUNT * FP32_LANES_PER_SM * peak_mhz * 1e6
    band_ms, band_cells = acc["band_ms"], acc["band_cells"]
    achieved_ops = band_cells * OPS_PER_CELL / (band_ms / 1e3) if band_ms > 0 else 0.0
    cells_per_launch = band_cells / max(1, acc["band_launches"])
    traffic = measured_traffic(cells_per_launch) if prec == mad.MAD_FP32 else None
    roof = {"bound": "alu", "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
            "frac": achieved_ops / peak_ops if peak_ops else None, "traffic": traffic,
            "kernel": "k_band (FP32 diagonal recurrence, append mode)" if prec == mad.MAD_FP32
            else "k_band (%s)" % args.precision,
            "ops_per_cell": OPS_PER_CELL, "band_cells_per_step": band_cells / K,
            "band_ms_per_step": band_ms / K}
    if prec == mad.MAD_SPLIT_TC and acc["direct_ms"] > 0:
        peaks, src = measured_peaks()
        flops = 3.0 * acc["direct_flops"]
        ach = flops / (acc["direct_ms"] / 1e3) / 1e12
        roof_tc = {"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
                   "frac": ach / peaks["bf16_tflops_sustained"], "traffic": None,
                   "kernel": "k_direct_tc (tcgen05, FP16 hi+lo, 3 products per lag, FP32 accumulation)",
                   "peak_source": "BF16 dense sustained, " + src + " (FP16 runs at the BF16 rate)",
                   "flops_per_step": flops / K, "direct_ms_per_step": acc["direct_ms"] / K}
        if acc["direct_ms"] > band_ms:
            roof_tc["band_kernel"] = roof
            roof = roof_tc
        else:
            roof["tensor_core_direct_path"] = roof_tc
    kernels = {"band_ms_per_step": band_ms / K, "direct_ms_per_step": acc["direct_ms"] / K,
               "rows_ms_per_step": acc["rows_ms"] / K,
               "other_ms_per_step": ms_per_step - (band_ms + acc["direct_ms"] + acc["rows_ms"]) / K}
    pruning = {"rows_after_lmin": acc["rows_after"] // K,
               "recomputed_frac_after_lmin": (acc["recomputed_after"] / acc["rows_after"]) if acc["rows_after"] else None,
               "direct_rows_per_step": acc["direct_rows"] // K,
               "paper_recomputed_frac": "<= 0.002 (motifs, default parameters, real data)"}

    cfg = {**workload_config(args.workload, w), "precision": args.precision, "band_form": args.band_form,
           "l2": "flushed between timed steps (512 MB write)", "parallelism": "replicas",
           "graph_replay": bool(acc["graph"]), "graphs_option": args.graphs}
    if args.precision == "split_tc":
        cfg["tc_column_tiles"] = "tma" if args.tc_tma else "built"
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
           "config": cfg, "roofline": roof, "kernels": kernels, "pruning": pruning,
           "gpu_launches": int(round(launches_per_step * args.steps)), "clocks": clk}

    # plain FP64 GPU path: one warm-up step, then timed steps (median); on a
    # stated sub-range of lengths for the largest workloads, with the chosen
    # path timed again on the same sub-range
    if rank == 0 and not args.no_fp64_path and prec != mad.MAD_FP64:
        sub = parse_range(args.fp64_lrange) if args.fp64_lrange else None
        lo = [sub[0]] * ns if sub else w.lmin
        hi = [sub[1]] * ns if sub else w.lmax
        cells_sub = float(sum(len(sx) ** 2 * (b - a + 1) for sx, a, b in zip(w.series, lo, hi)))

        def step_sub(c):
            if batch:
                mad.mad_profile_batch(c, lo, hi, p)
            else:
                mad.mad_profile(c, lo[0], hi[0], p)
            return readouts(c)

        def timed(c, reps):
            step_sub(c)
            ts = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.fill_(7)
                torch.cuda.synchronize()
                e0.record(stream)
                step_sub(c)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return ts

        if batch:
            c64 = mad.mad_create_batch(w.series, precision=mad.MAD_FP64, k_max=k, m_max=m, stream=stream,
                                       band_form=args.band_form)
        else:
            c64 = mad.mad_create_device(xt, precision=mad.MAD_FP64, k_max=k, m_max=m, stream=stream,
                                        band_form=args.band_form)
        try:
            t64 = timed(c64, args.fp64_steps)
        finally:
            mad.mad_destroy(c64)
        ms64 = statistics.median(t64)
        ms_same = ms_per_step
        if sub:
            ms_same = statistics.median(timed(ctx, args.fp64_steps))
        out["fp64_path"] = {"value": cells_sub / (ms64 / 1e3), "ms_per_step": ms64, "steps": len(t64), "warmup": 1,
                            "ms_all": t64, "lengths": "all" if not sub else "%d..%d" % sub,
                            "cells_per_step": cells_sub,
                            "speedup_of_%s" % args.precision: ms64 / ms_same}

    # motif mode (Algorithm 1 with ComputeSubMP): the same workload, only the
    # motif of each length guaranteed; one warm-up step, one timed step
    if rank == 0 and not args.no_motif_path and m == 1 and not batch:
        cm = mad.mad_create_device(xt, precision=prec, k_max=k, m_max=1, stream=stream, mode=1)
        try:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for rep in range(2):
                flush.fill_(7)
                torch.cuda.synchronize()
                e0.record(stream)
                profile(cm)
                mot1 = mad.mad_motifs(cm, 0, k)
                e1.record(stream)
                torch.cuda.synchronize()
            ms1 = e0.elapsed_time(e1)
            st1 = mad.mad_stats(cm, 0)
            rows = sum(s["rows"] for s in st1)
            comp = sum(s["rows"] if (i == 0 or s["full_profile"]) else s["recomputed"] for i, s in enumerate(st1))
            out["motif_mode_path"] = {
                "value": cells / (ms1 / 1e3), "ms_per_step": ms1,
                "rows_computed_frac": comp / rows,
                "full_profile_lengths": int(sum(s["full_profile"] for s in st1[1:])),
                "top_motif": {kk: mot1[0][kk] for kk in ("a", "b", "len", "dist", "dist_recheck")} if mot1 else None}
        finally:
            mad.mad_destroy(cm)

    # discord mode (Algorithm 7 driving Algorithm 10): the same workload, the
    # Top-k m-th discords with the paper's pruning; one warm-up, one timed step
    if rank == 0 and not args.no_discord_path and not batch:
        cd = mad.mad_create_device(xt, precision=prec, k_max=k, m_max=m, stream=stream, mode=2)
        try:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for rep in range(2):
                flush.fill_(7)
                torch.cuda.synchronize()
                e0.record(stream)
                profile(cd)
                dis2 = mad.mad_discords(cd, 0, k, m)
                e1.record(stream)
                torch.cuda.synchronize()
            ms2 = e0.elapsed_time(e1)
            st2 = mad.mad_stats(cd, 0)
            rows = sum(s["rows"] for s in st2)
            comp = st2[0]["rows"] + sum(s["recomputed"] for s in st2[1:])
            out["discord_mode_path"] = {
                "value": cells / (ms2 / 1e3), "ms_per_step": ms2,
                "rows_computed_frac": comp / rows,
                "top_discord": {kk: dis2[0][kk] for kk in ("off", "len", "dist", "dist_recheck")} if dis2 else None}
        finally:
            mad.mad_destroy(cd)

    # end to end through the public API with host buffers (pinned input):
    # create from host memory, profile, read-outs and VALMP back to the host,
    # destroy; one untimed repetition, then the median of timed ones
    pinned = [torch.from_numpy(np.ascontiguousarray(sx)).pin_memory() for sx in w.series]
    hosts = [pt.numpy() for pt in pinned]
    e2e_ms = []
    for rep in range(1 + args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if batch:
            c2 = mad.mad_create_batch(hosts, precision=prec, k_max=k, m_max=m, stream=stream,
                                      band_form=args.band_form)
        else:
            c2 = mad.mad_create(hosts[0], precision=prec, k_max=k, m_max=m, stream=stream, band_form=args.band_form)
        try:
            mot, dis = step(c2)
            vms = [mad.mad_valmp(c2, s, len(w.series[s]) - w.lmin[s] + 1) for s in range(ns)]
        finally:
            mad.mad_destroy(c2)
        if rep > 0:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e = max_over_ranks(statistics.median(e2e_ms), pg, dev)
    n0s = [len(sx) - a + 1 for sx, a in zip(w.series, w.lmin)]
    d2h = sum(n0 * (8 + 8 + 4 + 4) for n0 in n0s) + ns * (k * 56 + k * m * 56)
    out["e2e"] = {"value": job_throughput(cells, world, e2e), "unit": UNIT,
                  "h2d_bytes_per_step": int(sum(len(sx) * 8 for sx in w.series)),
                  "d2h_bytes_per_step": d2h, "ms_per_step": e2e, "steps": len(e2e_ms)}
    mot0, dis0 = mot[0], dis[0]
    out["result"] = {"top_motif": {k2: mot0[0][k2] for k2 in ("a", "b", "len", "dist", "dist_recheck")} if mot0 else None,
                     "top_discord": {k2: dis0[0][k2] for k2 in ("off", "len", "dist", "dist_recheck")} if dis0 else None,
                     "valmp_len_mean": float(np.mean(np.concatenate([v["len"] for v in vms])))}
    mad.mad_destroy(ctx)
    if rank == 0 and not args.no_cpu_baseline:
        cb = cpu_oracle_sample(w, args.cpu_seconds)
        out["cpu_baseline"] = {k2: cb[k2] for k2 in ("value", "unit", "cores", "kind", "sample")}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
