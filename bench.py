#!/usr/bin/env python3
"""Benchmark: GAP pull PageRank trials on one GB300 (or N independent replicas).

A step is one paper-compliant PageRank trial (paper §2.3: scratch allocation,
degree binning, every iteration until the summed change < 1e-4, output) on the
Kronecker scale-26 graph (edge factor 16, A/B/C = 0.57/0.19/0.19, symmetrized,
duplicates and self-loops removed, IDs randomly relabelled; paper §2.2 "Kron"
shape), built once on the device before timing (graph construction is
outside the trial, paper §1 and §2.3).  The CSC (8+ GB) is larger than L2, so
no L2 flush is needed between steps.

value = arcs traversed per second over the timed trials = sum(m * iterations)
/ time, in Gedges/s (m = stored directed arcs).  With N ranks each rank runs
its own replica (the path has no exchange step on one graph per GPU: "replicas
only"), time is the max over ranks and value sums all ranks' arcs.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PageRank Gedges/s per iter, %HBM peak; FP32 vs FP64 at L1<=1e-4; PPR p99 ms"
UNIT = "Gedges/s"
DAMPING = 0.85
TOL = 1e-4
MAX_ITERS = 100
FALLBACK_HBM_GBS = 6800.0

# ncu DRAM bytes (read + write) per launch, from one capture of the launch list
# (profiles/pull_segmented_kron26.md); only kernels unchanged since then.
NCU_TRAFFIC = {"k_pull_group_seg<32>": 0.8855e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gap", choices=["gap", "reference"])
    ap.add_argument("--graph", default="kron", choices=["kron", "urand"],
                    help="kron: Kronecker (symmetrized); urand: uniform random digraph")
    ap.add_argument("--scale", type=int, default=26, help="log2 of the vertex count")
    ap.add_argument("--edge-factor", type=int, default=16)
    ap.add_argument("--seed", type=lambda s: int(s, 0), default=0x26)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="convergence loop driver (host: one launch per kernel, visible to ncu)")
    ap.add_argument("--segment-bytes", type=int, default=0, help="L2 blocking segment size (0 = default)")
    return ap.parse_args()


def workload_config(a):
    if a.graph == "urand":
        return {"workload": f"urand{a.scale}-deg{a.edge_factor} directed pull PageRank FP32, d=0.85, "
                            f"tol=1e-4", "graph": "uniform random digraph", "scale": a.scale,
                "edge_factor": a.edge_factor, "symmetrized": False, "seed": hex(a.seed),
                "trial": "alloc+binning+iterations+output (paper §2.3)",
                "l2": "inputs larger than L2 (CSC > 129 MB), no flush"}
    return {"workload": f"kron{a.scale}-ef{a.edge_factor}-sym pull PageRank FP32, d=0.85, tol=1e-4",
            "graph": "kronecker", "scale": a.scale, "edge_factor": a.edge_factor,
            "A_B_C": [0.57, 0.19, 0.19], "symmetrized": True, "seed": hex(a.seed),
            "trial": "alloc+binning+iterations+output (paper §2.3)",
            "l2": "inputs larger than L2 (CSC > 129 MB), no flush"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max((float(r[2]) for r in rows if r[2].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def roofline_entry(sp, m, n, segments, contrib_bytes=4):
    """Roofline of the dominant pull kernel from a timing=1 trial: algorithmic
    bytes of its degree bin (8 B per arc: index + gathered contribution; 24 B per
    row: offsets, out-degree, x read/write, c write) over its launch time."""
    from paper_1508_03619_gb300 import gap
    pulls = list(gap.PULL_PHASES)
    dom = max(pulls, key=lambda k: sp["phase_ms"][k])
    q = pulls.index(dom)
    b = sp["bins"][q]
    per_arc = 4 + contrib_bytes
    per_row = 20 + contrib_bytes
    alg_bin = per_arc * b["arcs"] + per_row * b["rows"]
    launches = max(1, sp["phase_launches"][dom])
    iters = max(1, sp["iterations"])
    per_launch_alg = alg_bin * iters / launches
    per_launch_ms = sp["phase_ms"][dom] / launches
    peak, peak_kind = measured_hbm_peak()
    achieved = per_launch_alg / (per_launch_ms / 1e3) / 1e9
    lanes = b["lanes"]
    kname = {0: "k_pull_hub_chunks", 256: "k_pull_cta"}.get(
        lanes, ("k_pull_group_seg<%d>" if b["segmented"] else "k_pull_group<%d>") % lanes)
    if q == 0:
        kname = "k_pull_zero"
    elif q == 1 and lanes == 1:
        kname = "k_pull_short"
    loop_ms = sum(sp["phase_ms"][k] for k in pulls + ["hub_fixup", "finalize"])
    iter_ms = loop_ms / iters
    iter_bytes = per_arc * m + per_row * n
    total_ms = sum(sp["phase_ms"].values())
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(kname),
            "kernel": f"{kname} (bin {q}: in-degree <= {b['max_degree']}, "
                      f"{'segmented' if b['segmented'] else 'whole rows'})",
            "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)" if peak_kind == "measured"
            else "fallback 6.8 TB/s",
            "alg_bytes_per_launch": per_launch_alg, "launch_ms": per_launch_ms,
            "share_of_trial": sp["phase_ms"][dom] / total_ms if total_ms else None,
            "segments": segments,
            "iteration": {"alg_bytes": iter_bytes, "ms": iter_ms,
                          "achieved_gbs": iter_bytes / (iter_ms / 1e3) / 1e9,
                          "frac": iter_bytes / (iter_ms / 1e3) / 1e9 / peak,
                          "gedges_per_s": m / (iter_ms / 1e3) / 1e9},
            "phase_ms": sp["phase_ms"], "bins": sp["bins"]}


def cpu_baseline(a, seconds=12.0):
    """The oracle (single-threaded FP64 push PageRank) on a bounded sample of
    the workload: the same generator at a smaller scale, fixed iterations."""
    import gapgen
    import oracle
    scale = min(a.scale, 21)
    n = 1 << scale
    src, dst = gapgen.kron(scale, a.edge_factor, a.seed)
    off, idx = oracle.build_csr(n, src, dst, symmetrize=True)
    m = len(idx)
    t0 = time.perf_counter()
    oracle.pagerank(off, idx, DAMPING, 0.0, 1)
    t1 = time.perf_counter() - t0
    iters = max(1, min(30, int(seconds / max(t1, 1e-3))))
    t0 = time.perf_counter()
    _, k, _ = oracle.pagerank(off, idx, DAMPING, 0.0, iters)
    dt = time.perf_counter() - t0
    return {"value": m * k / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"kron scale {scale} (n={n}, m={m}), {k} FP64 push iterations, single thread, "
                      f"{dt:.1f} s"}


def run_reference(a, ws, rank):
    if rank != 0:
        return
    import gapgen
    import oracle
    scale = min(a.scale, 21)
    n = 1 << scale
    src, dst = gapgen.kron(scale, a.edge_factor, a.seed)
    off, idx = oracle.build_csr(n, src, dst, symmetrize=True)
    m = len(idx)
    for _ in range(a.warmup):
        oracle.pagerank(off, idx, DAMPING, 0.0, 1)
    t0 = time.perf_counter()
    total_iters = 0
    for _ in range(a.steps):
        _, k, _ = oracle.pagerank(off, idx, DAMPING, 0.0, 2)
        total_iters += k
    dt = time.perf_counter() - t0
    value = m * total_iters / dt / 1e9
    sample = (f"kron scale {scale} (n={n}, m={m}) sample of the kron{a.scale} workload; each step = "
              f"2 FP64 push iterations of the single-threaded oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(a),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    a = parse()
    ws, rank, local = dist_env()
    if a.impl == "reference":
        run_reference(a, ws, rank)
        return

    import numpy as np
    import torch

    import gapgen
    from paper_1508_03619_gb300 import gap

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    # ---- graph (untimed) ----
    if a.graph == "urand":
        src, dst = gapgen.urand_device(1 << a.scale, a.edge_factor << a.scale, a.seed, device=dev)
        g = gap.Graph.from_edges(1 << a.scale, src, dst, symmetrize=False)
    else:
        src, dst = gapgen.kron_device(a.scale, a.edge_factor, a.seed, device=dev)
        g = gap.Graph.from_edges(1 << a.scale, src, dst, symmetrize=True)
    del src, dst
    torch.cuda.empty_cache()
    n, m = g.n, g.m
    stream = torch.cuda.current_stream(dev)
    scores = torch.empty(n, dtype=torch.float32, device=dev)
    opts = gap.gap_pr_options_default()
    opts.loop = gap.GAP_LOOP_HOST if a.loop == "host" else gap.GAP_LOOP_GRAPH
    opts.segment_bytes = a.segment_bytes

    def trial(out, o=opts):
        gap.gap_pr_run_ex(g.handle, DAMPING, TOL, MAX_ITERS, o, out)

    for _ in range(a.warmup):
        trial(scores)
    gap.gap_pr_stats(g.handle)

    # ---- timed region: K trials, device-resident inputs ----
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    if pg:
        pg.barrier()
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(a.steps):
        trial(scores)
        status, st = gap.gap_pr_stats(g.handle)  # per-trial iteration count (syncs)
        iters.append(st["iterations"])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches = st["kernel_launches"] * a.steps
    if pg:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    arcs = m * sum(iters) * ws
    value = arcs / (ms / 1e3) / 1e9

    # ---- end to end through the C ABI with a pinned host output buffer ----
    host_scores = torch.empty(n, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_iters = []
    e0.record(stream)
    for _ in range(a.steps):
        trial(host_scores)
        _, st_e = gap.gap_pr_stats(g.handle)
        e_iters.append(st_e["iterations"])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e_ms = e0.elapsed_time(e1)
    e2e = {"value": m * sum(e_iters) / (e_ms / 1e3) / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 4 * n,
           "note": "gap_pr_run into pinned host memory (D2H of the FP32 scores inside the step); "
                   "the graph stays resident between trials (paper §2.3)"}

    # ---- per-kernel durations (CUDA events around every launch) ----
    prof = gap.gap_pr_options_default()
    prof.timing = 1
    prof.segment_bytes = a.segment_bytes
    trial(scores, prof)
    _, sp = gap.gap_pr_stats(g.handle)
    roofline = roofline_entry(sp, m, n, sp["segments"])

    # ---- FP64 GPU path on the same graph (metric: FP32 vs FP64 at L1 <= 1e-4) ----
    fp64 = None
    if not a.no_fp64:
        o64 = gap.gap_pr_options_default()
        o64.precision = gap.GAP_PREC_F64
        x64 = torch.empty(n, dtype=torch.float64, device=dev)
        gap.gap_pr_run_ex(g.handle, DAMPING, TOL, MAX_ITERS, o64, x64)
        gap.gap_pr_stats(g.handle)
        k64 = max(1, min(3, a.steps))
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        it64 = 0
        f0.record(stream)
        for _ in range(k64):
            gap.gap_pr_run_ex(g.handle, DAMPING, TOL, MAX_ITERS, o64, x64)
            _, s64 = gap.gap_pr_stats(g.handle)
            it64 += s64["iterations"]
        f1.record(stream)
        torch.cuda.synchronize(dev)
        v64 = m * it64 / (f0.elapsed_time(f1) / 1e3) / 1e9
        l1 = float((x64 - scores.double()).abs().sum().item())
        fp64 = {"value": v64, "unit": UNIT, "fp32_speedup": value / ws / v64 if v64 else None,
                "l1_fp32_vs_fp64": l1, "iterations": s64["iterations"]}

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**workload_config(a), "n": n, "m": m,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "iterations": iters, "clocks": clk, "e2e": e2e, "gpu_launches": launches,
        "roofline": roofline, "fp64": fp64,
    }
    if not a.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(a)
    print(json.dumps(line))
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
