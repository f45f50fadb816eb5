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

The same JSON line also carries (rank 0, N = 1, default --workload all):
  "batch": PageRank on the uneven batch of 256 graphs (128 R-MAT + 128 grids,
           2^10..2^18 vertices) in one persistent launch, Gedges/s and the
           persistent kernel's roofline;
  "ppr":   personalized-PageRank serving on a Chung-Lu graph (2^24 vertices,
           5e8 arc draws, exponent 2.1): saturated queries/s, Poisson arrivals
           at 0.25/0.5/0.9 of it with p50/p99 latency, and one-at-a-time
           queries/s;
  "cc":    Connected Components (paper §2.1 CC) trials on the same graph as the
           main line: trial time, arcs per second and a bandwidth figure;
  "bfs":   direction-optimizing BFS (paper §2.1 BFS) from 64 sources of
           non-zero degree on the same graph (§2.3): trial times and arcs per
           second.
--workload batch|ppr|cc|bfs prints a line for that workload alone.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--workload all|pagerank|batch|ppr|cc|bfs]
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

# ncu DRAM bytes of one k_batch_persistent launch on the 256-graph batch with this
# tuning (one capture of that launch; the batch is its own small case)
BATCH_NCU_TRAFFIC = None  # no capture of the current kernel yet
BATCH_NCU_TUNING = {"heavy_min_degree": 512, "chunk_arcs": 2048, "block_threads": 512, "blocks_per_sm": 0}
# ncu DRAM bytes (read + write) of one launch of each segmented pull kernel on the
# small case (kron26 at edge factor 4: the benchmark's vertex count and source
# segments, a quarter of its arcs), with the arcs that launch streams and the bytes
# it streams per arc (column index; the packed COO pass also streams the row id).
# Full-size traffic per launch = the captured bytes with the streamed part rescaled
# to the full launch's arcs; the rest (one segment of contributions, row data, the
# COO pass's running row sums) is per launch and does not grow with the arcs.
NCU_SMALL = {  # kernel: (DRAM bytes, arcs in the launch, streamed bytes per arc)
    "k_pull_group_seg<32>": (143.52e6, 184692430 / 8, 4),
    "k_pull_group_seg<8>": (124.96e6, 97466713 / 8, 4),
    "k_pull_small_coo<float,8,32>": (783.79e6, 234491820 / 8, 8),
    "k_pull_hub_chunks": (38.70e6, 16262037 / 8, 4),
}


def scaled_traffic(kname, arcs_per_launch):
    """DRAM bytes per launch of kernel kname at arcs_per_launch streamed arcs,
    from its small-case capture (None when the kernel has no capture)."""
    if kname not in NCU_SMALL:
        return None
    small, small_arcs, per_arc = NCU_SMALL[kname]
    return small + per_arc * (arcs_per_launch - small_arcs)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=16, help="timed trials (the paper runs 16)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gap", choices=["gap", "reference"])
    ap.add_argument("--graph", default="kron", choices=["kron", "urand"],
                    help="kron: Kronecker (symmetrized); urand: uniform random digraph")
    ap.add_argument("--scale", type=int, default=26, help="log2 of the vertex count")
    ap.add_argument("--edge-factor", type=int, default=16)
    ap.add_argument("--seed", type=lambda s: int(s, 0), default=0x26)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the full-size FP64 oracle run behind error_vs_oracle")
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="convergence loop driver (host: one launch per kernel, visible to ncu)")
    ap.add_argument("--segment-bytes", type=int, default=0, help="L2 blocking segment size (0 = default)")
    ap.add_argument("--workload", default="all", choices=["all", "pagerank", "batch", "ppr", "cc", "bfs"],
                    help="all: the PageRank line with batch, ppr, cc and bfs entries; "
                         "the others: one line for that workload alone")
    ap.add_argument("--ppr-seconds", type=float, default=6.0, help="arrival window per load level")
    ap.add_argument("--ppr-scale", type=int, default=24)
    ap.add_argument("--ppr-edges", type=float, default=5e8)
    ap.add_argument("--ppr-cols", type=int, default=128, help="server columns (power of two, <= 128)")
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
        with open(self.path) as f:
            lines = f.readlines()
        os.unlink(self.path)
        return parse_clock_samples(lines)


def parse_clock_samples(lines):
    """Median SM clock under load, the maximum clock, and the throttle reasons
    seen, from nvidia-smi CSV lines (index, clocks.sm, clocks.max.sm, power,
    active reasons, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap)."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
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
    if lanes == -1:  # vertex-order warp-merge of the small rows
        kname = "k_pull_small_coo<float,8,32>" if segments > 1 else "k_pull_small<float,4>"
    elif lanes == 0:
        kname = "k_pull_hub_chunks"
    elif lanes == 256:
        kname = "k_pull_cta"
    else:
        kname = ("k_pull_group_seg<%d>" if b["segmented"] else "k_pull_group<%d>") % lanes
    loop_ms = sum(sp["phase_ms"][k] for k in pulls + ["hub_fixup", "finalize"])
    iter_ms = loop_ms / iters
    iter_bytes = per_arc * m + per_row * n
    total_ms = sum(sp["phase_ms"].values())
    traffic = scaled_traffic(kname, b["arcs"] * iters / launches)
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch on kron26 at "
                              "edge factor 4, streamed arc bytes rescaled to this launch's arcs",
            "useful_byte_efficiency": (per_launch_alg / traffic) if traffic else None,
            "kernel": f"{kname} (bin {q}: in-degree <= {b['max_degree']}, "
                      + ("packed COO, one pass per source segment)" if lanes == -1 and segments > 1 else
                         "segmented)" if b["segmented"] else "whole rows)"),
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
    the workload: the same generator at a smaller scale, fixed iterations.  Also
    a multi-core FP64 pull loop (OpenMP, all host cores) on the same sample."""
    import numpy as np

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
    out = {"value": m * k / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"kron scale {scale} (n={n}, m={m}), {k} FP64 push iterations, single thread, "
                     f"{dt:.1f} s"}
    # the symmetrized sample's CSR is its CSC
    outdeg = np.diff(off).astype(np.int32)
    oracle.cpu_pagerank_pull(off, idx, outdeg, DAMPING, 0.0, 1)
    t0 = time.perf_counter()
    _, kp, threads = oracle.cpu_pagerank_pull(off, idx, outdeg, DAMPING, TOL, MAX_ITERS)
    dtp = time.perf_counter() - t0
    out["openmp_pull"] = {"value": m * kp / dtp / 1e9, "unit": UNIT, "cores": threads,
                          "sample": f"same graph, FP64 pull over the CSC to tol 1e-4 ({kp} iterations), "
                                    f"{threads} OpenMP threads, {dtp:.2f} s"}
    return out


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


def combine_ranks(ms, arcs, pg, device):
    """Whole-job figures of N replicas: the slowest rank's time and every rank's
    arcs.  Without a process group the local figures are returned."""
    if pg is None:
        return ms, arcs
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    c = torch.tensor([float(arcs)], device=device, dtype=torch.float64)
    pg.all_reduce(c, op=pg.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def oracle_cache_dir(a):
    """Where the full-size oracle run of this workload is kept (outside the
    repository), keyed by everything that fixes the graph and the method."""
    root = os.environ.get("GAP_ORACLE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "gap_oracle"))
    key = f"{a.graph}{a.scale}-ef{a.edge_factor}-seed{a.seed:#x}-d{DAMPING}-tol{TOL}-v1"
    return os.path.join(root, key)


def oracle_leg(graph, scale, edge_factor, seed, outdir):
    """The oracle on the full workload, run in a spawned child process while
    the GPU is measured: the same host draws as the device generator makes,
    the oracle's own CSR (row-partitioned builder, identical to the serial
    one), then the single-threaded FP64 push iteration to tol, keeping the
    iterates before, at and after the stop so the GPU's results can be held
    against the oracle's iterate of the same count."""
    import numpy as np

    # lowest priority and two cores left free: the parent's host work (graph
    # capture, launches, synchronizations) runs inside its timed trials
    os.nice(19)
    threads = max(1, (os.cpu_count() or 1) - 2)
    os.environ["GAPGEN_THREADS"] = str(threads)
    import gapgen
    import oracle
    t0 = time.perf_counter()
    n = 1 << scale
    if graph == "urand":
        src, dst = gapgen.urand(n, edge_factor << scale, seed)
        sym = False
    else:
        src, dst = gapgen.kron(scale, edge_factor, seed)
        sym = True
    off, idx = oracle.build_csr(n, src, dst, symmetrize=sym, threads=threads)
    del src, dst
    t1 = time.perf_counter()
    prev = None
    x, k, hist = oracle.pagerank(off, idx, DAMPING, 0.0, 1)
    deltas = [float(hist[0])]
    while deltas[-1] >= TOL and k < MAX_ITERS:
        prev = x
        x, _, h = oracle.pagerank_from(off, idx, x, 1, DAMPING)
        k += 1
        deltas.append(float(h[0]))
    nxt, _, _ = oracle.pagerank_from(off, idx, x, 1, DAMPING)
    t2 = time.perf_counter()
    os.makedirs(outdir, exist_ok=True)
    for name, arr in (("x_prev", prev), ("x_stop", x), ("x_next", nxt)):
        if arr is not None:
            np.save(os.path.join(outdir, name + ".npy"), arr)
    with open(os.path.join(outdir, "meta.json"), "w") as f:
        json.dump({"iterations": k, "deltas": deltas, "m": int(len(idx)), "build_s": t1 - t0,
                   "iterate_s": t2 - t1, "threads_build": threads}, f)


def start_oracle_leg(a):
    """Spawn the oracle leg (nothing to do when its result is cached)."""
    out = oracle_cache_dir(a)
    if os.path.exists(os.path.join(out, "meta.json")):
        return None, out
    import multiprocessing as mp
    p = mp.get_context("spawn").Process(target=oracle_leg, args=(a.graph, a.scale, a.edge_factor, a.seed, out))
    p.start()
    return p, out


def error_vs_oracle(proc, out, gpu):
    """L1 and max relative error of each GPU result (name -> (scores, its
    iteration count)) against the oracle's iterate of the same count."""
    import numpy as np
    t0 = time.perf_counter()
    if proc is not None:
        proc.join()
        if proc.exitcode != 0:
            return {"error": f"oracle leg exited with {proc.exitcode}"}
    with open(os.path.join(out, "meta.json")) as f:
        meta = json.load(f)
    k = meta["iterations"]
    res = {"oracle": "FP64 single-threaded push iterations (paper §2.1 equation) on the oracle's own CSR "
                     "from the same draws; errors against the oracle iterate with the GPU's iteration count",
           "oracle_iterations": k, "oracle_final_delta": meta["deltas"][-1], "m": meta["m"],
           "oracle_seconds": {"csr_build": meta["build_s"], "iterations": meta["iterate_s"],
                              "build_threads": meta["threads_build"]},
           "wait_s": None}
    files = {k - 1: "x_prev", k: "x_stop", k + 1: "x_next"}
    cache = {}
    for name, (x, iters) in gpu.items():
        if iters is None:  # not an iterate of the classical iteration: against the oracle's stop iterate
            xo = cache.get("x_stop")
            if xo is None:
                xo = cache["x_stop"] = np.load(os.path.join(out, "x_stop.npy"))
            diff = np.abs(x - xo)
            res[name] = {"l1_vs_oracle_stop_iterate": float(diff.sum()),
                         "note": "both within d tol / (1 - d) of the fixed point"}
            continue
        f = files.get(iters)
        if f is None or not os.path.exists(os.path.join(out, f + ".npy")):
            res[name] = {"iterations": iters, "l1": None, "max_rel": None,
                         "note": "iteration count more than one away from the oracle's"}
            continue
        if f not in cache:
            cache[f] = np.load(os.path.join(out, f + ".npy"))
        xo = cache[f]
        diff = np.abs(x - xo)
        res[name] = {"iterations": iters, "l1": float(diff.sum()), "max_rel": float(np.max(diff / xo))}
    res["wait_s"] = time.perf_counter() - t0
    return res


def run_pagerank(a, ws, rank, local, dev, pg, want_oracle=False):
    """The headline line: K PageRank trials on the kron (or urand) graph."""
    import torch

    import gapgen
    from paper_1508_03619_gb300 import gap

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
    from paper_1508_03619_gb300 import tuning

    def options():
        """This GPU model's tuned options (autotuner table), --segment-bytes over them."""
        o = tuning.pagerank_options(local)
        if a.segment_bytes:
            o.segment_bytes = a.segment_bytes
        return o

    opts = options()
    opts.loop = gap.GAP_LOOP_HOST if a.loop == "host" else gap.GAP_LOOP_GRAPH

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
    tev = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    ev0.record(stream)
    tev[0].record(stream)
    for k in range(a.steps):
        trial(scores)
        tev[k + 1].record(stream)
        status, st = gap.gap_pr_stats(g.handle)  # per-trial iteration count (syncs)
        iters.append(st["iterations"])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    trial_ms = [tev[k].elapsed_time(tev[k + 1]) for k in range(a.steps)]
    launches = st["kernel_launches"] * a.steps
    ms, arcs = combine_ranks(ms, m * sum(iters), pg, dev)
    value = arcs / (ms / 1e3) / 1e9

    # ---- end to end through the C ABI: every step uploads the graph's CSR from
    #      pinned host memory (gap_graph_create_csc: copy + device check), runs the
    #      trial into pinned host scores, and releases the uploaded graph ----
    host_scores = torch.empty(n, dtype=torch.float32).pin_memory()
    h_off = torch.empty(n + 1, dtype=torch.int64).pin_memory()
    h_idx = torch.empty(m, dtype=torch.int32).pin_memory()
    gap.gap_graph_export_csr(g.handle, 1, h_off, h_idx)
    e_steps = max(1, min(a.steps, 8))
    torch.cuda.synchronize(dev)
    e_iters = []
    t_e0 = time.perf_counter()
    for _ in range(e_steps):
        gu = gap.Graph.from_csc(n, h_off, h_idx)
        gap.gap_pr_run_ex(gu.handle, DAMPING, TOL, MAX_ITERS, opts, host_scores)
        _, st_e = gap.gap_pr_stats(gu.handle)  # the scores are on the host when it returns
        e_iters.append(st_e["iterations"])
        gu.close()
    e_s = time.perf_counter() - t_e0
    e2e = {"value": m * sum(e_iters) / e_s / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": 8 * (n + 1) + 4 * m, "d2h_bytes_per_step": 4 * n, "steps": e_steps,
           "ms_per_step": e_s / e_steps * 1e3,
           "note": "per step, host clock: the in-direction CSR uploaded from pinned host memory "
                   "(gap_graph_create_csc: copy, device structure check, out-degrees), one trial into "
                   "pinned host scores, the uploaded graph released"}
    # the same trials with the graph kept on the device (paper §2.3: only the graph is reused)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r_iters = []
    e0.record(stream)
    for _ in range(a.steps):
        trial(host_scores)
        _, st_r = gap.gap_pr_stats(g.handle)
        r_iters.append(st_r["iterations"])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    e2e["resident_graph"] = {"value": m * sum(r_iters) / (e0.elapsed_time(e1) / 1e3) / 1e9, "unit": UNIT,
                             "d2h_bytes_per_step": 4 * n,
                             "note": "gap_pr_run into pinned host memory, graph resident on the device"}
    del h_off, h_idx
    # The oracle child starts here, not earlier. Its CSR build holds ~40 GB of host
    # memory. While it existed, even stopped, the upload above ran at 208 instead
    # of 139 ms per step. A spawned child does not inherit this process's CUDA
    # state, so starting it after CUDA is initialised is safe.
    oracle_proc = start_oracle_leg(a) if want_oracle else None

    # ---- per-kernel durations (CUDA events around every launch) ----
    prof = options()
    prof.timing = 1
    trial(scores, prof)
    _, sp = gap.gap_pr_stats(g.handle)
    roofline = roofline_entry(sp, m, n, sp["segments"])

    # ---- FP64 GPU path on the same graph (metric: FP32 vs FP64 at L1 <= 1e-4) ----
    gpu_results = {"fp32": (scores.double().cpu().numpy(), iters[-1])}
    fp64 = None
    if not a.no_fp64:
        o64 = options()
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
        gpu_results["fp64"] = (x64.cpu().numpy(), s64["iterations"])
        fp64 = {"value": v64, "unit": UNIT, "fp32_speedup": value / ws / v64 if v64 else None,
                "l1_fp32_vs_fp64": l1, "iterations": s64["iterations"]}

    # ---- BF16-stored contributions (Kahan sums on hub rows), error vs the FP64 GPU path ----
    bf16 = None
    if not a.no_fp64:
        bf16 = {}
        xb = torch.empty(n, dtype=torch.float32, device=dev)
        for label, ladder in (("ladder", -10), ("bf16_only", gap.GAP_NO_LADDER)):
            ob = options()
            ob.contrib = gap.GAP_CONTRIB_BF16
            ob.bf16_until_log2_delta = ladder
            gap.gap_pr_run_ex(g.handle, DAMPING, TOL, MAX_ITERS, ob, xb)
            gap.gap_pr_stats(g.handle)
            kb = max(1, min(3, a.steps))
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            itb = 0
            b0.record(stream)
            for _ in range(kb):
                gap.gap_pr_run_ex(g.handle, DAMPING, TOL, MAX_ITERS, ob, xb)
                _, sb = gap.gap_pr_stats(g.handle)
                itb += sb["iterations"]
            b1.record(stream)
            torch.cuda.synchronize(dev)
            vb = m * itb / (b0.elapsed_time(b1) / 1e3) / 1e9
            gpu_results["bf16_" + label] = (xb.double().cpu().numpy(), sb["iterations"])
            bf16[label] = {"value": vb, "unit": UNIT, "vs_fp32": vb / (value / ws),
                           "l1_vs_fp64": float((x64 - xb.double()).abs().sum().item()),
                           "iterations": sb["iterations"], "bf16_iterations": sb["bf16_iters"],
                           "final_delta": sb["final_delta"]}
        bf16["note"] = ("contributions stored as BF16 with Kahan-compensated sums on rows above 10^4 "
                        "in-arcs; 'ladder' switches to FP32 contributions once delta <= 2^-10")
        del xb

    # ---- residual algorithm (rounds of pulls or frontier pushes) on the same graph ----
    delta = None
    if not a.no_fp64:
        od = options()
        od.algorithm = gap.GAP_ALGO_DELTA
        xd = torch.empty(n, dtype=torch.float32, device=dev)
        gap.gap_pr_run_ex(g.handle, DAMPING, TOL, MAX_ITERS, od, xd)
        gap.gap_pr_stats(g.handle)
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kd = max(1, min(3, a.steps))
        d0.record(stream)
        for _ in range(kd):
            gap.gap_pr_run_ex(g.handle, DAMPING, TOL, MAX_ITERS, od, xd)
            _, sd = gap.gap_pr_stats(g.handle)
        d1.record(stream)
        torch.cuda.synchronize(dev)
        dms = d0.elapsed_time(d1) / kd
        delta = {"ms_per_trial": dms, "vs_pull_trial": (ms / a.steps) / dms, "rounds": sd["iterations"],
                 "sparse_rounds": sd["sparse_rounds"], "arcs_traversed": sd["arcs_traversed"],
                 "pull_arcs_traversed": m * iters[-1], "final_residual": sd["final_delta"],
                 "note": "options.algorithm = GAP_ALGO_DELTA: stops on the exact residual sum |J(x) - x| < tol "
                         "and returns J(x); a round pulls d P r or pushes a frontier's residual"}
        gpu_results["delta"] = (xd.double().cpu().numpy(), None)
        del xd

    cc = bfs = None
    if a.workload == "all":
        cc = measure_cc(g, dev, stream, max(1, a.steps), max(3, a.warmup), a.graph != "urand")
        bfs = measure_bfs(g, dev, stream, gap.bfs_sources(g.export_outdeg(), 64), max(3, a.warmup))
    oracle_err = None
    if oracle_proc is not None:
        oracle_err = error_vs_oracle(*oracle_proc, gpu_results)
    del gpu_results

    g.close()
    del scores, host_scores
    if not a.no_fp64:
        del x64
    torch.cuda.empty_cache()
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**workload_config(a), "n": n, "m": m,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "iterations": iters, "clocks": clk, "e2e": e2e, "gpu_launches": launches,
        "trials_ms": {"all": trial_ms, "min": min(trial_ms),
                      "median": sorted(trial_ms)[len(trial_ms) // 2],
                      "note": "each trial: allocation, binning, iterations to tol, output (paper §2.3); "
                              "the stats read between trials is outside these events"},
        "roofline": roofline, "fp64": fp64, "bf16": bf16, "delta": delta,
    }
    if oracle_err is not None:
        line["error_vs_oracle"] = oracle_err
    if a.workload == "all" and rank == 0:
        line["l2_window"] = measure_l2_window(dev)
    if cc is not None:
        line["cc"] = cc
    if bfs is not None:
        line["bfs"] = bfs
    if not a.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(a)
    return line



def measure_l2_window(dev, steps=8):
    """options.l2_window on the one benchmark-shaped graph where it engages: a
    uniform random digraph of 2^22 vertices (degree 16), whose two FP32
    contribution arrays (32 MB) fit the persisting L2 carve-out and need no L2
    blocking.  Trials with the window off and on, graph loop, median times."""
    import torch

    import gapgen
    from paper_1508_03619_gb300 import gap, tuning
    scale = 22
    src, dst = gapgen.urand_device(1 << scale, 16 << scale, 0x22, device=dev)
    g = gap.Graph.from_edges(1 << scale, src, dst, symmetrize=False)
    del src, dst
    x = torch.empty(g.n, dtype=torch.float32, device=dev)
    out = {"workload": f"urand{scale} directed, degree 16, FP32 pull PageRank to tol 1e-4 (whole rows, "
                       f"no L2 blocking)", "n": g.n, "m": g.m}
    for win in (0, 1):
        o = tuning.pagerank_options()
        o.l2_window = win
        for _ in range(3):
            gap.gap_pr_run_ex(g.handle, DAMPING, TOL, MAX_ITERS, o, x)
            gap.gap_pr_stats(g.handle)
        ms, it = [], 0
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gap.gap_pr_run_ex(g.handle, DAMPING, TOL, MAX_ITERS, o, x)
            e1.record()
            _, st = gap.gap_pr_stats(g.handle)
            ms.append(e0.elapsed_time(e1))
            it = st["iterations"]
        med = sorted(ms)[len(ms) // 2]
        out["on" if win else "off"] = {"ms_per_trial": med, "iterations": it,
                                       "value": g.m * it / (med / 1e3) / 1e9, "unit": UNIT,
                                       "window_bytes": st["l2_window_bytes"]}
    out["speedup"] = out["off"]["ms_per_trial"] / out["on"]["ms_per_trial"]
    g.close()
    del x
    torch.cuda.empty_cache()
    return out


# Bytes per vertex that one CC trial moves at the least (init 4; two sampling
# rounds of offsets 8 + sampled index 4 + two label reads 8 + a hook 4; three
# compress passes of 8; the final pass's offsets 8 + label 4; the count 4);
# a directed graph's pass over the out-direction adds 12.
CC_BYTES_PER_VERTEX = 92
CC_BYTES_PER_VERTEX_OUT_PASS = 12


def measure_cc(g, dev, stream, steps, warmup, symmetric):
    """Connected Components trials on graph g (labels into a device buffer)."""
    import torch

    from paper_1508_03619_gb300 import gap
    lab = torch.empty(g.n, dtype=torch.int32, device=dev)
    for _ in range(max(1, warmup)):  # the first call builds a directed graph's out-direction
        gap.gap_cc_run(g.handle, lab)
    gap.gap_cc_stats(g.handle)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in ev:
        e0.record(stream)
        gap.gap_cc_run(g.handle, lab)
        e1.record(stream)
    torch.cuda.synchronize(dev)
    _, st = gap.gap_cc_stats(g.handle)
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    med = sorted(ms)[len(ms) // 2]
    per_v = CC_BYTES_PER_VERTEX + (0 if symmetric else CC_BYTES_PER_VERTEX_OUT_PASS)
    peak, kind = measured_hbm_peak()
    achieved = per_v * g.n / (med / 1e3) / 1e9
    del lab
    return {"value": g.m / (med / 1e3) / 1e9, "unit": "Gedges/s (stored arcs / trial time)",
            "ms_per_trial": {"all": ms, "min": min(ms), "median": med},
            "components": st["components"], "giant_size": st["giant_size"],
            "gpu_launches_per_trial": st["kernel_launches"],
            "bandwidth": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                          "frac": achieved / peak, "bytes_per_vertex": per_v,
                          "peak_source": f"{kind} hbm_gbs",
                          "note": "bytes a trial moves at the least over its median time; the giant "
                                  "component's remaining arcs are skipped by the method"}}


def measure_bfs(g, dev, stream, sources, warmup):
    """BFS trials on graph g, one per source (parents into a device buffer)."""
    import torch

    from paper_1508_03619_gb300 import gap
    par = torch.empty(g.n, dtype=torch.int32, device=dev)
    for s in sources[:max(1, warmup)]:  # the first call builds a directed graph's out-direction
        gap.gap_bfs_run(g.handle, s, par)
    gap.gap_bfs_stats(g.handle)
    ms, reached, levels, td, bu, launches = [], [], [], [], [], 0
    for s in sources:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gap.gap_bfs_run(g.handle, s, par)
        e1.record(stream)
        st = gap.gap_bfs_stats(g.handle)  # synchronizes; outside the events
        ms.append(e0.elapsed_time(e1))
        reached.append(st["reached"])
        levels.append(st["levels"])
        td.append(st["top_down_steps"])
        bu.append(st["bottom_up_steps"])
        launches += st["kernel_launches"]
    del par
    med = sorted(ms)[len(ms) // 2]
    return {"value": g.m / (med / 1e3) / 1e9, "unit": "Gedges/s (stored arcs / median trial time)",
            "trials": len(sources), "sources": "splitmix64 draws of vertices with out-arcs, seed 0x5EED",
            "ms_per_trial": {"all": ms, "min": min(ms), "median": med},
            "reached": {"min": min(reached), "max": max(reached)},
            "levels": {"min": min(levels), "max": max(levels)},
            "steps": {"top_down_mean": sum(td) / len(td), "bottom_up_mean": sum(bu) / len(bu)},
            "gpu_launches_per_trial": launches / len(sources),
            "note": "each trial ends when the host has seen the last step's counters; the host reads "
                    "two counters per step to choose the direction"}


def batch_tuning():
    """The per-GPU tuning table entry for this device (autotuned), else None
    (the library's built-in values)."""
    from paper_1508_03619_gb300 import tuning
    return tuning.batch_tuning_for_device()


def measure_batch(a, dev, steps, warmup):
    """PageRank on the uneven 256-graph batch in one persistent launch per
    step (tol 1e-4, each graph stops on its own).  The batch's CSCs (about
    1 GB of indices) exceed L2, so no flush between steps."""
    import numpy as np
    import torch

    import gapgen
    from paper_1508_03619_gb300 import gap

    specs = gapgen.batch_specs()
    graphs = [gap.Graph.from_edges(s.n, *s.edges(), symmetrize=True) for s in specs]
    ns = np.array([g.n for g in graphs], np.int64)
    ms = np.array([g.m for g in graphs], np.int64)
    xs = [torch.empty(g.n, dtype=torch.float32, device=dev) for g in graphs]
    hs = graphs  # Graph objects: the binding knows each n without a library call
    tu = batch_tuning()
    for _ in range(warmup):
        st = gap.gap_pr_run_batch(hs, xs, DAMPING, TOL, MAX_ITERS, tuning=tu)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        gap.gap_pr_run_batch(hs, xs, DAMPING, TOL, MAX_ITERS, stats=False, tuning=tu)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_step = e0.elapsed_time(e1) / steps
    # iteration counts (the same in every call) and device phase times, untimed
    loop_ms = []
    for _ in range(3):
        st = gap.gap_pr_run_batch(hs, xs, DAMPING, TOL, MAX_ITERS, tuning=tu)
        loop_ms.append(st[0]["phase_ms"]["pull0"])
    its = np.array([t["iterations"] for t in st], np.int64)
    arcs = float((its * ms).sum())
    # algorithmic bytes: 8 per arc (index + gathered contribution), 24 per row
    # per iteration (offsets, out-degree, x read and write, contribution write)
    alg = float((its * (8 * ms + 24 * ns)).sum())
    kern_ms = float(np.median(loop_ms))
    peak, kind = measured_hbm_peak()
    achieved = alg / (kern_ms / 1e3) / 1e9
    out = {
        "workload": "batch of 256 graphs: 128 R-MAT (2^10..2^18 vertices, edge factor 8..32, symmetrized) "
                    "+ 128 grids (2^10..2^18 vertices, 5% edge deletions), FP32, d=0.85, tol=1e-4 per graph",
        "graphs": len(graphs), "n_total": int(ns.sum()), "m_total": int(ms.sum()),
        "iterations": {"min": int(its.min()), "max": int(its.max()), "mean": float(its.mean())},
        "value": arcs / (ms_step / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms_step, "steps": steps,
        "gpu_launches_per_step": st[0]["kernel_launches"],
        "tuning": tu if tu is not None else gap.gap_batch_tuning_default().to_dict(),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": BATCH_NCU_TRAFFIC if tu == BATCH_NCU_TUNING else None,
                     "kernel": "k_batch_persistent (all iterations of all graphs, one launch)",
                     "alg_bytes_per_launch": alg, "launch_ms": kern_ms,
                     "peak_source": f"{kind} hbm_gbs"},
        "phase_ms": {k: st[0]["phase_ms"][k] for k in ("prep", "pull0", "output")},
        "l2": "inputs larger than L2 (1+ GB of CSC per batch), no flush",
    }
    # the same graphs one trial at a time through gap_pr_run
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for g_, x in zip(graphs, xs):
        gap.gap_pr_run(g_.handle, DAMPING, TOL, MAX_ITERS, x)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    seq_ms = e0.elapsed_time(e1)
    out["one_graph_at_a_time"] = {"ms": seq_ms, "value": arcs / (seq_ms / 1e3) / 1e9,
                                  "batch_speedup": seq_ms / ms_step}
    for g in graphs:
        g.close()
    del xs
    torch.cuda.empty_cache()
    return out


def measure_ppr(a, dev):
    """Personalized-PageRank serving: a continuous-batching server over a
    resident Chung-Lu graph.  Saturated throughput (a burst of queries), then
    Poisson arrivals at 0.25/0.5/0.9 of it for --ppr-seconds each; latency is
    completion minus scheduled arrival.  One-at-a-time: gap_ppr_batch with one
    query per call."""
    import numpy as np
    import torch

    import gapgen
    from paper_1508_03619_gb300 import gap

    n = 1 << a.ppr_scale
    m_draw = int(a.ppr_edges)
    src, dst = gapgen.chung_lu_device(n, m_draw, 2.1, 0x5C, device=dev)
    g = gap.Graph.from_edges(n, src, dst, symmetrize=False)
    del src, dst
    torch.cuda.empty_cache()
    outdeg = g.export_outdeg()
    cand = np.flatnonzero(outdeg > 0)
    rng = np.random.default_rng(0x5E)

    def draw():
        return rng.choice(cand, size=int(rng.integers(1, 65))).astype(np.int32)

    res = {"workload": f"PPR serving on Chung-Lu n=2^{a.ppr_scale}, {m_draw:.3g} arc draws, exponent 2.1, "
                       f"directed; queries of 1..64 seeds; FP32; d=0.85, tol=1e-4 per query",
           "n": g.n, "m": g.m}
    # one query at a time (one column per call)
    one = torch.empty(n, dtype=torch.float32, device=dev)
    gap.gap_ppr_batch(g.handle, np.array([0, 3], np.int64), draw()[:3], DAMPING, TOL, MAX_ITERS, one)
    t0 = time.perf_counter()
    k1 = 3
    its1 = []
    for _ in range(k1):
        q = draw()
        st = gap.gap_ppr_batch(g.handle, np.array([0, len(q)], np.int64), q, DAMPING, TOL, MAX_ITERS, one)
        its1.append(st[0]["iterations"])
    res["one_at_a_time_qps"] = k1 / (time.perf_counter() - t0)
    res["one_at_a_time_iterations"] = its1
    del one

    srv = gap.PprServer(g.handle, max_cols=a.ppr_cols, hbm_reserve=16 << 30, damping=DAMPING, tol=TOL,
                        max_iters=MAX_ITERS)
    cols = srv.info()["columns"]
    ring = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(3 * cols)]
    owner = [None] * len(ring)
    res["columns"] = cols

    def run_arrivals(times):
        """Submit at the scheduled times; returns (latencies_ms, makespan_s, iterations)."""
        lat, iters = [], []
        pending = []
        start = time.perf_counter()
        for j, ts in enumerate(times):
            slot = j % len(ring)
            if owner[slot] is not None:  # reuse a buffer only after its query finished
                tk, t_sched, t_sub = owner[slot]
                info = srv.wait(tk)
                lat.append((t_sub - t_sched) * 1e3 + info["latency_ms"])
                iters.append(info["iterations"])
                pending.remove(slot)
            now = time.perf_counter() - start
            if ts > now:
                time.sleep(ts - now)
            t_sub = time.perf_counter() - start
            owner[slot] = (srv.submit(draw(), ring[slot]), ts, t_sub)
            pending.append(slot)
        for slot in list(pending):
            tk, t_sched, t_sub = owner[slot]
            info = srv.wait(tk)
            lat.append((t_sub - t_sched) * 1e3 + info["latency_ms"])
            iters.append(info["iterations"])
        for slot in range(len(owner)):
            owner[slot] = None
        return np.array(lat), time.perf_counter() - start, iters

    run_arrivals([0.0] * cols)  # warm-up burst
    burst = 2 * cols
    steps0 = srv.info()["steps"]
    lat, span, iters = run_arrivals([0.0] * burst)
    steps = srv.info()["steps"] - steps0
    sat = burst / span
    # roofline of the SpMM iterations of the burst: per iteration 4 B index + 4·cols B
    # of gathered contribution row per arc, (8 + 4 + 12·cols) B per row
    step_ms = span * 1e3 / max(steps, 1)
    alg = (4 + 4 * cols) * g.m + (12 + 12 * cols) * g.n
    peak, kind = measured_hbm_peak()
    res["roofline"] = {"bound": "hbm", "achieved": alg / (step_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                       "frac": alg / (step_ms / 1e3) / 1e9 / peak, "traffic": None,
                       "kernel": f"k_ppr_spmm<{cols // 4}> (+ finalize), one engine iteration",
                       "alg_bytes_per_iteration": alg, "iteration_ms": step_ms, "iterations": steps,
                       "peak_source": f"{kind} hbm_gbs",
                       "note": "iteration time = burst span / engine iterations (admission and copies included)"}
    res["saturated_qps"] = sat
    res["saturated_iterations_mean"] = float(np.mean(iters))
    loads = []
    for f in (0.25, 0.5, 0.9):
        lam = f * sat
        gaps = rng.exponential(1.0 / lam, size=int(lam * a.ppr_seconds * 1.5) + 8)
        times = np.cumsum(gaps)
        times = times[times < a.ppr_seconds].tolist()
        lat, span, _ = run_arrivals(times)
        loads.append({"load": f, "arrival_qps": lam, "queries": len(times),
                      "served_qps": len(times) / span if span > 0 else None,
                      "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))})
    res["poisson"] = loads
    res["batching_gain"] = sat / res["one_at_a_time_qps"]
    res["server"] = srv.info()  # engine widths and how often the server changed width
    srv.close()
    g.close()
    del ring
    torch.cuda.empty_cache()
    return res


def main():
    a = parse()
    ws, rank, local = dist_env()
    if a.impl == "reference":
        run_reference(a, ws, rank)
        return

    want_oracle = (a.workload in ("all", "pagerank") and ws == 1 and rank == 0 and not a.no_oracle_check
                   and not a.no_fp64)

    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    line = None
    if a.workload in ("all", "pagerank"):
        line = run_pagerank(a, ws, rank, local, dev, pg, want_oracle)
        if line is not None and a.workload == "all" and ws == 1:
            line["batch"] = measure_batch(a, dev, max(1, a.steps), max(3, a.warmup))
            line["ppr"] = measure_ppr(a, dev)
    elif rank == 0:
        if a.workload == "batch":
            b = measure_batch(a, dev, max(1, a.steps), max(1, a.warmup))
            line = {"metric": METRIC, "value": b.pop("value"), "unit": UNIT, "n_gpus": 1,
                    "steps": b["steps"], "warmup": a.warmup, "ms_per_step": b.pop("ms_per_step"),
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                    "data": "synthetic", "config": {"workload": b.pop("workload")},
                    "roofline": b.pop("roofline"), "batch": b}
        elif a.workload in ("cc", "bfs"):
            import gapgen
            from paper_1508_03619_gb300 import gap
            if a.graph == "urand":
                src, dst = gapgen.urand_device(1 << a.scale, a.edge_factor << a.scale, a.seed, device=dev)
            else:
                src, dst = gapgen.kron_device(a.scale, a.edge_factor, a.seed, device=dev)
            g = gap.Graph.from_edges(1 << a.scale, src, dst, symmetrize=a.graph != "urand")
            del src, dst
            torch.cuda.empty_cache()
            stream = torch.cuda.current_stream(dev)
            if a.workload == "cc":
                r = measure_cc(g, dev, stream, max(1, a.steps), max(1, a.warmup), a.graph != "urand")
            else:
                r = measure_bfs(g, dev, stream, gap.bfs_sources(g.export_outdeg(), max(1, a.steps)),
                                max(1, a.warmup))
            cfg = workload_config(a)
            g.close()
            line = {"metric": METRIC, "value": r.pop("value"), "unit": r.pop("unit"), "n_gpus": 1,
                    "steps": a.steps, "warmup": a.warmup, "higher_is_better": True, "scaling": "weak",
                    "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                    "config": {**cfg, "workload": cfg["workload"].split(" pull")[0]
                               + (" connected components" if a.workload == "cc"
                                  else f" BFS from {max(1, a.steps)} sources"), "kernel": a.workload},
                    a.workload: r}
        else:
            p = measure_ppr(a, dev)
            line = {"metric": METRIC, "value": p["saturated_qps"], "unit": "queries/s", "n_gpus": 1,
                    "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                    "data": "synthetic", "config": {"workload": p.pop("workload")}, "ppr": p}
    if line is not None:
        print(json.dumps(line))
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
