"""Autotuner: pick the launch and split parameters of this GPU model once, on a
tuning set of synthetic graphs disjoint from the evaluation graphs, and write
the fixed table that ``tuning.py`` loads.

Tuned here:
  batch path    heavy_min_degree (rows above it are split into chunk tasks),
                chunk_arcs, block_threads (CTA shape), blocks_per_sm;
  single graph  segment_bytes (L2 blocking of the contribution array), the
                degree-bin bounds (small_max_degree: bin 0, the vertex-order
                kernel; group_max_degree: bin 4; cta_max_degree: bin 5, above
                it hubs), the lanes per row of bin 4 and the hub chunk size.
Tuning set: the uneven batch generator with its own seed (not the evaluation
batch's), and Kronecker / uniform-random graphs at scale 26 (the benchmark's
size) with their own seeds.  Each candidate is timed with CUDA events (median of several trials,
inputs larger than L2).  Greedy coordinate search: one parameter at a time,
starting from the built-in values, two passes.

Usage: python -m paper_1508_03619_gb300.autotune [--out FILE] [--quick]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

D = 0.85
TOL = 1e-4
TUNE_BATCH_SEED = 0xA7  # the evaluation batch uses gapgen.batch_specs' default seed
TUNE_GRAPH_SEEDS = {"kron": 0xA24, "urand": 0xA25}  # the evaluation graphs use 0x26

BATCH_SPACE = {
    "heavy_min_degree": [64, 128, 256, 512, 1024],
    "chunk_arcs": [512, 1024, 2048, 4096, 8192],
    "block_threads": [128, 256, 512],
    "blocks_per_sm": [0, 2, 4],
}
PAGERANK_SPACE = {  # 0: the library's built-in value
    "segment_bytes": [0, 8 << 20, 16 << 20, 64 << 20, -1],  # -1: never segment
    "small_max_degree": [0, 32, 64, 128, 255],
    "group_max_degree": [0, 256, 1024, 2048, 4096],
    "cta_max_degree": [0, 8192, 16384, 65536],
    "hub_chunk_arcs": [0, 2048, 8192, 32768],
    "group_lanes": [0, 8, 32],
}


def _timer(torch):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ts.sort()
        return ts[len(ts) // 2]
    return timed


def coordinate_search(space, start, cost, passes=2, log=print):
    """Greedy search: for each parameter in turn, keep the value of least
    cost with the others fixed."""
    best = dict(start)
    best_cost = cost(best)
    for _ in range(passes):
        changed = False
        for k, values in space.items():
            for v in values:
                if v == best[k]:
                    continue
                cand = dict(best, **{k: v})
                c = cost(cand)
                log(f"  {cand} -> {c:.3f} ms")
                if c < best_cost * 0.995:
                    best, best_cost, changed = cand, c, True
        if not changed:
            break
    return best, best_cost


def tune_batch(gap, gapgen, torch, reps, log):
    specs = gapgen.batch_specs(seed=TUNE_BATCH_SEED)
    graphs = [gap.Graph.from_edges(s.n, *s.edges(), symmetrize=True) for s in specs]
    xs = [torch.empty(g.n, dtype=torch.float32, device="cuda") for g in graphs]
    hs = [g.handle for g in graphs]
    timed = _timer(torch)

    def cost(tu):
        gap.gap_pr_run_batch(hs, xs, D, TOL, 100, stats=False, tuning=tu)
        return timed(lambda: gap.gap_pr_run_batch(hs, xs, D, TOL, 100, stats=False, tuning=tu), reps)

    start = gap.gap_batch_tuning_default().to_dict()
    base = cost(start)
    best, c = coordinate_search(BATCH_SPACE, start, cost, log=log)
    for g in graphs:
        g.close()
    return best, {"batch_ms_builtin": base, "batch_ms_tuned": c}


def tune_pagerank(gap, gapgen, torch, reps, scale, log):
    n = 1 << scale
    gs = []
    src, dst = gapgen.kron_device(scale, 16, TUNE_GRAPH_SEEDS["kron"])
    gs.append(gap.Graph.from_edges(n, src, dst, symmetrize=True))
    src, dst = gapgen.urand_device(n, 16 * n, TUNE_GRAPH_SEEDS["urand"])
    gs.append(gap.Graph.from_edges(n, src, dst, symmetrize=False))
    del src, dst
    torch.cuda.empty_cache()
    x = torch.empty(n, dtype=torch.float32, device="cuda")
    timed = _timer(torch)

    def cost(p):
        o = gap.gap_pr_options_default()
        for k, v in p.items():
            setattr(o, k, v)
        total = 0.0
        for g in gs:
            def run():
                gap.gap_pr_run_ex(g.handle, D, 0.0, 20, o, x)
                gap.gap_pr_stats(g.handle)
            run()
            total += timed(run, reps)
        return total

    start = {k: 0 for k in PAGERANK_SPACE}
    base = cost(start)
    best, c = coordinate_search(PAGERANK_SPACE, start, cost, log=log)
    for g in gs:
        g.close()
    return best, {"pagerank_ms_builtin": base, "pagerank_ms_tuned": c}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None, help="table file (default tuning/<device>.json)")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--scale", type=int, default=26)
    ap.add_argument("--skip", default="", help="comma list: batch,pagerank")
    a = ap.parse_args(argv)
    import torch

    import gapgen
    from . import gap
    from .tuning import TABLE_DIR, device_key

    name, sms = device_key()
    log = lambda s: print(s, file=sys.stderr, flush=True)  # noqa: E731
    table = {"device": name, "sms": sms,
             "tuning_set": (f"batch_specs(seed={TUNE_BATCH_SEED:#x}) for the batch path; "
                            f"kron{a.scale} (seed {TUNE_GRAPH_SEEDS['kron']:#x}, ef 16, symmetrized) and "
                            f"urand{a.scale} (seed {TUNE_GRAPH_SEEDS['urand']:#x}, degree 16) for the "
                            f"single-graph path, 20 fixed iterations"),
             "method": "greedy coordinate search, 2 passes, median of CUDA-event timings",
             "date": time.strftime("%Y-%m-%d"), "measured": {}}
    skip = set(filter(None, a.skip.split(",")))
    if "batch" not in skip:
        log("batch path:")
        table["batch"], m = tune_batch(gap, gapgen, torch, a.reps, log)
        table["measured"].update(m)
    if "pagerank" not in skip:
        log("single-graph path:")
        table["pagerank"], m = tune_pagerank(gap, gapgen, torch, a.reps, a.scale, log)
        table["measured"].update(m)
    out = a.out or os.path.join(TABLE_DIR, name.replace(" ", "_").lower() + ".json")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    with open(out, "w") as f:
        json.dump(table, f, indent=1)
    print(json.dumps(table))


if __name__ == "__main__":
    main()
