"""Batch of uneven graphs in one persistent launch vs the FP64 oracle, graph
by graph, plus independence: a graph's result is bit-identical alone and in any
batch, and a graph that stopped stays as it stopped."""
import numpy as np
import pytest

import gapgen
import oracle
from gpu_helpers import D, FP32_L1, FP32_REL, exact_l1_change, exact_sum, gpu_graph, oracle_graph
from paper_1508_03619_gb300 import gap

pytestmark = pytest.mark.gpu


def make_batch(specs, extra=()):
    """Host edge lists for the specs (both kinds undirected), plus extra
    (n, src, dst, symmetrize) members."""
    members = [(s.n, *s.edges(), True) for s in specs]
    members.extend(extra)
    return members


def run_batch(graphs, tol, iters):
    import torch
    xs = [torch.empty(g.n, dtype=torch.float32, device="cuda:0") for g in graphs]
    st = gap.gap_pr_run_batch([g.handle for g in graphs], xs, D, tol, iters)
    return [x.cpu().numpy().astype(np.float64) for x in xs], st


def edge_members():
    """Degenerate members: one vertex, no arcs at all, a directed graph with
    dangling vertices, a star."""
    rs = np.random.default_rng(5)
    n3 = 300
    src3, dst3 = gapgen.urand(n3, 600, 0x61)
    star_n = 40
    ssrc = np.zeros(star_n - 1, np.int32)
    sdst = np.arange(1, star_n, dtype=np.int32)
    return [
        (1, np.zeros(0, np.int32), np.zeros(0, np.int32), False),
        (7, np.zeros(0, np.int32), np.zeros(0, np.int32), False),
        (n3, src3, dst3, False),
        (star_n, ssrc, sdst, True),
        (33, rs.integers(0, 33, 90).astype(np.int32), rs.integers(0, 33, 90).astype(np.int32), False),
    ]


def check_member(x, st, n, src, dst, sym, tol, iters, csr=None):
    """One batch member against the oracle.  Fixed iterations: the FP32 bars
    element by element.  Tolerance mode: converged within one iteration of the
    oracle, the paper's §3 verifier (< 1e-4) on the scores, and the FP32 bars
    against the oracle run for the member's own iteration count."""
    off, idx = csr if csr is not None else oracle_graph(n, src, dst, sym)
    if tol == 0.0:
        assert st["iterations"] == iters
        xo, _, _ = oracle.pagerank(off, idx, D, 0.0, iters)
    else:
        _, ko, _ = oracle.pagerank(off, idx, D, tol, iters)
        assert st["converged"] == 1
        assert abs(st["iterations"] - ko) <= 1, (st["iterations"], ko)
        assert oracle.verify(off, idx, x, D) < 1e-4
        xo, _, _ = oracle.pagerank(off, idx, D, 0.0, st["iterations"])
    assert np.abs(x - xo).sum() <= FP32_L1
    assert np.max(np.abs(x - xo) / xo, initial=0.0) <= FP32_REL
    assert abs(st["mass"] - x.sum()) <= 1e-6 * max(1.0, x.sum())
    assert (x >= 0).all()


def test_small_uneven_batch_matches_oracle(cuda_device):
    specs = gapgen.batch_specs(count=12, seed=0x71, min_exp=5, max_exp=12)
    members = make_batch(specs, edge_members())
    graphs = [gpu_graph(n, s, d, sym) for (n, s, d, sym) in members]
    try:
        xs, st = run_batch(graphs, 0.0, 20)
        for (n, s, d, sym), x, t in zip(members, xs, st):
            check_member(x, t, n, s, d, sym, 0.0, 20)
        xs, st = run_batch(graphs, 1e-4, 100)
        for (n, s, d, sym), x, t in zip(members, xs, st):
            check_member(x, t, n, s, d, sym, 1e-4, 100)
        # graphs stop at different iterations
        assert len({t["iterations"] for t in st}) > 1
    finally:
        for g in graphs:
            g.close()


def test_batch_member_alone_equals_mixed(cuda_device):
    specs = gapgen.batch_specs(count=10, seed=0x72, min_exp=8, max_exp=13)
    members = make_batch(specs)
    graphs = [gpu_graph(n, s, d, sym) for (n, s, d, sym) in members]
    try:
        xm, stm = run_batch(graphs, 1e-4, 100)
        for j in (0, 4, 9):
            xa, sta = run_batch([graphs[j]], 1e-4, 100)
            assert sta[0]["iterations"] == stm[j]["iterations"]
            assert sta[0]["final_delta"] == stm[j]["final_delta"]
            assert np.array_equal(xa[0], xm[j])
        perm = [3, 9, 0, 7, 1]
        xp, stp = run_batch([graphs[p] for p in perm], 1e-4, 100)
        for newj, oldj in enumerate(perm):
            assert np.array_equal(xp[newj], xm[oldj])
        # the batch agrees with the single-graph entry point within the FP32 bar
        import torch
        x1 = torch.empty(graphs[2].n, dtype=torch.float32, device="cuda:0")
        gap.gap_pr_run(graphs[2].handle, D, 0.0, stm[2]["iterations"], x1)
        assert np.abs(x1.cpu().numpy().astype(np.float64) - xm[2]).sum() <= FP32_L1
    finally:
        for g in graphs:
            g.close()


def test_full_batch_256(cuda_device):
    """The 256-graph uneven batch (128 R-MAT + 128 grids, 2^10..2^18
    vertices), every member against the oracle: 20 fixed iterations element by
    element (FP32 bars), and tolerance mode (iterations within one of the
    oracle's, the §3 verifier, scores at the member's own iteration count)."""
    specs = gapgen.batch_specs()
    members = make_batch(specs)
    graphs = [gpu_graph(n, s, d, sym) for (n, s, d, sym) in members]
    try:
        csrs = [oracle_graph(n, s, d, sym) for (n, s, d, sym) in members]
        xs, st = run_batch(graphs, 0.0, 20)
        for (n, s, d, sym), x, t, csr in zip(members, xs, st, csrs):
            check_member(x, t, n, s, d, sym, 0.0, 20, csr)
        xs, st = run_batch(graphs, 1e-4, 100)
        for (n, s, d, sym), x, t, csr in zip(members, xs, st, csrs):
            assert t["final_delta"] < 1e-4
            assert 0.0 < t["mass"] <= 1.0 + 1e-4
            check_member(x, t, n, s, d, sym, 1e-4, 100, csr)
        assert len({t["iterations"] for t in st}) > 1
    finally:
        for g in graphs:
            g.close()


def test_batch_edge_arguments(cuda_device):
    import torch
    n = 64
    src, dst = gapgen.urand(n, 256, 0x73)
    g = gpu_graph(n, src, dst)
    try:
        assert gap.gap_pr_run_batch([], [], D, 1e-4, 10) == []
        x = torch.full((n,), -1.0, dtype=torch.float32, device="cuda:0")
        st = gap.gap_pr_run_batch([g.handle], [x], D, 1e-4, 0)
        assert st[0]["iterations"] == 0
        assert torch.allclose(x, torch.full_like(x, 1.0 / n))
        with pytest.raises(gap.GapError) as e:
            gap.gap_pr_run_batch([g.handle], [x], 1.5, 1e-4, 10)
        assert e.value.status == gap.GAP_ERR_INVALID_ARG
        with pytest.raises(gap.GapError):
            gap.gap_pr_run_batch([g.handle], [torch.empty(n, dtype=torch.float32).pin_memory()], D,
                                 1e-4, 10)
        with pytest.raises(ValueError):
            gap.gap_pr_run_batch([g.handle], [torch.empty(n - 1, dtype=torch.float32,
                                                          device="cuda:0")], D, 1e-4, 10)
    finally:
        g.close()


def test_batch_tunings(cuda_device):
    """Launch shape changes nothing (bit-identical); the heavy-row split only
    reorders sums (FP32 bar vs the oracle).  A star with a hub of in-degree
    3000 exercises rows of many chunks."""
    hub_n = 3001
    hsrc = np.arange(1, hub_n, dtype=np.int32)
    hdst = np.zeros(hub_n - 1, np.int32)
    specs = gapgen.batch_specs(count=6, seed=0x74, min_exp=9, max_exp=13)
    members = make_batch(specs, [(hub_n, hsrc, hdst, True)])
    graphs = [gpu_graph(n, s, d, sym) for (n, s, d, sym) in members]
    try:
        ref, st_ref = run_batch(graphs, 0.0, 15)
        import torch
        for tu in ({"block_threads": 128}, {"block_threads": 512}, {"blocks_per_sm": 1}):
            xs = [torch.empty(g.n, dtype=torch.float32, device="cuda:0") for g in graphs]
            st = gap.gap_pr_run_batch([g.handle for g in graphs], xs, D, 0.0, 15, tuning=tu)
            for a, b, sa, sb in zip(xs, ref, st, st_ref):
                assert np.array_equal(a.cpu().numpy().astype(np.float64), b)
                assert sa["final_delta"] == sb["final_delta"]
        for tu in ({"heavy_min_degree": 32, "chunk_arcs": 32}, {"heavy_min_degree": 100000},
                   {"heavy_min_degree": 64, "chunk_arcs": 1000}):
            xs = [torch.empty(g.n, dtype=torch.float32, device="cuda:0") for g in graphs]
            st = gap.gap_pr_run_batch([g.handle for g in graphs], xs, D, 0.0, 15, tuning=tu)
            for (n, s, d, sym), x, t in zip(members, xs, st):
                check_member(x.cpu().numpy().astype(np.float64), t, n, s, d, sym, 0.0, 15)
        for bad in ({"heavy_min_degree": 8}, {"chunk_arcs": 0}, {"block_threads": 96},
                    {"blocks_per_sm": -1}):
            with pytest.raises(gap.GapError) as e:
                gap.gap_pr_run_batch([graphs[0].handle], [torch.empty(graphs[0].n, device="cuda:0")],
                                     D, 0.0, 5, tuning=bad)
            assert e.value.status == gap.GAP_ERR_INVALID_ARG
    finally:
        for g in graphs:
            g.close()


def test_batch_delta_is_the_exact_l1_change(cuda_device):
    """Each graph's delta of iteration k is sum |x_k - x_(k-1)| taken exactly
    (fixed point in units of 2^-60, integer sums), for members of every kind."""
    members = make_batch(gapgen.batch_specs(count=8, min_exp=10, max_exp=12), edge_members())
    graphs = [gpu_graph(n, s, d, sym) for n, s, d, sym in members]
    try:
        prev = [np.full(g.n, np.float32(1.0 / g.n), np.float64) for g in graphs]
        for k in (1, 2):
            xs, st = run_batch(graphs, 0.0, k)
            for i, g in enumerate(graphs):
                assert st[i]["iterations"] == k
                assert st[i]["deltas"][k - 1] == exact_l1_change(xs[i], prev[i]), (i, k)
                assert st[i]["mass"] == exact_sum(xs[i])
            prev = xs
    finally:
        for g in graphs:
            g.close()
