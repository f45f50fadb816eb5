"""Personalized PageRank (multi-column SpMM) vs the FP64 oracle, and the
column-independence property: a query's result is bit-identical alone and in
any mix of other queries (and whatever slot it occupies)."""
import numpy as np
import pytest

import gapgen
import oracle
from gpu_helpers import D, FP32_L1, gpu_graph, oracle_graph
from paper_1508_03619_gb300 import gap

pytestmark = pytest.mark.gpu


def make_queries(rng, n, q, outdeg, max_seeds=64):
    """Seeds drawn from vertices with out-edges (as a serving workload would)."""
    cand = np.flatnonzero(outdeg > 0)
    offs = [0]
    seeds = []
    for _ in range(q):
        k = int(rng.integers(1, max_seeds + 1))
        seeds.extend(rng.choice(cand, size=k).tolist())
        offs.append(len(seeds))
    return np.array(offs, np.int64), np.array(seeds, np.int32)


def run_ppr(g, offs, seeds, tol, iters):
    import torch
    q = len(offs) - 1
    out = torch.empty(q * g.n, dtype=torch.float32, device="cuda:0")
    st = gap.gap_ppr_batch(g.handle, offs, seeds, D, tol, iters, out)
    return out.cpu().numpy().reshape(q, g.n).astype(np.float64), st


def _hub_graph():
    """A hub with 3000 in-arcs (12 chunks of 256) plus a sparse random part."""
    n = 3001
    rs = np.random.default_rng(7)
    src = np.concatenate([np.arange(1, n), rs.integers(0, n, 6000)]).astype(np.int32)
    dst = np.concatenate([np.zeros(n - 1, np.int64), rs.integers(0, n, 6000)]).astype(np.int32)
    return src, dst


CASES = [
    ("kron13", 1 << 13, *gapgen.kron(13, 16, 0x51), True),
    ("chunglu", 1 << 13, *gapgen.chung_lu(1 << 13, 16 << 13, 2.1, 0x52), False),
    ("hub", 3001, *_hub_graph(), False),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_ppr_matches_oracle(cuda_device, case):
    name, n, src, dst, sym = case
    off, idx = oracle_graph(n, src, dst, sym)
    outdeg = np.diff(off)
    rng = np.random.default_rng(1)
    offs, seeds = make_queries(rng, n, 9, outdeg)
    g = gpu_graph(n, src, dst, sym)
    try:
        x, st = run_ppr(g, offs, seeds, 0.0, 20)
        for j in range(len(offs) - 1):
            s = seeds[offs[j]:offs[j + 1]]
            xo, ko, _ = oracle.ppr(off, idx, s, D, 0.0, 20)
            assert st[j]["iterations"] == 20
            l1 = np.abs(x[j] - xo).sum()
            big = xo > 1e-6
            rel = np.max(np.abs(x[j][big] - xo[big]) / xo[big])
            assert l1 <= FP32_L1 and rel <= 1e-3, (j, l1, rel)
        xt, stt = run_ppr(g, offs, seeds, 1e-4, 100)
        for j in range(len(offs) - 1):
            s = seeds[offs[j]:offs[j + 1]]
            xo, ko, _ = oracle.ppr(off, idx, s, D, 1e-4, 100)
            assert stt[j]["converged"]
            assert abs(stt[j]["iterations"] - ko) <= 1
    finally:
        g.close()


def test_ppr_alone_equals_mixed(cuda_device):
    name, n, src, dst, sym = CASES[0]
    off, idx = oracle_graph(n, src, dst, sym)
    rng = np.random.default_rng(2)
    offs, seeds = make_queries(rng, n, 37, np.diff(off))
    g = gpu_graph(n, src, dst, sym)
    try:
        xm, stm = run_ppr(g, offs, seeds, 1e-4, 100)  # 37 columns -> width 64
        for j in (0, 5, 36):
            one = np.array([0, offs[j + 1] - offs[j]], np.int64)
            xa, sta = run_ppr(g, one, seeds[offs[j]:offs[j + 1]], 1e-4, 100)  # width 4
            assert sta[0]["iterations"] == stm[j]["iterations"]
            assert np.array_equal(xa[0], xm[j])
        # the same query in another slot of another mix
        perm = rng.permutation(37)
        offs2 = np.concatenate([[0], np.cumsum([offs[p + 1] - offs[p] for p in perm])]).astype(np.int64)
        seeds2 = np.concatenate([seeds[offs[p]:offs[p + 1]] for p in perm]).astype(np.int32)
        xp, stp = run_ppr(g, offs2, seeds2, 1e-4, 100)
        for newj, oldj in enumerate(perm):
            assert np.array_equal(xp[newj], xm[oldj])
            assert stp[newj]["iterations"] == stm[oldj]["iterations"]
    finally:
        g.close()


def test_ppr_chunks_and_edge_cases(cuda_device):
    n = 2000
    src, dst = gapgen.urand(n, 12000, 0x53)
    off, idx = oracle_graph(n, src, dst, False)
    outdeg = np.diff(off)
    g = gpu_graph(n, src, dst, False)
    try:
        rng = np.random.default_rng(3)
        offs, seeds = make_queries(rng, n, 130, outdeg, max_seeds=3)  # 2 chunks of <= 128
        dangling = int(np.flatnonzero(outdeg == 0)[0]) if (outdeg == 0).any() else 0
        # query 0: repeated seeds; query 1: a dangling seed
        seeds[offs[0]:offs[1]] = seeds[offs[0]]
        seeds[offs[1]] = dangling
        x, st = run_ppr(g, offs, seeds, 0.0, 15)
        for j in (0, 1, 129):
            xo, _, _ = oracle.ppr(off, idx, seeds[offs[j]:offs[j + 1]], D, 0.0, 15)
            assert np.abs(x[j] - xo).sum() <= FP32_L1
        # all vertices as seeds is plain PageRank
        allv = np.array([0, n], np.int64)
        xa, _ = run_ppr(g, allv, np.arange(n, dtype=np.int32), 0.0, 15)
        xpr, _, _ = oracle.pagerank(off, idx, D, 0.0, 15)
        assert np.abs(xa[0] - xpr).sum() <= FP32_L1
    finally:
        g.close()


def test_ppr_rejects_bad_queries(cuda_device):
    n = 100
    src, dst = gapgen.urand(n, 500, 0x54)
    g = gpu_graph(n, src, dst)
    import torch
    out = torch.empty(2 * n, dtype=torch.float32, device="cuda:0")
    try:
        with pytest.raises(gap.GapError) as e:
            gap.gap_ppr_batch(g.handle, np.array([0, 1, 2], np.int64), np.array([0, n], np.int32), D,
                              1e-4, 10, out)
        assert e.value.status == gap.GAP_ERR_INVALID_ARG
        with pytest.raises(gap.GapError):
            gap.gap_ppr_batch(g.handle, np.array([0, 1, 1], np.int64), np.array([0], np.int32), D,
                              1e-4, 10, out)
    finally:
        g.close()
