"""Pins for the CPU oracle: checks against things other than the oracle itself.

Each test ties one part of the oracle to a fact fixed by the paper or by
mathematics — closed forms of the §2.1 PageRank equation on small graphs, a
dense linear solve of its fixed point, the contraction that the §2.1
tolerance argument rests on, brute-force CSR construction (§2.3) — so that a
plausible slip in the oracle (a dropped d, 1/n vs 1, in- vs out-degree, a
transposed operand, dangling mass redistributed, '<=' for '<', returning the
older iterate) fails at least one of them.
"""
import numpy as np
import pytest

import oracle

D = 0.85


# ---------------------------------------------------------------- helpers ---

def csr_from_arcs(n, arcs):
    """Tiny out-CSR from an explicit arc list, no cleaning."""
    src = np.array([a for a, _ in arcs], np.int32)
    dst = np.array([b for _, b in arcs], np.int32)
    return oracle.build_csr(n, src, dst, symmetrize=False, dedup=False, drop_self_loops=False)


def dense_fixed_point(n, arcs, d=D, teleport=None):
    """Solve (I - d * A^T D^-1) x = (1-d) t with numpy (library solve).
    A[u, v] counts arcs u->v; dangling columns (out-degree 0) are zero."""
    A = np.zeros((n, n))
    for u, v in arcs:
        A[u, v] += 1.0
    outdeg = A.sum(axis=1)
    P = np.zeros((n, n))
    for u in range(n):
        if outdeg[u] > 0:
            P[:, u] = A[u, :] / outdeg[u]
    t = np.full(n, 1.0 / n) if teleport is None else teleport
    return np.linalg.solve(np.eye(n) - d * P, (1.0 - d) * t)


def random_arcs(rng, n, m, self_loops=True):
    arcs = []
    for _ in range(m):
        u, v = int(rng.integers(n)), int(rng.integers(n))
        if not self_loops and u == v:
            continue
        arcs.append((u, v))
    return arcs


# --------------------------------------------------------- CSR builder §2.3 ---

@pytest.mark.parametrize("symmetrize", [False, True])
@pytest.mark.parametrize("dedup", [False, True])
@pytest.mark.parametrize("drop", [False, True])
@pytest.mark.parametrize("seed", range(6))
def test_csr_matches_brute_force(symmetrize, dedup, drop, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 12))
    m = int(rng.integers(0, 40))
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    arcs = []
    for u, v in zip(src.tolist(), dst.tolist()):
        if drop and u == v:
            continue
        arcs.append((u, v))
        if symmetrize:
            arcs.append((v, u))
    if dedup:
        arcs = sorted(set(arcs))
    rows = [sorted(v for (u, v) in arcs if u == r) for r in range(n)]
    off, idx = oracle.build_csr(n, src, dst, symmetrize, dedup, drop)
    assert off[0] == 0 and len(off) == n + 1
    for r in range(n):
        assert idx[off[r]:off[r + 1]].tolist() == rows[r]
    assert off[n] == len(idx) == sum(len(r) for r in rows)


@pytest.mark.parametrize("threads", [2, 3, 7])
@pytest.mark.parametrize("symmetrize", [False, True])
@pytest.mark.parametrize("dedup,drop", [(True, True), (False, False), (True, False)])
def test_threaded_csr_equals_serial(threads, symmetrize, dedup, drop):
    """The row-partitioned builder gives the serial builder's CSR bit for bit
    (which the brute-force pin above fixes), for any thread count, with
    duplicates, self-loops, hubs and isolated vertices in the draws."""
    import gapgen
    cases = [(1 << 12, *gapgen.kron(12, 8, 0xC1)), (5000, *gapgen.urand(5000, 30000, 0xC2))]
    rng = np.random.default_rng(0xC3)
    n = 37
    src = rng.integers(0, n, 400).astype(np.int32)
    dst = rng.integers(0, n, 400).astype(np.int32)
    dst[:50] = 5  # a hub with repeated arcs
    src[50:60] = dst[50:60]  # self-loops
    cases.append((n, src, dst))
    cases.append((1, np.zeros(3, np.int32), np.zeros(3, np.int32)))
    cases.append((9, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    for n, src, dst in cases:
        a = oracle.build_csr(n, src, dst, symmetrize, dedup, drop)
        b = oracle.build_csr(n, src, dst, symmetrize, dedup, drop, threads=threads)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    with pytest.raises(ValueError):
        oracle.build_csr(3, np.array([0, 3], np.int32), np.array([1, 1], np.int32), threads=2)


def test_pagerank_from_continues_the_iteration():
    """Continuing x_k for j iterations gives x_{k+j} of one uninterrupted run
    bit for bit, with the same deltas; the stop test applies to new deltas."""
    import gapgen
    n = 1 << 11
    off, idx = oracle.build_csr(n, *gapgen.kron(11, 16, 0xC4), symmetrize=True)
    x20, _, h20 = oracle.pagerank(off, idx, D, 0.0, 20)
    x7, _, _ = oracle.pagerank(off, idx, D, 0.0, 7)
    x, k, h = oracle.pagerank_from(off, idx, x7, 13, D)
    assert k == 13 and np.array_equal(x, x20) and np.array_equal(h, h20[7:])
    xt, kt, _ = oracle.pagerank(off, idx, D, 1e-4, 100)
    xr, kr, hr = oracle.pagerank_from(off, idx, x7, 100, D, 1e-4)
    assert 7 + kr == kt and np.array_equal(xr, xt) and hr[-1] < 1e-4
    x0 = np.full(n, 1.0 / n)
    xs, ks, _ = oracle.pagerank_from(off, idx, x0, 5, D)
    assert np.array_equal(xs, oracle.pagerank(off, idx, D, 0.0, 5)[0])


def test_csc_is_transpose():
    rng = np.random.default_rng(7)
    n, m = 30, 200
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    off, idx = oracle.build_csr(n, src, dst)
    coff, cidx = oracle.build_csc(n, src, dst)
    out_arcs = {(u, int(v)) for u in range(n) for v in idx[off[u]:off[u + 1]]}
    in_arcs = {(int(u), v) for v in range(n) for u in cidx[coff[v]:coff[v + 1]]}
    assert out_arcs == in_arcs
    assert all(u != v for u, v in out_arcs)


def test_csr_rejects_bad_ids():
    with pytest.raises(ValueError):
        oracle.build_csr(3, np.array([0, 3], np.int32), np.array([1, 1], np.int32))


# ------------------------------------------------------ closed forms §2.1 ---

@pytest.mark.parametrize("n", [1, 2, 7, 64])
def test_directed_cycle_is_uniform(n):
    arcs = [(i, (i + 1) % n) for i in range(n)] if n > 1 else []
    off, idx = csr_from_arcs(n, arcs)
    if n == 1:
        pytest.skip("a 1-cycle is a self-loop; covered by the empty-graph test")
    x, k, deltas = oracle.pagerank(off, idx, tol=0.0, max_iters=5)
    assert k == 5
    np.testing.assert_allclose(x, 1.0 / n, rtol=0, atol=1e-16)
    assert deltas[0] < 1e-15


@pytest.mark.parametrize("n", [2, 5, 16])
def test_complete_digraph_is_uniform(n):
    arcs = [(u, v) for u in range(n) for v in range(n) if u != v]
    off, idx = csr_from_arcs(n, arcs)
    x, _, deltas = oracle.pagerank(off, idx, tol=0.0, max_iters=4)
    np.testing.assert_allclose(x, 1.0 / n, rtol=1e-15)
    assert max(deltas) < 1e-14


@pytest.mark.parametrize("k", [1, 3, 10, 63])
def test_undirected_star_closed_form(k):
    # Fixed point of the §2.1 equation on a star with centre 0 and k leaves:
    #   C = (1-d)/n + d*k*L,  L = (1-d)/n + d*C/k   (n = k+1)
    # => C = (1+dk)/(n(1+d)),  L = (1-d)/n + d(1+dk)/(k n (1+d)).
    n = k + 1
    arcs = [(0, i) for i in range(1, n)] + [(i, 0) for i in range(1, n)]
    off, idx = csr_from_arcs(n, arcs)
    x, _, _ = oracle.pagerank(off, idx, tol=1e-15, max_iters=2000)
    C = (1 + D * k) / (n * (1 + D))
    L = (1 - D) / n + D * (1 + D * k) / (k * n * (1 + D))
    assert abs(x[0] - C) < 1e-13
    np.testing.assert_allclose(x[1:], L, rtol=0, atol=1e-13)
    assert abs(x.sum() - 1.0) < 1e-12


@pytest.mark.parametrize("k", [1, 4, 50])
def test_in_star_drops_dangling_mass(k):
    # Leaves point at a centre that has no out-edges (dangling).  Leaves have no
    # in-edges, so from iteration 1 on they hold (1-d)/n; the centre receives
    # d * k * (previous leaf score).  Exact after two iterations, and the mass
    # (1-d)(n+dk)/n < 1 shows the dangling mass is dropped, not redistributed.
    n = k + 1
    arcs = [(i, 0) for i in range(1, n)]
    off, idx = csr_from_arcs(n, arcs)
    x1, _, _ = oracle.pagerank(off, idx, tol=0.0, max_iters=1)
    assert x1[0] == pytest.approx((1 - D) / n + D * k / n, rel=1e-15)
    x, iters, deltas = oracle.pagerank(off, idx, tol=0.0, max_iters=4)
    leaf = (1 - D) / n
    assert x[0] == pytest.approx(leaf * (1 + D * k), rel=1e-14)
    np.testing.assert_allclose(x[1:], leaf, rtol=1e-15)
    assert x.sum() == pytest.approx((1 - D) * (n + D * k) / n, rel=1e-14)
    assert deltas[2] == 0.0 and deltas[3] == 0.0
    # max_iters = 2 must return the second iterate (the newest), already exact
    x2, k2, _ = oracle.pagerank(off, idx, tol=0.0, max_iters=2)
    assert k2 == 2 and x2[0] == x[0]


@pytest.mark.parametrize("n", [1, 4, 1000])
def test_empty_graph(n):
    off, idx = csr_from_arcs(n, [])
    x, k, deltas = oracle.pagerank(off, idx)  # tol = 1e-4
    np.testing.assert_allclose(x, (1 - D) / n, rtol=1e-15)
    assert deltas[0] == pytest.approx(D, rel=1e-12)
    assert k == 2 and deltas[1] == 0.0


def test_stop_rule_is_strict():
    # §2.1 tolerance equation uses '<': with tol equal to the first change, the
    # oracle must not stop after iteration 1.
    off, idx = csr_from_arcs(8, [])
    _, _, deltas = oracle.pagerank(off, idx, tol=0.0, max_iters=3)
    _, k, _ = oracle.pagerank(off, idx, tol=float(deltas[0]), max_iters=10)
    assert k == 2
    _, k, _ = oracle.pagerank(off, idx, tol=float(np.nextafter(deltas[0], 1.0)), max_iters=10)
    assert k == 1


# ------------------------------------------------- dense solve, n <= 64 ---

@pytest.mark.parametrize("seed", range(12))
def test_matches_dense_solve(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 65))
    arcs = random_arcs(rng, n, int(rng.integers(0, 4 * n)), self_loops=False)
    off, idx = csr_from_arcs(n, arcs)  # multigraph: repeated arcs each count
    x, k, _ = oracle.pagerank(off, idx, tol=1e-15, max_iters=5000)
    xs = dense_fixed_point(n, arcs)
    assert np.abs(x - xs).sum() <= 1e-12
    # the contraction the §2.1 tolerance argument rests on:
    #   ||x_k - x*||_1 <= d^k ||x_0 - x*||_1
    e0 = np.abs(1.0 / n - xs).sum()
    for kk in (1, 2, 5, 10):
        xk, _, _ = oracle.pagerank(off, idx, tol=0.0, max_iters=kk)
        assert np.abs(xk - xs).sum() <= D ** kk * e0 + 1e-14


def test_directed_asymmetry_pins_operand_order():
    # 0 -> 1, 0 -> 2, 1 -> 2 : pushing along reversed arcs or dividing by
    # in-degree gives a different fixed point than the dense solve.
    arcs = [(0, 1), (0, 2), (1, 2)]
    off, idx = csr_from_arcs(3, arcs)
    x, _, _ = oracle.pagerank(off, idx, tol=1e-15, max_iters=1000)
    b = (1 - D) / 3
    x1 = b + D * b / 2
    x2 = b + D * (b / 2 + x1)
    np.testing.assert_allclose(x, [b, x1, x2], rtol=1e-14)
    np.testing.assert_allclose(x, dense_fixed_point(3, arcs), rtol=1e-13)


# ------------------------------------------------------------ invariants ---

@pytest.mark.parametrize("seed", range(8))
def test_invariants(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(5, 300))
    src = rng.integers(0, n, 6 * n).astype(np.int32)
    dst = rng.integers(0, n, 6 * n).astype(np.int32)
    sym = bool(seed % 2)
    off, idx = oracle.build_csr(n, src, dst, symmetrize=sym)
    outdeg = np.diff(off)
    x, k, deltas = oracle.pagerank(off, idx, tol=0.0, max_iters=30)
    assert np.all(x >= (1 - D) / n * (1 - 1e-15))
    if np.all(outdeg > 0):
        assert abs(x.sum() - 1.0) < 1e-12
    else:
        assert x.sum() <= 1.0 + 1e-12
    for a, b in zip(deltas[:-1], deltas[1:]):
        assert b <= D * a + 1e-15 * n


# -------------------------------------------------------- verifier (§3) ---

def test_verifier_agrees_with_next_delta():
    rng = np.random.default_rng(3)
    n = 200
    src = rng.integers(0, n, 1500).astype(np.int32)
    dst = rng.integers(0, n, 1500).astype(np.int32)
    off, idx = oracle.build_csr(n, src, dst)
    x5, _, _ = oracle.pagerank(off, idx, tol=0.0, max_iters=5)
    _, _, d6 = oracle.pagerank(off, idx, tol=0.0, max_iters=6)
    assert oracle.verify(off, idx, x5) == d6[5]
    x, k, deltas = oracle.pagerank(off, idx)
    assert deltas[-1] < 1e-4 and oracle.verify(off, idx, x) < 1e-4
    bad = x.copy()
    bad[:10] += 1e-3
    assert oracle.verify(off, idx, bad) > 1e-4


def test_iteration_band_on_paper_shaped_graphs():
    # §2.1: 1e-4 gives "5 - 20" iterations for most graphs (a sanity band).
    import gapgen
    for src, dst, n, sym in [(*gapgen.kron(12, 16, 9), 1 << 12, True),
                             (*gapgen.urand(1 << 12, 16 << 12, 9), 1 << 12, False)]:
        off, idx = oracle.build_csr(n, src, dst, symmetrize=sym)
        _, k, _ = oracle.pagerank(off, idx)
        assert 5 <= k <= 20


# --------------------------------------------------- personalized PR ---

def test_ppr_all_seeds_is_pagerank():
    rng = np.random.default_rng(11)
    n = 120
    src = rng.integers(0, n, 700).astype(np.int32)
    dst = rng.integers(0, n, 700).astype(np.int32)
    off, idx = oracle.build_csr(n, src, dst)
    x, _, _ = oracle.pagerank(off, idx, tol=0.0, max_iters=25)
    y, _, _ = oracle.ppr(off, idx, np.arange(n, dtype=np.int32), tol=0.0, max_iters=25)
    assert np.abs(x - y).sum() < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_ppr_matches_dense_solve(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(3, 65))
    arcs = random_arcs(rng, n, 3 * n, self_loops=False)
    off, idx = csr_from_arcs(n, arcs)
    seeds = rng.integers(0, n, int(rng.integers(1, 6))).astype(np.int32)
    x, _, _ = oracle.ppr(off, idx, seeds, tol=1e-15, max_iters=5000)
    t = np.zeros(n)
    t[np.unique(seeds)] = 1.0 / len(np.unique(seeds))
    xs = dense_fixed_point(n, arcs, teleport=t)
    assert np.abs(x - xs).sum() <= 1e-12
    # repeated seeds count once
    y, _, _ = oracle.ppr(off, idx, np.unique(seeds), tol=1e-15, max_iters=5000)
    np.testing.assert_array_equal(x, y)


def test_ppr_single_seed_star():
    # Seed at the centre of an undirected star with k leaves: by symmetry the
    # fixed point solves C = (1-d) + d*k*L, L = d*C/k.
    k = 9
    n = k + 1
    arcs = [(0, i) for i in range(1, n)] + [(i, 0) for i in range(1, n)]
    off, idx = csr_from_arcs(n, arcs)
    x, _, _ = oracle.ppr(off, idx, np.array([0], np.int32), tol=1e-15, max_iters=5000)
    C = (1 - D) / (1 - D * D)
    L = D * C / k
    assert x[0] == pytest.approx(C, rel=1e-13)
    np.testing.assert_allclose(x[1:], L, rtol=1e-13)


# ------------------------------------------------ cross-machine fixture ---

def test_oracle_golden_fingerprint():
    """The oracle and generator give the same bits on every machine (x86 here,
    Arm on the GPU host): FP64 with no FMA contraction and integer-only draws."""
    import json
    import os
    import sys
    here = os.path.join(os.path.dirname(__file__), "golden")
    sys.path.insert(0, here)
    try:
        import make_golden
    finally:
        sys.path.remove(here)
    with open(os.path.join(here, "urand4096_oracle.json")) as f:
        want = json.load(f)
    assert make_golden.fingerprint() == want


def test_pr_rows_is_one_pull_iteration():
    """The sampled-row update (used at sizes the full serial iteration cannot
    reach) is the §2.1 equation: on every row it equals the next push
    iterate, and it agrees with a dense evaluation y' = b + d A^T D^-1 x."""
    rng = np.random.default_rng(11)
    n = 300
    src = rng.integers(0, 250, 2000).astype(np.int32)  # vertices >= 250 are dangling
    dst = rng.integers(0, n // 2, 2000).astype(np.int32)  # vertices >= n/2 without in-arcs
    src[:40] = dst[:40]                                    # self-loops, removed by the builder
    off, idx = oracle.build_csr(n, src, dst)
    in_off, in_idx = oracle.build_csc(n, src, dst)
    outdeg = np.diff(off).astype(np.int32)
    assert (outdeg == 0).any()
    x5, _, _ = oracle.pagerank(off, idx, tol=0.0, max_iters=5)
    x6, _, _ = oracle.pagerank(off, idx, tol=0.0, max_iters=6)
    y = oracle.pr_rows(in_off, in_idx, outdeg, x5, np.arange(n))
    assert np.max(np.abs(y - x6)) <= 1e-15
    A = np.zeros((n, n))
    for u in range(n):
        A[u, idx[off[u]:off[u + 1]]] = 1.0
    c = np.where(outdeg > 0, x5 / np.maximum(outdeg, 1), 0.0)
    dense = (1 - oracle.DAMPING) / n + oracle.DAMPING * (A.T @ c)
    assert np.max(np.abs(y - dense)) <= 1e-15
    sub = rng.choice(n, 17, replace=False)
    assert np.array_equal(oracle.pr_rows(in_off, in_idx, outdeg, x5, sub), y[sub])
    # sampled estimate of the verifier's summed change is unbiased: full sample = exact
    assert abs(np.abs(y - x5).sum() - oracle.verify(off, idx, x5)) <= 1e-15


def test_ppr_rows_is_one_ppr_iteration():
    """The sampled-row personalized update equals the next iterate of the
    oracle's PPR run on every row (repeated seeds count once)."""
    rng = np.random.default_rng(12)
    n = 250
    src = rng.integers(0, 200, 1500).astype(np.int32)
    dst = rng.integers(0, n, 1500).astype(np.int32)
    off, idx = oracle.build_csr(n, src, dst)
    in_off, in_idx = oracle.build_csc(n, src, dst)
    outdeg = np.diff(off).astype(np.int32)
    seeds = np.array([3, 17, 3, 240, 17, 99], np.int32)
    x4, _, _ = oracle.ppr(off, idx, seeds, tol=0.0, max_iters=4)
    x5, _, _ = oracle.ppr(off, idx, seeds, tol=0.0, max_iters=5)
    y = oracle.ppr_rows(in_off, in_idx, outdeg, x4, seeds, np.arange(n))
    assert np.max(np.abs(y - x5)) <= 1e-15
    # the teleport lands on the 4 distinct seeds only
    assert np.count_nonzero(oracle.ppr_rows(in_off, in_idx, outdeg, np.zeros(n), seeds, np.arange(n))) == 4


def test_cpu_pull_baseline_agrees_with_oracle():
    """The multi-core CPU baseline (pull over the CSC) computes the same
    iterates as the oracle, to FP64 rounding."""
    import gapgen
    n = 1 << 12
    src, dst = gapgen.kron(12, 16, 13)
    off, idx = oracle.build_csr(n, src, dst, symmetrize=True)
    in_off, in_idx = oracle.build_csc(n, src, dst, symmetrize=True)
    x, k, threads = oracle.cpu_pagerank_pull(in_off, in_idx, np.diff(off).astype(np.int32), tol=0.0, max_iters=20)
    xo, _, _ = oracle.pagerank(off, idx, tol=0.0, max_iters=20)
    assert k == 20 and threads >= 1
    assert np.abs(x - xo).sum() <= 1e-12


# ------------------------------------------------- connected components ---
# §2.1 CC: same label exactly when an undirected path joins two vertices; the
# oracle labels each component by its smallest vertex id.

def _min_id_labels(n, comp):
    """Relabel any component numbering by the smallest member id."""
    mins = np.full(comp.max() + 1 if n else 0, np.iinfo(np.int64).max, np.int64)
    np.minimum.at(mins, comp, np.arange(n))
    return mins[comp].astype(np.int32)


def _bfs_components(n, arcs):
    """Brute force: undirected adjacency sets, BFS from every unlabelled vertex
    in ascending order (so the first vertex reached is the smallest)."""
    adj = [set() for _ in range(n)]
    for u, v in arcs:
        adj[u].add(v)
        adj[v].add(u)
    lab = [-1] * n
    for s in range(n):
        if lab[s] >= 0:
            continue
        lab[s] = s
        frontier = [s]
        while frontier:
            nxt = []
            for u in frontier:
                for w in adj[u]:
                    if lab[w] < 0:
                        lab[w] = s
                        nxt.append(w)
            frontier = nxt
    return np.array(lab, np.int32)


def test_cc_closed_forms():
    n = 9
    # no arcs: every vertex is its own component (zero-degree vertices get their own label)
    off, idx = csr_from_arcs(n, [])
    assert oracle.cc(off, idx).tolist() == list(range(n))
    # a directed path is one weak component, whichever way it points
    fwd = [(i, i + 1) for i in range(n - 1)]
    bwd = [(i + 1, i) for i in range(n - 1)]
    for arcs in (fwd, bwd):
        off, idx = csr_from_arcs(n, arcs)
        assert oracle.cc(off, idx).tolist() == [0] * n
    # in-star onto the last vertex: arcs only point inwards, still one component
    off, idx = csr_from_arcs(n, [(i, n - 1) for i in range(n - 1)])
    assert oracle.cc(off, idx).tolist() == [0] * n
    # two directed cycles {0,2,4,6,8} and {1,3,5,7} plus a self-loop on 7
    arcs = [(0, 2), (2, 4), (4, 6), (6, 8), (8, 0), (7, 5), (5, 3), (3, 1), (1, 7), (7, 7)]
    off, idx = csr_from_arcs(n, arcs)
    assert oracle.cc(off, idx).tolist() == [0, 1, 0, 1, 0, 1, 0, 1, 0]


def test_cc_matches_brute_force_on_every_small_digraph():
    """All 2^12 digraphs on 4 vertices without self-loops, and random ones
    on 7 vertices with multi-arcs and self-loops."""
    pairs = [(u, v) for u in range(4) for v in range(4) if u != v]
    for mask in range(1 << len(pairs)):
        arcs = [p for b, p in enumerate(pairs) if mask >> b & 1]
        off, idx = csr_from_arcs(4, arcs)
        assert np.array_equal(oracle.cc(off, idx), _bfs_components(4, arcs)), arcs
    rng = np.random.default_rng(0xCC)
    for _ in range(300):
        k = int(rng.integers(0, 12))
        arcs = [tuple(map(int, rng.integers(0, 7, 2))) for _ in range(k)]
        off, idx = csr_from_arcs(7, arcs)
        assert np.array_equal(oracle.cc(off, idx), _bfs_components(7, arcs))


@pytest.mark.parametrize("kind", ["urand_sparse", "kron_sym", "grid_deleted"])
def test_cc_matches_scipy_weak_components(kind):
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    import gapgen
    if kind == "urand_sparse":  # below the giant-component threshold: many components
        n = 20000
        src, dst = gapgen.urand(n, 9000, seed=0xC1)
        off, idx = oracle.build_csr(n, src, dst)
    elif kind == "kron_sym":
        n = 1 << 14
        src, dst = gapgen.kron(14, 4, seed=0xC2)
        off, idx = oracle.build_csr(n, src, dst, symmetrize=True)
    else:
        src, dst = gapgen.grid(64, 96, 0.45, seed=0xC3)
        n = 64 * 96
        off, idx = oracle.build_csr(n, src, dst, symmetrize=True)
    A = sp.csr_matrix((np.ones(len(idx)), idx, off), shape=(n, n))
    k, comp = csg.connected_components(A, directed=True, connection="weak")
    want = _min_id_labels(n, comp)
    got = oracle.cc(off, idx)
    assert k > 1
    assert np.array_equal(got, want)
    assert len(np.unique(got)) == k


def test_cc_verifier_accepts_components_and_rejects_merges_and_splits():
    import gapgen
    n = 4000
    src, dst = gapgen.urand(n, 2500, seed=0xC4)
    off, idx = oracle.build_csr(n, src, dst)
    lab = oracle.cc(off, idx)
    assert oracle.cc_verify(off, idx, lab)
    # any other member id per component is as good a label
    uniq = np.unique(lab)
    other = {}
    for l in uniq:
        members = np.flatnonzero(lab == l)
        other[l] = members[-1]
    relab = np.array([other[l] for l in lab], np.int32)
    assert oracle.cc_verify(off, idx, relab)
    # two components under one label: one of them is never reached
    sizes = {l: int((lab == l).sum()) for l in uniq}
    big = [l for l in uniq if sizes[l] > 1]
    merged = lab.copy()
    merged[lab == big[1]] = big[0]
    assert not oracle.cc_verify(off, idx, merged)
    # one component split in two labels: a traversal meets a different label
    split = lab.copy()
    members = np.flatnonzero(lab == big[0])
    split[members[-1]] = members[-1]
    assert not oracle.cc_verify(off, idx, split)
    # isolated vertices under one shared label are also a merge
    iso = np.flatnonzero((np.diff(off) == 0) & (np.bincount(idx, minlength=n) == 0))
    assert len(iso) >= 2
    shared = lab.copy()
    shared[iso[1]] = iso[0]
    assert not oracle.cc_verify(off, idx, shared)


# ------------------------------------------------- breadth-first search ---
# §2.1 BFS: parent[source] = source, -1 where unreachable, an arc parent -> v,
# depth[parent] = depth[v] - 1; §3: depths from a serial BFS.

def test_bfs_depth_closed_forms():
    n = 12
    off, idx = csr_from_arcs(n, [(i, i + 1) for i in range(n - 1)])  # directed path
    assert oracle.bfs_depths(off, idx, 0).tolist() == list(range(n))
    k = 5
    assert oracle.bfs_depths(off, idx, k).tolist() == [-1] * k + list(range(n - k))
    off, idx = csr_from_arcs(n, [(0, i) for i in range(1, n)])  # out-star
    assert oracle.bfs_depths(off, idx, 0).tolist() == [0] + [1] * (n - 1)
    assert oracle.bfs_depths(off, idx, 3).tolist() == [-1, -1, -1, 0] + [-1] * (n - 4)
    import gapgen
    rows, cols = 9, 14  # full lattice: depth = Manhattan distance
    src, dst = gapgen.grid(rows, cols, 0.0, seed=1)
    off, idx = oracle.build_csr(rows * cols, src, dst, symmetrize=True)
    s = 3 * cols + 7
    d = oracle.bfs_depths(off, idx, s)
    r, c = np.divmod(np.arange(rows * cols), cols)
    assert np.array_equal(d, np.abs(r - 3) + np.abs(c - 7))


@pytest.mark.parametrize("kind", ["urand_dir", "kron_sym"])
def test_bfs_depths_match_scipy(kind):
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    import gapgen
    if kind == "urand_dir":
        n = 3000
        s, d = gapgen.urand(n, 4000, seed=0xB1)
        off, idx = oracle.build_csr(n, s, d)
    else:
        n = 1 << 12
        s, d = gapgen.kron(12, 4, seed=0xB2)
        off, idx = oracle.build_csr(n, s, d, symmetrize=True)
    A = sp.csr_matrix((np.ones(len(idx)), idx, off), shape=(n, n))
    for source in (0, 17, n - 1, int(np.argmax(np.diff(off)))):
        dist = csg.shortest_path(A, directed=True, unweighted=True, indices=source)
        want = np.where(np.isinf(dist), -1, dist).astype(np.int32)
        assert np.array_equal(oracle.bfs_depths(off, idx, source), want)


def _parents_from_depths(off, idx, depth, source, pick):
    """A valid parent array built by hand from the depths: for every reached v,
    the smallest (pick=min) or largest (pick=max) u with an arc u->v and
    depth[u] = depth[v] - 1."""
    n = len(off) - 1
    cand = [[] for _ in range(n)]
    for u in range(n):
        for v in idx[off[u]:off[u + 1]]:
            if depth[u] >= 0 and depth[v] == depth[u] + 1:
                cand[v].append(u)
    par = np.full(n, -1, np.int32)
    for v in range(n):
        if cand[v]:
            par[v] = pick(cand[v])
    par[source] = source
    return par


def test_bfs_verifier_accepts_every_valid_tree_and_rejects_each_broken_rule():
    import gapgen
    n = 2000
    s, d = gapgen.urand(n, 3000, seed=0xB3)
    off, idx = oracle.build_csr(n, s, d)
    source = int(np.argmax(np.diff(off)))
    depth = oracle.bfs_depths(off, idx, source)
    lo = _parents_from_depths(off, idx, depth, source, min)
    hi = _parents_from_depths(off, idx, depth, source, max)
    assert (lo != hi).any()  # more than one correct answer exists here
    assert oracle.bfs_verify(off, idx, source, lo) and oracle.bfs_verify(off, idx, source, hi)
    reached = np.flatnonzero((depth > 1))
    unreached = np.flatnonzero(depth < 0)
    assert len(reached) and len(unreached)
    v = int(reached[0])
    bad = lo.copy(); bad[source] = -1                        # source is not its own parent
    assert not oracle.bfs_verify(off, idx, source, bad)
    for out_of_range in (n, -2):                             # a parent that is no vertex
        bad = lo.copy(); bad[int(reached[-1])] = out_of_range
        assert not oracle.bfs_verify(off, idx, source, bad)
    bad = lo.copy(); bad[v] = -1                             # a reachable vertex left out
    assert not oracle.bfs_verify(off, idx, source, bad)
    bad = lo.copy(); bad[int(unreached[0])] = source         # an unreachable vertex given a parent
    assert not oracle.bfs_verify(off, idx, source, bad)
    same = [u for u in range(n) if depth[u] == depth[v] and u != v]
    bad = lo.copy(); bad[v] = same[0]                        # parent at the same depth (and no arc)
    assert not oracle.bfs_verify(off, idx, source, bad)
    # parent one level up but without an arc to v
    up = [u for u in range(n) if depth[u] == depth[v] - 1 and not np.isin(v, idx[off[u]:off[u + 1]])]
    bad = lo.copy(); bad[v] = up[0]
    assert not oracle.bfs_verify(off, idx, source, bad)
    # an arc into v from a vertex one level deeper: an arc, but the wrong depth
    deeper = [u for u in range(n) if depth[u] == depth[v] + 1 and np.isin(v, idx[off[u]:off[u + 1]])]
    if deeper:
        bad = lo.copy(); bad[v] = deeper[0]
        assert not oracle.bfs_verify(off, idx, source, bad)
