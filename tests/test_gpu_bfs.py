"""Breadth-first search on the GPU (§2.1 BFS) against the oracle.

Several parent arrays are correct for one source, so every GPU result is
checked by the paper's verifier (oracle.bfs_verify: parent[source] = source,
-1 exactly where the oracle's serial BFS finds no path, an arc parent -> v,
and the oracle's depths one apart), and the reached count must equal the
oracle's.  Cases: symmetric Kronecker and directed uniform graphs (both
directions of the search run), many unreachable vertices, a high-diameter
lattice (top-down nearly throughout), a long directed path, a hub whose out-row is far
longer than a top-down chunk, sources without out-arcs, host and device
buffers.  At full size (2^26 vertices, the bench's graphs) the definition is
checked with torch library operations: every parent is an in-neighbour, tree
depths never let an arc skip a level, and no arc leaves the reached set."""
import numpy as np
import pytest

import gapgen
import oracle
from gpu_helpers import gpu_graph
from paper_1508_03619_gb300 import gap

pytestmark = pytest.mark.gpu


def _run(g, source, on_device=True):
    import torch
    if on_device:
        par = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
    else:
        par = np.full(g.n, -7, np.int32)
    gap.gap_bfs_run(g.handle, source, par)
    st = gap.gap_bfs_stats(g.handle)
    return (par.cpu().numpy() if on_device else par), st


def _check_sources(g, off, idx, sources, on_device=True):
    stats = []
    for s in sources:
        par, st = _run(g, s, on_device)
        assert oracle.bfs_verify(off, idx, s, par), f"source {s}"
        depth = oracle.bfs_depths(off, idx, s)
        assert st["reached"] == int((depth >= 0).sum())
        assert st["levels"] >= int(depth.max()) + 1
        stats.append(st)
    return stats


def _case(kind):
    if kind == "kron_sym":
        n = 1 << 15
        s, d = gapgen.kron(15, 16, seed=0xB10)
        return n, s, d, True
    if kind == "urand_dir_dense":
        n = 1 << 15
        s, d = gapgen.urand(n, 16 * n, seed=0xB11)
        return n, s, d, False
    if kind == "urand_dir_sparse":
        n = 30000 + 13
        s, d = gapgen.urand(n, 36000, seed=0xB12)
        return n, s, d, False
    if kind == "grid_deleted":
        s, d = gapgen.grid(120, 150, 0.05, seed=0xB13)
        return 120 * 150, s, d, True
    if kind == "backward_path":
        n = 4000 + 7
        s = np.arange(1, n, dtype=np.int32)
        return n, s, s - 1, False
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["kron_sym", "urand_dir_dense", "urand_dir_sparse", "grid_deleted",
                                  "backward_path"])
def test_bfs_matches_oracle(cuda_device, kind):
    n, s, d, sym = _case(kind)
    off, idx = oracle.build_csr(n, s, d, symmetrize=sym)
    with gpu_graph(n, s, d, symmetrize=sym) as g:
        sources = gap.bfs_sources(g.export_outdeg(), 6, seed=0xB0 + len(kind))
        if kind == "backward_path":
            sources = [n - 1, n // 2, 1]
        stats = _check_sources(g, off, idx, sources)
        _check_sources(g, off, idx, sources[:2], on_device=False)
        if kind in ("kron_sym", "urand_dir_dense"):
            assert any(st["bottom_up_steps"] > 0 for st in stats)  # the search turned bottom-up
            assert all(st["top_down_steps"] > 0 for st in stats)
        if kind in ("grid_deleted", "backward_path"):
            # thin frontiers stay top-down until few unexplored arcs remain
            assert all(st["top_down_steps"] > st["bottom_up_steps"] for st in stats)


def test_bfs_hub_rows_and_sources_without_out_arcs(cuda_device):
    """A hub with 50,000 out-arcs (many top-down chunks of one row) feeding a
    random graph; a source with no out-arcs reaches only itself."""
    base_s, base_d = gapgen.urand(60000, 200000, seed=0xB14)
    hub = 60000
    leaves = np.arange(0, 50000, dtype=np.int32)
    src = np.concatenate([base_s, np.full(len(leaves), hub, np.int32), np.array([hub + 1], np.int32)])
    dst = np.concatenate([base_d, leaves, np.array([hub], np.int32)])
    n = hub + 3  # hub+2 has no arcs at all
    off, idx = oracle.build_csr(n, src, dst)
    with gpu_graph(n, src, dst) as g:
        _check_sources(g, off, idx, [hub, hub + 1, 7])
        par, st = _run(g, hub + 2)
        assert st["reached"] == 1 and par[hub + 2] == hub + 2 and (np.delete(par, hub + 2) == -1).all()
        deg = g.export_outdeg()
        z = int(np.flatnonzero(deg == 0)[0])
        par, st = _run(g, z)
        assert oracle.bfs_verify(off, idx, z, par) and st["reached"] == 1


def test_bfs_degenerate_and_bad_arguments(cuda_device):
    import torch
    with gpu_graph(1, np.zeros(0, np.int32), np.zeros(0, np.int32)) as g:
        par, st = _run(g, 0)
        assert par.tolist() == [0] and st["reached"] == 1
    with gpu_graph(3, np.array([0, 1], np.int32), np.array([1, 2], np.int32)) as g:
        par, st = _run(g, 0)
        assert par.tolist() == [0, 0, 1] and st["reached"] == 3 and st["levels"] == 3
        par, st = _run(g, 2)
        assert par.tolist() == [-1, -1, 2]
        for bad in (-1, 3):
            with pytest.raises(gap.GapError):
                gap.gap_bfs_run(g.handle, bad, torch.empty(3, dtype=torch.int32, device="cuda"))
        with pytest.raises(ValueError):
            gap.gap_bfs_run(g.handle, 0, torch.empty(3, dtype=torch.float32, device="cuda"))
        with pytest.raises(ValueError):
            gap.gap_bfs_run(g.handle, 0, torch.empty(2, dtype=torch.int32, device="cuda"))


def _check_bfs_definition_torch(in_off, in_idx, n, source, parent):
    """§2.1 BFS definition at full size with torch operations on the device:
    parent[source] = source; each other reached v has parent[v] among its
    in-neighbours (rows of the CSC are sorted, so the keys row*2^32 + source
    are sorted and searchsorted finds an arc); depths of the parent tree (by
    pointer doubling) let no arc u->v skip a level, and no arc leaves the
    reached set.  Tree depths that no arc can shorten are BFS distances, so
    every parent sits one level above its child."""
    import torch
    dev = torch.device("cuda")
    p = parent.long()
    assert int(p[source]) == source
    reached = p >= 0
    v_all = torch.arange(n, device=dev)
    # depth by pointer doubling over the tree
    anc = torch.where(reached, p, v_all)
    dep = (reached & (v_all != source)).long()
    for _ in range(40):
        if bool((anc[anc] == anc).all()):
            break
        dep, anc = dep + dep[anc], anc[anc]
    assert bool((anc[reached] == source).all())  # every tree path ends at the source
    bounds = np.unique(np.concatenate([np.searchsorted(in_off, np.arange(0, in_off[-1], 1 << 27), "right") - 1,
                                       [n]]))
    off_d = torch.from_numpy(in_off).to(dev)
    idx_d = torch.from_numpy(in_idx).to(dev)
    deg = off_d[1:] - off_d[:-1]
    for r0, r1 in zip(bounds[:-1].tolist(), bounds[1:].tolist()):
        a0, a1 = int(in_off[r0]), int(in_off[r1])
        if a1 == a0:
            continue
        rows = torch.repeat_interleave(torch.arange(r0, r1, device=dev), deg[r0:r1], output_size=a1 - a0)
        srcs = idx_d[a0:a1].long()
        # no arc from a reached vertex to an unreached one; no arc skips a level
        ru = reached[srcs]
        assert bool((reached[rows] | ~ru).all())
        both = ru & reached[rows]
        assert bool((dep[rows[both]] <= dep[srcs[both]] + 1).all())
        # parent of every reached, non-source row of this chunk is one of its in-neighbours
        keys = rows * (1 << 32) + srcs
        vs = torch.arange(r0, r1, device=dev)
        want = reached[r0:r1] & (vs != source)
        q = vs[want] * (1 << 32) + p[r0:r1][want]
        pos = torch.searchsorted(keys, q).clamp(max=len(keys) - 1)
        assert bool((keys[pos] == q).all())
        del rows, srcs, keys, ru, both
    return int(reached.sum()), int(dep.max())


@pytest.mark.parametrize("kind", ["kron26", "urand26"])
def test_bfs_full_size(cuda_device, kind):
    import torch
    n = 1 << 26
    if kind == "kron26":
        src, dst = gapgen.kron_device(26, 16, 0x26)
        g = gap.Graph.from_edges(n, src, dst, symmetrize=True)
    else:
        src, dst = gapgen.urand_device(n, 16 * n, 0x26)
        g = gap.Graph.from_edges(n, src, dst, symmetrize=False)
    del src, dst
    torch.cuda.empty_cache()
    try:
        in_off, in_idx = g.export_csr(1)
        par = torch.empty(n, dtype=torch.int32, device="cuda")
        for s in gap.bfs_sources(g.export_outdeg(), 2, seed=0x26):
            gap.gap_bfs_run(g.handle, s, par)
            st = gap.gap_bfs_stats(g.handle)
            reached, depth = _check_bfs_definition_torch(in_off, in_idx, n, s, par)
            assert st["reached"] == reached and reached > n // 3
            assert st["bottom_up_steps"] > 0 and st["levels"] >= depth + 1
    finally:
        g.close()
        torch.cuda.empty_cache()


def test_bfs_and_cc_on_a_road_like_lattice(cuda_device):
    """A 256 x 256 lattice with 5 % of its edges deleted (the road-like shape
    of the batch workload): hundreds of thin levels, one step per level plus
    the step that finds nothing, and connected components on the same graph."""
    import torch
    rows = cols = 256
    s, d = gapgen.grid(rows, cols, 0.05, seed=0xB15)
    n = rows * cols
    off, idx = oracle.build_csr(n, s, d, symmetrize=True)
    with gpu_graph(n, s, d, symmetrize=True) as g:
        for src in (0, n // 2 + cols // 2, n - 1):
            par, st = _run(g, src)
            depth = oracle.bfs_depths(off, idx, src)
            assert oracle.bfs_verify(off, idx, src, par)
            assert st["levels"] == int(depth.max()) + 1 and st["levels"] > 250
        lab = torch.empty(n, dtype=torch.int32, device="cuda")
        gap.gap_cc_run(g.handle, lab)
        _, cst = gap.gap_cc_stats(g.handle)
        want = oracle.cc(off, idx)
        assert np.array_equal(lab.cpu().numpy(), want) and cst["components"] == len(np.unique(want))
