"""Connected Components on the GPU (§2.1 CC) against the oracle.

Labels are each component's smallest vertex id on both sides, so the CUDA
result must equal the oracle's union-find element by element, and pass the
paper's verifier (§3: one traversal per label).  Cases cover symmetric and
directed graphs, many small components, a hub outside the giant component
(the warp-wide path), vertices joined only through their out-arcs (the
directed final pass), empty and ragged sizes, host and device label buffers.
At full size (2^26 vertices, the bench's graphs) the labels are checked
against min-label propagation run with torch library operations."""
import numpy as np
import pytest

import gapgen
import oracle
from gpu_helpers import gpu_graph
from paper_1508_03619_gb300 import gap

pytestmark = pytest.mark.gpu


def _run(g, on_device=True):
    import torch
    if on_device:
        lab = torch.full((g.n,), -7, dtype=torch.int32, device="cuda")
    else:
        lab = np.full(g.n, -7, np.int32)
    gap.gap_cc_run(g.handle, lab)
    status, st = gap.gap_cc_stats(g.handle)
    assert status == gap.GAP_OK and st["device_error"] == 0
    out = lab.cpu().numpy() if on_device else lab
    return out, st


def _check(g, n, src, dst, symmetrize):
    off, idx = oracle.build_csr(n, src, dst, symmetrize=symmetrize)
    want = oracle.cc(off, idx)
    got, st = _run(g)
    assert np.array_equal(got, want)
    assert oracle.cc_verify(off, idx, got)
    assert st["components"] == len(np.unique(want))
    assert st["giant_size"] == int((want == st["giant_label"]).sum())
    got_host, _ = _run(g, on_device=False)
    assert np.array_equal(got_host, want)
    return want, st


def _case(kind):
    if kind == "kron_sym":
        n = 1 << 14
        s, d = gapgen.kron(14, 8, seed=0xC10)
        return n, s, d, True
    if kind == "urand_dir_dense":
        n = 1 << 15
        s, d = gapgen.urand(n, 16 * n, seed=0xC11)
        return n, s, d, False
    if kind == "urand_dir_sparse":  # below the giant threshold: thousands of components
        n = 20000 + 37
        s, d = gapgen.urand(n, 9000, seed=0xC12)
        return n, s, d, False
    if kind == "grid_deleted":
        s, d = gapgen.grid(96, 130, 0.45, seed=0xC13)
        return 96 * 130, s, d, True
    if kind == "backward_path":  # every arc points to a smaller id
        n = 5003
        s = np.arange(1, n, dtype=np.int32)
        return n, s, s - 1, False
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["kron_sym", "urand_dir_dense", "urand_dir_sparse", "grid_deleted",
                                  "backward_path"])
def test_cc_matches_oracle(cuda_device, kind):
    n, s, d, sym = _case(kind)
    with gpu_graph(n, s, d, symmetrize=sym) as g:
        want, st = _check(g, n, s, d, sym)
        if kind == "urand_dir_sparse":
            assert st["components"] > 1000
        if kind in ("kron_sym", "urand_dir_dense"):
            assert st["giant_size"] > n // 2


def test_cc_hub_outside_the_giant_and_out_arc_only_vertices(cuda_device):
    """A random giant on 0..9999; a directed out-star (hub 20000 -> 6000
    leaves) that never touches it, so its hub's row is walked warp-wide; and
    100 vertices whose only arc points into the giant from a large id (late in
    their target's in-list, beyond the sampled positions), found only by the
    final pass over out-arcs."""
    rng_s, rng_d = gapgen.urand(10000, 80000, seed=0xC14)
    hub = 20000
    leaves = np.arange(20001, 26001, dtype=np.int32)
    tails = np.arange(30000, 30100, dtype=np.int32)
    src = np.concatenate([rng_s, np.full(len(leaves), hub, np.int32), tails])
    dst = np.concatenate([rng_d, leaves, np.full(len(tails), 5, np.int32)])
    n = 30100 + 29  # a ragged tail of isolated vertices
    for sym in (False, True):
        with gpu_graph(n, src, dst, symmetrize=sym) as g:
            want, _ = _check(g, n, src, dst, sym)
            assert len(np.unique(want[leaves])) == 1 and want[hub] == hub
            assert np.all(want[tails] == want[5])


def test_cc_degenerate_graphs(cuda_device):
    for n in (1, 31, 100, 1000):
        with gpu_graph(n, np.zeros(0, np.int32), np.zeros(0, np.int32)) as g:
            got, st = _run(g)
            assert np.array_equal(got, np.arange(n, dtype=np.int32))
            assert st["components"] == n
    # two vertices, one arc, both directions of storage
    for sym in (False, True):
        with gpu_graph(2, np.array([1], np.int32), np.array([0], np.int32), symmetrize=sym) as g:
            got, st = _run(g)
            assert got.tolist() == [0, 0] and st["components"] == 1


def test_cc_repeat_runs_and_bad_buffers(cuda_device):
    import torch
    n, s, d, sym = _case("kron_sym")
    with gpu_graph(n, s, d, symmetrize=sym) as g:
        a, _ = _run(g)
        b, _ = _run(g)
        assert np.array_equal(a, b)
        with pytest.raises(ValueError):
            gap.gap_cc_run(g.handle, torch.empty(n, dtype=torch.float32, device="cuda"))
        with pytest.raises(ValueError):
            gap.gap_cc_run(g.handle, torch.empty(n - 1, dtype=torch.int32, device="cuda"))
    with pytest.raises(gap.GapError):
        gap.gap_cc_run(None, None)


def _min_label_propagation(in_off, in_idx, n):
    """Smallest id per weak component by repeated min over both ends of every
    arc plus pointer jumping (torch library operations on the device, in
    chunks of about 2^27 arcs)."""
    import torch
    dev = torch.device("cuda")
    bounds = np.unique(np.concatenate([np.searchsorted(in_off, np.arange(0, in_off[-1], 1 << 27), "right") - 1,
                                       [n]]))
    off = torch.from_numpy(in_off).to(dev)
    idx = torch.from_numpy(in_idx).to(dev)
    deg = off[1:] - off[:-1]
    lab = torch.arange(n, dtype=torch.int64, device=dev)
    for _ in range(200):
        new = lab.clone()
        for r0, r1 in zip(bounds[:-1].tolist(), bounds[1:].tolist()):
            a0, a1 = int(in_off[r0]), int(in_off[r1])
            if a1 == a0:
                continue
            rows = torch.repeat_interleave(torch.arange(r0, r1, device=dev), deg[r0:r1], output_size=a1 - a0)
            srcs = idx[a0:a1].long()
            mn = torch.minimum(lab[rows], lab[srcs])
            new.scatter_reduce_(0, rows, mn, reduce="amin")
            new.scatter_reduce_(0, srcs, mn, reduce="amin")
            del rows, srcs, mn
        new = new[new]  # jump: labels stay ids of the same component, never larger
        if torch.equal(new, lab):
            return lab
        lab = new
    raise AssertionError("label propagation did not settle")


@pytest.mark.parametrize("kind", ["kron26", "urand26"])
def test_cc_full_size(cuda_device, kind):
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
        lab = torch.empty(n, dtype=torch.int32, device="cuda")
        gap.gap_cc_run(g.handle, lab)  # first call builds the out-direction of a directed graph
        gap.gap_cc_run(g.handle, lab)
        status, st = gap.gap_cc_stats(g.handle)
        assert status == gap.GAP_OK
        in_off, in_idx = g.export_csr(1)
        want = _min_label_propagation(in_off, in_idx, n)
        assert torch.equal(lab.long(), want)
        assert st["components"] == int((want == torch.arange(n, device="cuda")).sum())
        # the sampled giant is the largest component (kron26 leaves about half its vertices isolated)
        assert st["giant_size"] == int(torch.bincount(want, minlength=n).max())
        assert st["giant_size"] == int((want == st["giant_label"]).sum())
    finally:
        g.close()
        torch.cuda.empty_cache()
