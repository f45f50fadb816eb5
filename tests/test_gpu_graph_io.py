"""Graph files on the GPU: a graph loaded from a text file equals the one the
builder makes from the same draws (bit for bit, and equal to the oracle's
CSR); a saved graph loads back bit-identical and gives bit-identical
PageRank scores; damaged or inconsistent serialized files are rejected and
leave the context usable."""
import re

import numpy as np
import pytest

import gapgen
import oracle
from gpu_helpers import D, assert_fp32_parity, gpu_graph
from paper_1508_03619_gb300 import gap

import gcsc_format

pytestmark = pytest.mark.gpu


def _same_graph(a, b):
    assert (a.n, a.m, a.n_dangling) == (b.n, b.m, b.n_dangling)
    for direction in (1, 0):
        oa, ia = a.export_csr(direction)
        ob, ib = b.export_csr(direction)
        assert np.array_equal(oa, ob) and np.array_equal(ia, ib)
    assert np.array_equal(a.export_outdeg(), b.export_outdeg())


def _scores(g, iters=20):
    import torch
    x = torch.empty(g.n, dtype=torch.float32, device="cuda")
    gap.gap_pr_run(g.handle, D, 0.0, iters, x)
    gap.gap_pr_stats(g.handle)
    return x.cpu().numpy()


def test_text_files_load_like_the_builder(cuda_device, tmp_path):
    scale = 12
    n = 1 << scale
    src, dst = gapgen.kron(scale, 8, seed=0x41)
    ref_dir = gpu_graph(n, src, dst)
    ref_sym = gpu_graph(n, src, dst, symmetrize=True)
    # edge list: n is 1 + the largest id, which the R-MAT draws reach at this size
    assert max(src.max(), dst.max()) == n - 1
    (tmp_path / "k.el").write_text("".join(f"{u} {v}\n" for u, v in zip(src.tolist(), dst.tolist())))
    with gap.Graph.load(tmp_path / "k.el") as g:
        _same_graph(g, ref_dir)
        assert g.build_flags == gap.GAP_DEDUP | gap.GAP_DROP_SELF_LOOPS
    with gap.Graph.load(tmp_path / "k.el", symmetrize=True) as g:
        _same_graph(g, ref_sym)
    # Matrix Market, symmetric: one triangle implies GAP_SYMMETRIZE
    off, idx = ref_sym.export_csr(1)
    rows = np.repeat(np.arange(n), np.diff(off))
    low = rows >= idx
    body = "".join(f"{r + 1} {c + 1}\n" for r, c in zip(rows[low].tolist(), idx[low].tolist()))
    (tmp_path / "k.mtx").write_text(f"%%MatrixMarket matrix coordinate pattern symmetric\n{n} {n} {low.sum()}\n"
                                    + body)
    with gap.Graph.load(tmp_path / "k.mtx") as g:
        _same_graph(g, ref_sym)
        assert g.build_flags & gap.GAP_SYMMETRIZE
    # METIS lists both directions
    lines = [f"{n} {len(idx) // 2}"] + [" ".join(str(j + 1) for j in idx[off[v]:off[v + 1]].tolist())
                                         for v in range(n)]
    (tmp_path / "k.graph").write_text("\n".join(lines) + "\n")
    with gap.Graph.load(tmp_path / "k.graph") as g:
        _same_graph(g, ref_sym)
        # and the loaded graph's PageRank meets the FP32 parity bars against the oracle
        ooff, oidx = oracle.build_csr(n, src, dst, True, True, True)
        x_ref, _, _ = oracle.pagerank(ooff, oidx, D, 0.0, 20)
        assert_fp32_parity(_scores(g).astype(np.float64), x_ref)
    ref_dir.close()
    ref_sym.close()


@pytest.mark.parametrize("kind", ["kron_sym", "urand_dir", "single_vertex"])
def test_save_load_round_trip(cuda_device, tmp_path, kind):
    if kind == "kron_sym":
        n = 1 << 14
        src, dst = gapgen.kron(14, 16, seed=0x42)
        g = gpu_graph(n, src, dst, symmetrize=True)
    elif kind == "urand_dir":
        n = 5000  # not a power of two: a ragged payload tail
        src, dst = gapgen.urand(n, 40000, seed=0x43)
        g = gpu_graph(n, src, dst)
    else:
        n = 1
        g = gpu_graph(1, np.zeros(0, np.int32), np.zeros(0, np.int32))
    p = tmp_path / "g.gcsc"
    g.save(p)
    # the file is what the format documents: header, the in-direction CSR, checksum
    fn, fm, fflags, _, foff, fidx = gcsc_format.read(p)
    off, idx = g.export_csr(1)
    assert (fn, fm, fflags) == (g.n, g.m, g.build_flags)
    assert np.array_equal(foff, off) and np.array_equal(fidx, idx)
    with gap.Graph.load(p) as h:
        _same_graph(h, g)
        assert h.build_flags == g.build_flags
        if g.m:
            assert np.array_equal(_scores(h), _scores(g))  # same arrays, same kernels: same bits
    # a file written by the independent writer loads too
    q = tmp_path / "h.gcsc"
    gcsc_format.write(q, g.n, off, idx, flags=g.build_flags)
    with gap.Graph.load(q) as h:
        _same_graph(h, g)
    g.close()


def test_damaged_or_inconsistent_files_are_rejected(cuda_device, tmp_path):
    n = 6
    # rows (in-direction): 0 <- {1, 2}; 1 <- {0}; 2 <- {}; 3 <- {0, 4, 5}; 4 <- {3}; 5 <- {}
    off = np.array([0, 2, 3, 3, 6, 7, 7], np.int64)
    idx = np.array([1, 2, 0, 0, 4, 5, 3], np.int32)
    good = tmp_path / "good.gcsc"
    gcsc_format.write(good, n, off, idx)
    with gap.Graph.load(good) as g:
        assert (g.n, g.m) == (6, 7)
        assert g.export_outdeg().tolist() == [2, 1, 1, 1, 1, 1]
        assert g.n_dangling == 0
    raw = bytearray(good.read_bytes())
    raw[64 + 8 * (n + 1) + 4] ^= 1  # one bit of the sources
    bad = tmp_path / "flip.gcsc"
    bad.write_bytes(bytes(raw))
    with pytest.raises(gap.GapError, match="checksum"):
        gap.gap_graph_load(bad)
    cases = {
        "unsorted": (off, np.array([2, 1, 0, 0, 4, 5, 3], np.int32), "not sorted"),
        "range": (off, np.array([1, 2, 0, 0, 4, 6, 3], np.int32), "outside [0, n)"),
        "negative": (off, np.array([1, 2, -1, 0, 4, 5, 3], np.int32), "outside [0, n)"),
        "monotone": (np.array([0, 2, 1, 3, 6, 7, 7], np.int64), idx, "monotone"),
        "ends": (np.array([0, 2, 3, 3, 6, 7, 6], np.int64), idx, "end at m"),
        "start": (np.array([1, 2, 3, 3, 6, 7, 7], np.int64), idx, "start at 0"),
    }
    for name, (o, i, msg) in cases.items():
        p = tmp_path / f"{name}.gcsc"
        gcsc_format.write(p, n, o, i)
        with pytest.raises(gap.GapError, match=re.escape(msg)) as ei:
            gap.gap_graph_load(p)
        assert ei.value.status == gap.GAP_ERR_INVALID_ARG
    # the context is intact: a graph still loads and runs
    with gap.Graph.load(good) as g:
        x = _scores(g, 5)
        assert np.all(np.isfinite(x)) and np.all(x > 0)


def test_loaded_graph_runs_cc_and_bfs_through_the_directed_paths(cuda_device, tmp_path):
    """A loaded graph does not trust the file's symmetrize flag, so CC and BFS
    take their directed code paths (out-direction built on first use) on
    symmetric data; the results must not change."""
    import torch
    n = 1 << 13
    src, dst = gapgen.kron(13, 8, seed=0x44)
    off, idx = oracle.build_csr(n, src, dst, symmetrize=True)
    with gpu_graph(n, src, dst, symmetrize=True) as g:
        p = tmp_path / "k.gcsc"
        g.save(p)
    with gap.Graph.load(p) as h:
        lab = torch.empty(n, dtype=torch.int32, device="cuda")
        gap.gap_cc_run(h.handle, lab)
        gap.gap_cc_stats(h.handle)
        assert np.array_equal(lab.cpu().numpy(), oracle.cc(off, idx))
        par = torch.empty(n, dtype=torch.int32, device="cuda")
        for s in gap.bfs_sources(h.export_outdeg(), 4, seed=0x13):
            gap.gap_bfs_run(h.handle, s, par)
            st = gap.gap_bfs_stats(h.handle)
            assert oracle.bfs_verify(off, idx, s, par.cpu().numpy())
            assert st["reached"] == int((oracle.bfs_depths(off, idx, s) >= 0).sum())
