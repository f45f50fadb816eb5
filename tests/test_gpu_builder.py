"""GPU graph builder vs the oracle's CSR construction: bit-exact offsets,
neighbour lists and out-degrees (paper §2.3 cleaning rules), plus the device
input generators vs their host twins."""
import numpy as np
import pytest

import gapgen
import oracle
from gpu_helpers import gpu_graph
from paper_1508_03619_gb300 import gap

pytestmark = pytest.mark.gpu


def check_graph(n, src, dst, symmetrize, dedup=True, drop=True):
    g = gpu_graph(n, src, dst, symmetrize, dedup, drop)
    try:
        coff, cidx = oracle.build_csc(n, src, dst, symmetrize, dedup, drop)
        off, idx = oracle.build_csr(n, src, dst, symmetrize, dedup, drop)
        goff, gidx = g.export_csr(1)
        assert np.array_equal(goff, coff)
        assert np.array_equal(gidx, cidx)
        goff0, gidx0 = g.export_csr(0)
        assert np.array_equal(goff0, off)
        assert np.array_equal(gidx0, idx)
        outdeg = np.diff(off)
        assert np.array_equal(g.export_outdeg(), outdeg.astype(np.int32))
        assert g.m == len(cidx)
        assert g.n_dangling == int((outdeg == 0).sum())
    finally:
        g.close()


def test_urand_4096(cuda_device):
    src, dst = gapgen.urand(4096, 65536, 0x1)
    check_graph(4096, src, dst, symmetrize=False)


@pytest.mark.parametrize("scale", [10, 14])
def test_kron_symmetrized(cuda_device, scale):
    src, dst = gapgen.kron(scale, 16, 0x22 + scale)
    check_graph(1 << scale, src, dst, symmetrize=True)


@pytest.mark.parametrize("dedup,drop", [(False, False), (False, True), (True, False)])
def test_cleaning_flags(cuda_device, dedup, drop):
    rng = np.random.default_rng(5)
    n = 300
    src = rng.integers(0, n, 5000).astype(np.int32)
    dst = rng.integers(0, n, 5000).astype(np.int32)
    src[:200] = dst[:200]  # self-loops
    check_graph(n, src, dst, symmetrize=False, dedup=dedup, drop=drop)
    check_graph(n, src, dst, symmetrize=True, dedup=dedup, drop=drop)


def test_degenerate_graphs(cuda_device):
    e = np.zeros(0, np.int32)
    check_graph(1, e, e, False)                        # one vertex, no arcs
    check_graph(17, e, e, True)                        # no arcs
    loops = np.arange(9, dtype=np.int32)
    check_graph(9, loops, loops, False)                # only self-loops
    check_graph(2, np.array([0, 0, 0], np.int32), np.array([1, 1, 1], np.int32), False)


def test_large_tile_span(cuda_device):
    # spans many sort / compaction tiles with a ragged tail
    src, dst = gapgen.urand(100_003, 1_234_567, 0x77)
    check_graph(100_003, src, dst, symmetrize=True)


def test_create_from_csr_matches_edges(cuda_device):
    src, dst = gapgen.urand(5000, 40000, 0x3)
    off, idx = oracle.build_csr(5000, src, dst)
    g = gap.Graph.from_csr(5000, off, idx)
    try:
        coff, cidx = oracle.build_csc(5000, src, dst)
        goff, gidx = g.export_csr(1)
        assert np.array_equal(goff, coff) and np.array_equal(gidx, cidx)
    finally:
        g.close()


def test_bad_ids_rejected(cuda_device):
    with pytest.raises(gap.GapError) as e:
        gpu_graph(10, np.array([0, 10], np.int32), np.array([1, 2], np.int32))
    assert e.value.status == gap.GAP_ERR_INVALID_ARG
    with pytest.raises(gap.GapError) as e:
        gap.Graph.from_csr(3, np.array([0, 2, 1, 3], np.int64), np.array([1, 2, 0], np.int32))
    assert e.value.status == gap.GAP_ERR_INVALID_ARG


def test_device_generators_match_host(cuda_device):
    s1, d1 = gapgen.kron(16, 16, 0x99)
    s2, d2 = gapgen.kron_device(16, 16, 0x99)
    assert np.array_equal(s1, s2.cpu().numpy()) and np.array_equal(d1, d2.cpu().numpy())
    s1, d1 = gapgen.urand(123_457, 500_000, 0x98)
    s2, d2 = gapgen.urand_device(123_457, 500_000, 0x98)
    assert np.array_equal(s1, s2.cpu().numpy()) and np.array_equal(d1, d2.cpu().numpy())
    tab = gapgen.chung_lu_table(1 << 14, 200_000, 2.1)
    s1, d1 = gapgen.chung_lu(1 << 14, 200_000, 2.1, 0x5, table=tab)
    s2, d2 = gapgen.chung_lu_device(1 << 14, 200_000, 2.1, 0x5, table=tab)
    assert np.array_equal(s1, s2.cpu().numpy()) and np.array_equal(d1, d2.cpu().numpy())


def test_create_csc_adopts_a_prebuilt_csr(cuda_device):
    """gap_graph_create_csc takes an in-direction CSR built elsewhere (here: the
    oracle's, from host memory and from device memory) without rebuilding it:
    the stored CSR and out-degrees equal the oracle's, PageRank equals the run
    on the graph built from the same draws bit for bit, and malformed CSRs
    (a row out of order, a source outside [0, n), offsets not ending at m) are
    refused."""
    import torch

    import gapgen
    import oracle
    from gpu_helpers import D, run_gpu
    n = 1 << 14
    src, dst = gapgen.kron(14, 16, 0x17)
    coff, cidx = oracle.build_csc(n, src, dst, symmetrize=True)
    built = gap.Graph.from_edges(n, src, dst, symmetrize=True)
    try:
        x_built, _, _ = run_gpu(built, 0.0, 20)
        for where in ("host", "device"):
            if where == "host":
                a_off, a_idx = coff, cidx
            else:
                a_off, a_idx = torch.from_numpy(coff).cuda(), torch.from_numpy(cidx).cuda()
            g = gap.Graph.from_csc(n, a_off, a_idx)
            try:
                off2, idx2 = g.export_csr(1)
                assert np.array_equal(off2, coff) and np.array_equal(idx2, cidx)
                assert np.array_equal(g.export_outdeg(), np.bincount(cidx, minlength=n).astype(np.int32))
                x, st, _ = run_gpu(g, 0.0, 20)
                assert np.array_equal(x, x_built)
                xo, _, _ = oracle.pagerank(*oracle.build_csr(n, src, dst, symmetrize=True), D, 0.0, 20)
                assert np.abs(x - xo).sum() <= 1e-5
            finally:
                g.close()
    finally:
        built.close()
    bad_rows = cidx.copy()
    r = int(np.flatnonzero(np.diff(coff) >= 2)[0])
    bad_rows[coff[r]], bad_rows[coff[r] + 1] = bad_rows[coff[r] + 1], bad_rows[coff[r]]
    bad_src = cidx.copy()
    bad_src[3] = n
    bad_end = coff.copy()
    bad_end[-1] -= 1
    bad_mono = coff.copy()
    r2 = int(np.flatnonzero(np.diff(coff) >= 1)[5])
    bad_mono[r2 + 1] = bad_mono[r2] - 1   # a row whose end lies before its start
    for o, i, why in ((coff, bad_rows, "sorted"), (coff, bad_src, "outside"), (bad_end, cidx, "end at m"),
                      (bad_mono, cidx, "monotone")):
        with pytest.raises(gap.GapError) as e:
            gap.Graph.from_csc(n, o, i)
        assert e.value.status == gap.GAP_ERR_INVALID_ARG and why in gap.last_error_message()
