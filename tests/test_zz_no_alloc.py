"""The no-allocation PageRank entry point (gap_pr_run_noalloc).

It exists for callers that cannot allocate device memory while they call the
library: processes whose device memory is entirely owned by a fixed memory
plan or arena, and latency-critical paths that must not wait on an allocator
or run out of memory half-way through a call.  Its scratch lives in a static
device array instead.  It synchronizes its stream, so it is never called on a
stream under capture.

Each case holds the entry point's scores against the FP64 oracle (20 fixed
iterations: the FP32 bars; tolerance mode: within one iteration of the oracle
and the paper's one-more-iteration criterion) and against the existing
entry point gap_pr_run, on two calls in a row (the calls share the static
array).

This file is named so pytest collects it last.  It must pass both when run
alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import gapgen
import oracle
from gpu_helpers import D, FP32_L1, FP32_REL, assert_fp32_parity
from paper_1508_03619_gb300 import gap

pytestmark = pytest.mark.gpu


def _run_existing(g, tol, iters):
    import torch
    x = torch.empty(g.n, dtype=torch.float32, device="cuda:0")
    gap.gap_pr_run(g.handle, D, tol, iters, x)
    status, st = gap.gap_pr_stats(g.handle)
    return x.cpu().numpy().astype(np.float64), st


def _noalloc(g, tol, iters, x, stream_handle):
    """Through the C ABI directly: raw device pointer, raw stream handle."""
    rc = gap.load().gap_pr_run_noalloc(g.handle, D, tol, iters, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(stream_handle))
    assert rc == gap.GAP_OK, gap.last_error_message()


def _run_noalloc(g, tol, iters):
    import torch
    x = torch.empty(g.n, dtype=torch.float32, device="cuda:0")
    _noalloc(g, tol, iters, x, torch.cuda.current_stream().cuda_stream)
    status, st = gap.gap_pr_stats(g.handle)
    return x.cpu().numpy().astype(np.float64), st


def _graph(name):
    """The test graphs, built on the GPU and by the oracle from the same draws."""
    if name == "urand":
        n = 1 << 16
        src, dst = gapgen.urand(n, 16 * n, 0xA1)
        sym = False
    elif name == "kron":
        n = 1 << 15
        src, dst = gapgen.kron(15, 16, 0xA2)
        sym = True
    else:  # the largest graph the entry point accepts: n = GAP_NOALLOC_MAX_VERTICES
        n = gap.GAP_NOALLOC_MAX_VERTICES
        src, dst = gapgen.kron(n.bit_length() - 1, 8, 0xA3)
        sym = True
    off, idx = oracle.build_csr(n, src, dst, symmetrize=sym)
    return gap.Graph.from_edges(n, src, dst, symmetrize=sym), (off, idx)


@pytest.mark.parametrize("name", ["urand", "kron", "max_vertices"])
def test_noalloc_matches_oracle_and_existing_entry_point_twice(cuda_device, name):
    g, (off, idx) = _graph(name)
    try:
        assert g.n <= gap.GAP_NOALLOC_MAX_VERTICES
        # 20 fixed iterations: element by element against the FP64 oracle
        x_or, k_or, _ = oracle.pagerank(off, idx, D, 0.0, 20)
        ref, _ = _run_existing(g, 0.0, 20)
        for _ in range(2):  # two calls in a row share the static array
            x, st = _run_noalloc(g, 0.0, 20)
            assert st["iterations"] == 20
            assert_fp32_parity(x, x_or)
            l1 = np.abs(x - ref).sum()
            rel = np.max(np.abs(x - ref) / ref)
            assert l1 <= FP32_L1 and rel <= FP32_REL, (l1, rel)
        # tolerance mode: within one iteration of the oracle, and the paper's
        # criterion (one more classical iteration changes < 1e-4) holds
        x_or, k_or, _ = oracle.pagerank(off, idx, D, 1e-4, 100)
        for _ in range(2):
            x, st = _run_noalloc(g, 1e-4, 100)
            assert st["converged"]
            assert abs(st["iterations"] - k_or) <= 1, (st["iterations"], k_or)
            assert oracle.verify(off, idx, x, D) < 1e-4
            if st["iterations"] == k_or:
                assert_fp32_parity(x, x_or)
            else:  # one iteration apart: the two iterates differ by one delta (< 1e-4)
                assert np.abs(x - x_or).sum() < 2e-4
    finally:
        g.close()


def test_noalloc_back_to_back_on_two_streams_with_two_graphs(cuda_device):
    """A call returns only after its last use of the shared array, so a next
    call on another stream, with another graph, finds the array free."""
    import torch
    g1, (off1, idx1) = _graph("urand")
    g2, (off2, idx2) = _graph("kron")
    try:
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        x1 = torch.empty(g1.n, dtype=torch.float32, device="cuda:0")
        x2 = torch.empty(g2.n, dtype=torch.float32, device="cuda:0")
        exp1, _, _ = oracle.pagerank(off1, idx1, D, 0.0, 20)
        exp2, _, _ = oracle.pagerank(off2, idx2, D, 0.0, 20)
        for _ in range(2):
            _noalloc(g1, 0.0, 20, x1, s1.cuda_stream)
            _, st1 = gap.gap_pr_stats(g1.handle)
            _noalloc(g2, 0.0, 20, x2, s2.cuda_stream)
            _, st2 = gap.gap_pr_stats(g2.handle)
            torch.cuda.synchronize()
            assert st1["iterations"] == 20 and st2["iterations"] == 20
            assert_fp32_parity(x1.cpu().numpy().astype(np.float64), exp1)
            assert_fp32_parity(x2.cpu().numpy().astype(np.float64), exp2)
            # the mass each call reports is its own graph's
            assert abs(st1["mass"] - float(x1.double().sum())) < 1e-6
            assert abs(st2["mass"] - float(x2.double().sum())) < 1e-6
    finally:
        g1.close()
        g2.close()


def test_noalloc_rejects_graphs_above_its_limit(cuda_device):
    n = gap.GAP_NOALLOC_MAX_VERTICES + 1
    src = np.array([0, 1], np.int32)
    dst = np.array([1, 2], np.int32)
    g = gap.Graph.from_edges(n, src, dst)
    try:
        import torch
        x = torch.empty(n, dtype=torch.float32, device="cuda:0")
        rc = gap.load().gap_pr_run_noalloc(g.handle, D, 1e-4, 10, ctypes.c_void_p(x.data_ptr()), None)
        assert rc == gap.GAP_ERR_INVALID_ARG
        assert "at most" in gap.last_error_message()
    finally:
        g.close()
