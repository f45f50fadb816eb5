"""The no-allocation PageRank entry point (gap_pr_run_noalloc).

It exists for callers that cannot allocate device memory while they call the
library: code running while a CUDA stream is being captured (where cudaMalloc
is not allowed), processes whose device memory is entirely owned by a fixed
memory plan, and latency-critical paths that must not wait on an allocator.
Its scratch lives in a static device array instead.

This file is named so pytest collects it last.  It must pass both when run
alone in a fresh process and after the rest of the suite.
"""
import ctypes

import numpy as np
import pytest

import gapgen
from gpu_helpers import D, FP32_L1, FP32_REL
from paper_1508_03619_gb300 import gap

pytestmark = pytest.mark.gpu


def _run_existing(g, tol, iters):
    import torch
    x = torch.empty(g.n, dtype=torch.float32, device="cuda:0")
    gap.gap_pr_run(g.handle, D, tol, iters, x)
    status, st = gap.gap_pr_stats(g.handle)
    return x.cpu().numpy().astype(np.float64), st


def _run_noalloc(g, tol, iters):
    """Through the C ABI directly: raw device pointer, torch's current stream."""
    import torch
    x = torch.empty(g.n, dtype=torch.float32, device="cuda:0")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = gap.load().gap_pr_run_noalloc(g.handle, D, tol, iters, ctypes.c_void_p(x.data_ptr()), stream)
    assert rc == gap.GAP_OK, gap.last_error_message()
    status, st = gap.gap_pr_stats(g.handle)
    return x.cpu().numpy().astype(np.float64), st


@pytest.mark.parametrize("name", ["urand", "kron"])
def test_noalloc_matches_existing_entry_point_twice(cuda_device, name):
    if name == "urand":
        n = 1 << 16
        src, dst = gapgen.urand(n, 16 * n, 0xA1)
        g = gap.Graph.from_edges(n, src, dst)
    else:
        n = 1 << 15
        src, dst = gapgen.kron(15, 16, 0xA2)
        g = gap.Graph.from_edges(n, src, dst, symmetrize=True)
    try:
        for tol, iters in ((0.0, 20), (1e-4, 100)):
            ref, st_ref = _run_existing(g, tol, iters)
            for _ in range(2):  # two calls in a row share the static array
                x, st = _run_noalloc(g, tol, iters)
                assert st["iterations"] == st_ref["iterations"] or tol > 0
                if tol > 0:
                    assert abs(st["iterations"] - st_ref["iterations"]) <= 1
                l1 = np.abs(x - ref).sum()
                rel = np.max(np.abs(x - ref) / ref)
                assert l1 <= FP32_L1 and rel <= FP32_REL, (l1, rel)
    finally:
        g.close()


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
