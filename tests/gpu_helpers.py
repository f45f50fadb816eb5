"""Shared helpers for the GPU tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs."""
import numpy as np

import oracle
from paper_1508_03619_gb300 import gap

D = 0.85

# Parity bars.  FP32 (scores and accumulation): after the same fixed number
# of iterations, L1 distance to the FP64 oracle <= 1e-5 and per-vertex
# relative error <= 1e-3.  FP64 (binned, reordered sums): each score carries
# at most a few ulps per iteration, so L1 <= 1e-12 on graphs with
# sum(x) <= 1.  FP64 deterministic mode: bit-identical.
FP32_L1 = 1e-5
FP32_REL = 1e-3
FP64_L1 = 1e-12


def torch_dev():
    import torch
    return torch.device("cuda:0")


def gpu_graph(n, src, dst, symmetrize=False, dedup=True, drop_self_loops=True):
    return gap.Graph.from_edges(n, np.ascontiguousarray(src, np.int32),
                                np.ascontiguousarray(dst, np.int32), symmetrize=symmetrize,
                                dedup=dedup, drop_self_loops=drop_self_loops)


def oracle_graph(n, src, dst, symmetrize=False, dedup=True, drop_self_loops=True):
    return oracle.build_csr(n, src, dst, symmetrize, dedup, drop_self_loops)


def seg_bytes_for(n):
    """A segment size that splits the contribution array of n vertices into
    about 4 (FP32) or 8 (FP64) power-of-two source segments, forcing the
    L2-blocked kernels."""
    return max(64, n)


def run_gpu(g, tol, max_iters, f64=False, host_scores=False, **opts):
    """One trial through gap_pr_run_ex; returns (x as float64 numpy, stats, status)."""
    import torch
    o = gap.gap_pr_options_default()
    if f64:
        o.precision = gap.GAP_PREC_F64
    for k, v in opts.items():
        setattr(o, k, v)
    dt = torch.float64 if f64 else torch.float32
    if host_scores:
        x = torch.empty(g.n, dtype=dt).pin_memory()
    else:
        x = torch.empty(g.n, dtype=dt, device=torch_dev())
    gap.gap_pr_run_ex(g.handle, D, tol, max_iters, o, x)
    status, st = gap.gap_pr_stats(g.handle)
    return x.cpu().numpy().astype(np.float64), st, status


def assert_fp32_parity(x_gpu, x_ref):
    l1 = np.abs(x_gpu - x_ref).sum()
    rel = np.max(np.abs(x_gpu - x_ref) / x_ref)
    assert l1 <= FP32_L1, f"L1 {l1:.3e} > {FP32_L1}"
    assert rel <= FP32_REL, f"max rel {rel:.3e} > {FP32_REL}"
    return l1, rel


def exact_l1_change(x, prev):
    """sum |x - prev| over FP32 scores, taken exactly: an FP32 score >= 2^-37 is a
    multiple of 2^-60, so x * 2^60 is an integer (held exactly by float64), the
    differences and their sum are Python integers, and the sum is converted to a
    double once and scaled by 2^-60 (both roundings match the library's)."""
    a = np.asarray(x, np.float32).astype(np.float64) * 2.0 ** 60
    b = np.asarray(prev, np.float32).astype(np.float64) * 2.0 ** 60
    total = sum(abs(int(p) - int(q)) for p, q in zip(a, b))
    return float(total) * 2.0 ** -60


def exact_sum(x):
    """sum x over FP32 scores taken exactly the same way (integers in units of
    2^-60, one conversion to double at the end): the reported mass."""
    a = np.asarray(x, np.float32).astype(np.float64) * 2.0 ** 60
    return float(sum(int(p) for p in a)) * 2.0 ** -60
