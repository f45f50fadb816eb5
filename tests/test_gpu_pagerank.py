"""CUDA PageRank vs the FP64 oracle, element by element, on seeded inputs.

Bars (stated in gpu_helpers): FP64 deterministic mode bit-identical to the
oracle; FP64 binned within L1 1e-12; FP32 within L1 1e-5 and per-vertex
relative 1e-3 after the same fixed iteration count, the same iteration count
+-1 in tolerance mode, and the paper's §3 verifier (< 1e-4) on every
tolerance-mode result.
"""
import numpy as np
import pytest

import gapgen
import oracle
from gpu_helpers import (D, FP64_L1, assert_fp32_parity, exact_l1_change, exact_sum, gpu_graph, oracle_graph,
                         run_gpu, seg_bytes_for)
from paper_1508_03619_gb300 import gap

pytestmark = pytest.mark.gpu


def graph_cases():
    """(name, n, src, dst, symmetrize): small, paper-shaped, several tiles."""
    yield ("urand4096", 4096, *gapgen.urand(4096, 65536, 0x1), False)
    yield ("kron14", 1 << 14, *gapgen.kron(14, 16, 0x14), True)
    yield ("grid96x97", 96 * 97, *gapgen.grid(96, 97, 0.05, 0x4), True)
    n = 1 << 13
    yield ("chunglu8k", n, *gapgen.chung_lu(n, 16 * n, 2.1, 0x5), False)


CASES = list(graph_cases())


def threshold_graph(seed=0x7):
    """Rows whose in-degrees sit at every bin boundary +-1, plus a hub above the
    hub-chunk size and a 1.2M-arc hub, on 2^21 vertices."""
    rng = np.random.default_rng(seed)
    n = 1 << 21
    degs = [0, 1, 4, 5, 16, 17, 64, 65, 2047, 2048, 2049, 9999, 10000, 10001, 32767, 32768,
            32769, 65537, 100_000, 1_200_000]
    src, dst = [], []
    for v, dg in enumerate(degs):
        s = rng.choice(n, size=dg, replace=False).astype(np.int32)
        s[s == v] = (v + 1) % n
        src.append(s)
        dst.append(np.full(dg, v, np.int32))
    s2, d2 = gapgen.urand(n, 4 * n, seed)  # background arcs so sources have out-degree
    src.append(s2)
    dst.append(d2)
    return n, np.concatenate(src), np.concatenate(dst)


@pytest.mark.parametrize("seg", [False, True], ids=["whole", "segmented"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp32_fixed_iterations(cuda_device, case, seg):
    name, n, src, dst, sym = case
    off, idx = oracle_graph(n, src, dst, sym)
    xo, _, _ = oracle.pagerank(off, idx, D, 0.0, 20)
    g = gpu_graph(n, src, dst, sym)
    x, st, status = run_gpu(g, 0.0, 20, segment_bytes=seg_bytes_for(n) if seg else 0)
    assert status == gap.GAP_OK and st["iterations"] == 20
    assert (st["segments"] > 1) == seg
    assert_fp32_parity(x, xo)
    g.close()


@pytest.mark.parametrize("seg", [False, True], ids=["whole", "segmented"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp32_tolerance_mode(cuda_device, case, seg):
    name, n, src, dst, sym = case
    off, idx = oracle_graph(n, src, dst, sym)
    xo, ko, do = oracle.pagerank(off, idx, D, 1e-4, 100)
    g = gpu_graph(n, src, dst, sym)
    x, st, status = run_gpu(g, 1e-4, 100, segment_bytes=seg_bytes_for(n) if seg else 0)
    assert status == gap.GAP_OK and st["converged"]
    assert abs(st["iterations"] - ko) <= 1
    assert oracle.verify(off, idx, x) < 1e-4  # paper §3 verifier
    np.testing.assert_allclose(st["deltas"], do[: st["iterations"]], rtol=1e-3, atol=1e-7)
    assert st["mass"] == pytest.approx(x.sum(), rel=1e-12)
    g.close()


@pytest.mark.parametrize("seg", [False, True], ids=["whole", "segmented"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp32_delta_is_the_exact_l1_change(cuda_device, case, seg):
    """The FP32 stop test's delta of iteration k equals sum |x_k - x_(k-1)| taken
    exactly (fixed point in units of 2^-60, integer sums): the FP32 scores of
    iterations 0..3 (x0 = float(1/n)) against the reported delta history."""
    name, n, src, dst, sym = case
    g = gpu_graph(n, src, dst, sym)
    try:
        prev = np.full(n, np.float32(1.0 / n), np.float64)
        for k in (1, 2, 3):
            x, st, _ = run_gpu(g, 0.0, k, segment_bytes=seg_bytes_for(n) if seg else 0)
            assert st["iterations"] == k
            assert st["deltas"][k - 1] == exact_l1_change(x, prev), (k, st["deltas"][k - 1])
            assert st["mass"] == exact_sum(x)
            prev = x
    finally:
        g.close()


def test_fp64_deterministic_bitexact(cuda_device):
    n, src, dst, sym = CASES[0][1:]
    off, idx = oracle_graph(n, src, dst, sym)
    g = gpu_graph(n, src, dst, sym)
    for tol, iters in ((0.0, 20), (1e-4, 100)):
        xo, ko, do = oracle.pagerank(off, idx, D, tol, iters)
        x, st, status = run_gpu(g, tol, iters, f64=True, deterministic=1)
        assert st["iterations"] == ko
        assert np.array_equal(x, xo), np.abs(x - xo).max()
        np.testing.assert_allclose(st["deltas"], do, rtol=1e-12)
    g.close()


@pytest.mark.parametrize("seg", [False, True], ids=["whole", "segmented"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp64_binned(cuda_device, case, seg):
    name, n, src, dst, sym = case
    off, idx = oracle_graph(n, src, dst, sym)
    xo, ko, _ = oracle.pagerank(off, idx, D, 0.0, 20)
    g = gpu_graph(n, src, dst, sym)
    x, st, _ = run_gpu(g, 0.0, 20, f64=True, segment_bytes=seg_bytes_for(n) if seg else 0)
    assert (st["segments"] > 1) == seg
    assert np.abs(x - xo).sum() <= FP64_L1
    g.close()


@pytest.mark.parametrize("seg", [False, True], ids=["whole", "segmented"])
def test_bin_boundaries_and_hubs(cuda_device, seg):
    n, src, dst = threshold_graph()
    off, idx = oracle_graph(n, src, dst, False)
    xo, _, _ = oracle.pagerank(off, idx, D, 0.0, 12)
    g = gpu_graph(n, src, dst, False)
    sb = seg_bytes_for(n) if seg else 0
    for kahan in (1, 0):
        x, st, _ = run_gpu(g, 0.0, 12, kahan_hubs=kahan, segment_bytes=sb)
        assert_fp32_parity(x, xo)
        hub_rel = np.abs(x[:20] - xo[:20]) / xo[:20]
        print(f"seg={seg} kahan={kahan}: max rel error on the 20 boundary/hub rows {hub_rel.max():.3e}")
        if kahan:
            assert hub_rel.max() < 1e-5
        rows = sum(b["rows"] for b in st["bins"])
        arcs = sum(b["arcs"] for b in st["bins"])
        assert rows == n and arcs == g.m
        assert st["bins"][6]["rows"] >= 4  # the hub bin holds the rows above 32768
    x64, _, _ = run_gpu(g, 0.0, 12, f64=True, segment_bytes=sb)
    assert np.abs(x64 - xo).sum() <= FP64_L1
    g.close()


@pytest.mark.parametrize("seg", [False, True], ids=["whole", "segmented"])
def test_reshaped_bins_keep_parity(cuda_device, seg):
    """Bin bounds, lanes and hub chunk size are tuning knobs: any setting the
    autotuner may pick keeps the FP32 and FP64 parity bars."""
    n, src, dst = threshold_graph()
    off, idx = oracle_graph(n, src, dst, False)
    xo, _, _ = oracle.pagerank(off, idx, D, 0.0, 12)
    g = gpu_graph(n, src, dst, False)
    sb = seg_bytes_for(n) if seg else 0
    try:
        for knobs in ({"group_max_degree": 16, "cta_max_degree": 100, "hub_chunk_arcs": 1024,
                       "group_lanes": 8},
                      {"group_max_degree": 4096, "cta_max_degree": 65536, "hub_chunk_arcs": 8192,
                       "group_lanes": 32},
                      {"small_max_degree": 32, "group_max_degree": 8}):
            x, st, _ = run_gpu(g, 0.0, 12, segment_bytes=sb, **knobs)
            assert_fp32_parity(x, xo)
            assert sum(b["arcs"] for b in st["bins"]) == g.m
            x64, _, _ = run_gpu(g, 0.0, 12, f64=True, segment_bytes=sb, **knobs)
            assert np.abs(x64 - xo).sum() <= FP64_L1
        with pytest.raises(gap.GapError) as e:
            run_gpu(g, 0.0, 2, group_lanes=16)
        assert e.value.status == gap.GAP_ERR_INVALID_ARG
    finally:
        g.close()


@pytest.mark.parametrize("seg", [False, True], ids=["whole", "segmented"])
def test_loop_modes_agree(cuda_device, seg):
    n, src, dst, sym = CASES[1][1:]
    g = gpu_graph(n, src, dst, sym)
    sb = seg_bytes_for(n) if seg else 0
    xa, sa, _ = run_gpu(g, 1e-4, 100, loop=gap.GAP_LOOP_GRAPH, segment_bytes=sb)
    xb, sb_, _ = run_gpu(g, 1e-4, 100, loop=gap.GAP_LOOP_HOST, segment_bytes=sb)
    assert sa["iterations"] == sb_["iterations"]
    assert np.array_equal(xa, xb)
    xc, sc, _ = run_gpu(g, 1e-4, 100, loop=gap.GAP_LOOP_GRAPH, segment_bytes=sb)
    assert np.array_equal(xa, xc)  # run-to-run reproducible
    xt, stt, _ = run_gpu(g, 1e-4, 100, timing=1, segment_bytes=sb)
    assert np.array_equal(xa, xt)
    assert stt["phase_launches"]["finalize"] == stt["iterations"]
    assert stt["kernel_launches"] > stt["iterations"]
    g.close()


def test_host_scores_buffer(cuda_device):
    n, src, dst, sym = CASES[0][1:]
    g = gpu_graph(n, src, dst, sym)
    xa, _, _ = run_gpu(g, 1e-4, 100)
    xb, _, _ = run_gpu(g, 1e-4, 100, host_scores=True)
    assert np.array_equal(xa, xb)
    g.close()


@pytest.mark.parametrize("seg", [False, True], ids=["whole", "segmented"])
def test_bf16_contributions_ladder(cuda_device, seg):
    n, src, dst, sym = CASES[1][1:]
    off, idx = oracle_graph(n, src, dst, sym)
    xo, ko, _ = oracle.pagerank(off, idx, D, 1e-4, 100)
    g = gpu_graph(n, src, dst, sym)
    sb = seg_bytes_for(n) if seg else 0
    x, st, status = run_gpu(g, 1e-4, 100, contrib=gap.GAP_CONTRIB_BF16, bf16_until_log2_delta=-10,
                            segment_bytes=sb)
    assert status == gap.GAP_OK
    assert st["bf16_iters"] >= 1
    assert st["bf16_iters"] < st["iterations"]
    assert oracle.verify(off, idx, x) < 1e-4
    l1 = np.abs(x - xo).sum()
    print(f"bf16 ladder: iters {st['iterations']} (bf16 {st['bf16_iters']}), L1 vs FP64 oracle {l1:.3e}")
    assert l1 < 1e-3
    # BF16 throughout: error is reported, not bounded by the FP32 bar
    x2, st2, _ = run_gpu(g, 1e-4, 100, contrib=gap.GAP_CONTRIB_BF16, segment_bytes=sb)
    assert st2["bf16_iters"] == st2["iterations"]
    print(f"bf16 always: L1 vs FP64 oracle {np.abs(x2 - xo).sum():.3e}")
    g.close()


def test_degenerate_runs(cuda_device):
    e = np.zeros(0, np.int32)
    g = gpu_graph(1, e, e)
    x, st, status = run_gpu(g, 1e-4, 100)
    assert st["iterations"] == 2 and x[0] == np.float32(1 - D)
    g.close()
    g = gpu_graph(1000, e, e)
    x, st, status = run_gpu(g, 0.0, 0)
    assert st["iterations"] == 0 and np.all(x == np.float32(1 / 1000))
    x, st, status = run_gpu(g, 1e-4, 1)
    assert status == gap.GAP_WARN_NOT_CONVERGED and st["iterations"] == 1
    x, st, status = run_gpu(g, 1e-4, 100, f64=True)
    assert st["iterations"] == 2 and np.allclose(x, (1 - D) / 1000, rtol=1e-15)
    g.close()


def test_kron22_full_config(cuda_device):
    """Kronecker scale 22, edge factor 16, symmetrized: FP32 and FP64 vs oracle."""
    scale = 22
    n = 1 << scale
    src, dst = gapgen.kron(scale, 16, 0x22)
    off, idx = oracle_graph(n, src, dst, True)
    g = gpu_graph(n, src, dst, True)
    coff, cidx = g.export_csr(1)
    assert np.array_equal(coff, off) and np.array_equal(cidx, idx)  # symmetric: CSC == CSR
    xo, ko, do = oracle.pagerank(off, idx, D, 0.0, 20)
    x, st, _ = run_gpu(g, 0.0, 20)
    l1, rel = assert_fp32_parity(x, xo)
    xs, sts, _ = run_gpu(g, 0.0, 20, segment_bytes=1 << 20)  # 16 source segments
    assert sts["segments"] == 16
    assert_fp32_parity(xs, xo)
    x64, _, _ = run_gpu(g, 0.0, 20, f64=True)
    assert np.abs(x64 - xo).sum() <= FP64_L1
    xt, stt, _ = run_gpu(g, 1e-4, 100)
    _, kt, _ = oracle.pagerank(off, idx, D, 1e-4, 100)
    assert abs(stt["iterations"] - kt) <= 1
    assert oracle.verify(off, idx, xt) < 1e-4
    print(f"kron22: m={g.m} fp32 L1 {l1:.3e} rel {rel:.3e} iters {stt['iterations']} (oracle {kt})")
    g.close()


def device_attribute(attr):
    """cudaDeviceGetAttribute through the CUDA runtime library (device 0)."""
    import ctypes
    for name in ("libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            continue
    else:
        pytest.skip("CUDA runtime library not found")
    v = ctypes.c_int(0)
    assert rt.cudaDeviceGetAttribute(ctypes.byref(v), attr, 0) == 0
    return v.value


CUDA_ATTR_MAX_PERSISTING_L2 = 108   # cudaDevAttrMaxPersistingL2CacheSize
CUDA_ATTR_MAX_WINDOW = 109          # cudaDevAttrMaxAccessPolicyWindowSize


def test_l2_window_engages_and_changes_no_result(cuda_device):
    """options.l2_window marks the two contribution arrays persisting in L2 when
    they fit the device's persisting carve-out and no L2 blocking runs.  At
    2^20 vertices (8 MB of contributions) it engages on a device whose limits
    allow it, and the scores meet the FP32 bars against the oracle and equal a
    run without the window bit for bit (graph and host loops)."""
    n = 1 << 20
    src, dst = gapgen.kron(20, 16, 0x81)
    off, idx = oracle_graph(n, src, dst, True)
    xo, _, _ = oracle.pagerank(off, idx, D, 0.0, 15)
    g = gpu_graph(n, src, dst, True)
    try:
        fits = min(device_attribute(CUDA_ATTR_MAX_PERSISTING_L2), device_attribute(CUDA_ATTR_MAX_WINDOW)) >= 8 * n
        x0, st0, _ = run_gpu(g, 0.0, 15)
        x1, st1, _ = run_gpu(g, 0.0, 15, l2_window=1)
        assert st0["l2_window_bytes"] == 0 and st1["segments"] == 1
        assert st1["l2_window_bytes"] == (2 * 4 * n if fits else 0)
        print(f"persisting L2 {device_attribute(CUDA_ATTR_MAX_PERSISTING_L2)} B, window max "
              f"{device_attribute(CUDA_ATTR_MAX_WINDOW)} B: window {st1['l2_window_bytes']} B")
        assert_fp32_parity(x1, xo)
        assert np.array_equal(x0, x1)
        assert st0["deltas"] == st1["deltas"]
        x2, st2, _ = run_gpu(g, 0.0, 15, l2_window=1, loop=gap.GAP_LOOP_HOST)
        assert st2["l2_window_bytes"] == st1["l2_window_bytes"]
        assert np.array_equal(x0, x2)
    finally:
        g.close()


@pytest.mark.parametrize("seg", [False, True], ids=["whole", "segmented"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_delta_algorithm_meets_the_criterion(cuda_device, case, seg):
    """options.algorithm = GAP_ALGO_DELTA (residual rounds, pull or frontier
    push): the returned scores pass the paper's §3 verifier (< 1e-4), and lie
    within d*tol/(1-d) (+ FP32 noise) of the oracle's converged vector in L1 --
    the bound a residual below tol gives, since one iteration contracts by d.
    The stats report rounds, the residual history and the arcs touched."""
    name, n, src, dst, sym = case
    off, idx = oracle_graph(n, src, dst, sym)
    x_star, _, _ = oracle.pagerank(off, idx, D, 1e-13, 1000)
    g = gpu_graph(n, src, dst, sym)
    try:
        tol = 1e-4
        x, st, status = run_gpu(g, tol, 100, algorithm=gap.GAP_ALGO_DELTA,
                                segment_bytes=seg_bytes_for(n) if seg else 0)
        assert status == gap.GAP_OK and st["converged"] and st["final_delta"] < tol
        assert st["segments"] > 1 if seg else st["segments"] == 1
        v = oracle.verify(off, idx, x, D)
        assert v < tol, v
        l1 = np.abs(x - x_star).sum()
        assert l1 <= D * tol / (1 - D) + 1e-5, l1
        assert 0 < st["arcs_traversed"] <= st["iterations"] * g.m
        assert len(st["deltas"]) == st["iterations"] and st["deltas"][-1] == st["final_delta"]
        print(f"{name} seg={seg}: rounds {st['iterations']} (sparse {st['sparse_rounds']}), "
              f"arcs {st['arcs_traversed']} = {st['arcs_traversed'] / g.m:.2f} m, verifier {v:.2e}, "
              f"L1 to x* {l1:.2e}")
        # a pull run of the same graph touches m arcs per iteration
        _, sp, _ = run_gpu(g, tol, 100, segment_bytes=seg_bytes_for(n) if seg else 0)
        assert sp["arcs_traversed"] == sp["iterations"] * g.m and sp["sparse_rounds"] == 0
    finally:
        g.close()


@pytest.mark.parametrize("case", ["path", "kron_and_path"])
def test_delta_algorithm_frontier_rounds(cuda_device, case):
    """Graphs whose residual stays local, so the residual algorithm pushes
    frontiers along out-arcs: a directed path (from x0 = 1/n only its first
    vertex has a residual, which travels one arc per round), and a Kronecker
    graph with a long directed path beside it.  The paper's criterion (§3
    verifier) and the contraction bound to the oracle's fixed point hold at
    tol 1e-6; the frontier rounds touch fewer arcs than full rounds would."""
    if case == "path":
        n = 4096
        src = np.arange(n - 1, dtype=np.int32)
        dst = src + 1
    else:
        k = 1 << 12
        ks, kd = gapgen.kron(12, 16, 0x33)
        ks = np.concatenate([ks, kd]).astype(np.int32)  # symmetric Kronecker part
        kd = np.concatenate([kd, gapgen.kron(12, 16, 0x33)[0]]).astype(np.int32)
        p = np.arange(k, 2 * k - 1, dtype=np.int32)
        n = 2 * k
        src = np.concatenate([ks, p])
        dst = np.concatenate([kd, p + 1])
    off, idx = oracle_graph(n, src, dst, False)
    x_star, _, _ = oracle.pagerank(off, idx, D, 1e-14, 2000)
    g = gpu_graph(n, src, dst, False)
    try:
        tol = 1e-6
        for seg in (0, seg_bytes_for(n)):
            x, st, status = run_gpu(g, tol, 1000, algorithm=gap.GAP_ALGO_DELTA, segment_bytes=seg)
            assert status == gap.GAP_OK and st["converged"]
            assert st["sparse_rounds"] >= 1
            assert st["arcs_traversed"] < st["iterations"] * g.m
            v = oracle.verify(off, idx, x, D)
            l1 = np.abs(x - x_star).sum()
            assert v < tol and l1 <= D * tol / (1 - D) + 1e-6, (v, l1)
            print(f"{case} seg={seg}: rounds {st['iterations']} (sparse {st['sparse_rounds']}), arcs "
                  f"{st['arcs_traversed'] / g.m:.2f} m, verifier {v:.2e}, L1 to x* {l1:.2e}")
    finally:
        g.close()


def test_delta_algorithm_edges(cuda_device):
    """No rounds at max_iters = 0 (x0 returned); an empty graph; FP64 or BF16
    with the residual algorithm are refused."""
    import torch
    n = 1000
    g = gpu_graph(n, np.zeros(0, np.int32), np.zeros(0, np.int32))
    try:
        x, st, _ = run_gpu(g, 1e-4, 0, algorithm=gap.GAP_ALGO_DELTA)
        assert st["iterations"] == 0 and np.allclose(x, 1.0 / n)
        x, st, _ = run_gpu(g, 1e-4, 100, algorithm=gap.GAP_ALGO_DELTA)
        assert st["converged"] and np.allclose(x, (1 - D) / n, rtol=1e-6)  # every vertex isolated
        for bad in ({"precision": gap.GAP_PREC_F64}, {"contrib": gap.GAP_CONTRIB_BF16}):
            with pytest.raises(gap.GapError) as e:
                run_gpu(g, 1e-4, 10, algorithm=gap.GAP_ALGO_DELTA, f64=bad.get("precision") is not None,
                        **{k: v for k, v in bad.items() if k != "precision"})
            assert e.value.status == gap.GAP_ERR_UNSUPPORTED
    finally:
        g.close()


@pytest.mark.parametrize("case", ["urand_directed", "kron_sym", "ragged_bins"])
def test_binned_algorithm_fp32_parity(cuda_device, case):
    """options.algorithm = GAP_ALGO_BINNED (scatter into target bins, shared-
    memory sums) meets the FP32 bars against the oracle, with several bins and
    a ragged last bin."""
    if case == "urand_directed":
        n = 70000
        src, dst = gapgen.urand(n, 16 * n, 0x91)
        sym = False
    elif case == "kron_sym":
        n = 1 << 17
        src, dst = gapgen.kron(17, 16, 0x92)
        sym = True
    else:
        n = 3 * 32768 + 17
        src, dst = gapgen.urand(n, 4 * n, 0x93)
        sym = True
    off, idx = oracle_graph(n, src, dst, sym)
    g = gpu_graph(n, src, dst, sym)
    try:
        x, st, status = run_gpu(g, 0.0, 20, algorithm=gap.GAP_ALGO_BINNED)
        xo, _, _ = oracle.pagerank(off, idx, D, 0.0, 20)
        assert st["iterations"] == 20
        assert_fp32_parity(x, xo)
        x, st, status = run_gpu(g, 1e-4, 100, algorithm=gap.GAP_ALGO_BINNED)
        _, ko, _ = oracle.pagerank(off, idx, D, 1e-4, 100)
        assert st["converged"] and abs(st["iterations"] - ko) <= 1
        assert oracle.verify(off, idx, x, D) < 1e-4
        xh, sth, _ = run_gpu(g, 0.0, 20, algorithm=gap.GAP_ALGO_BINNED, loop=gap.GAP_LOOP_HOST)
        assert_fp32_parity(xh, xo)
    finally:
        g.close()


def test_binned_algorithm_edges(cuda_device):
    import torch
    # no arcs: every score (1-d)/n after one iteration
    g = gpu_graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    try:
        x, st, _ = run_gpu(g, 0.0, 3, algorithm=gap.GAP_ALGO_BINNED)
        assert np.allclose(x, (1 - D) / 5, rtol=1e-6)
    finally:
        g.close()
    src, dst = gapgen.urand(100, 400, 0x94)
    g = gpu_graph(100, src, dst)
    try:
        for kw in ({"f64": True}, {"contrib": gap.GAP_CONTRIB_BF16}):
            with pytest.raises(gap.GapError) as e:
                run_gpu(g, 0.0, 3, algorithm=gap.GAP_ALGO_BINNED, **kw)
            assert e.value.status == gap.GAP_ERR_UNSUPPORTED
        o = gap.gap_pr_options_default()
        o.algorithm = 7
        with pytest.raises(gap.GapError) as e:
            gap.gap_pr_run_ex(g.handle, D, 0.0, 3, o, torch.empty(100, device="cuda:0"))
        assert e.value.status == gap.GAP_ERR_INVALID_ARG
    finally:
        g.close()
