"""Full-size graphs (2^26 vertices, the bench's workloads) in the bench's
launch configuration, held against the FP64 oracle on the same draws with the
oracle's own CSR (its row-partitioned builder, identical to the serial one):
  - FP32 (tuned bins, L2 segments, hub chunks): converged within one iteration
    of the oracle, L1 <= 1e-5 and per-vertex relative <= 1e-3 against the
    oracle's iterate of the same count, the §3 verifier < 1e-4;
  - FP64: L1 <= 1e-12 against the oracle's iterate of the same count;
  - BF16 contributions with the FP32 ladder: converged, the §3 verifier
    < 1e-4, errors against the oracle's iterate of the same count printed;
  - the residual algorithm (GAP_ALGO_DELTA): the §3 verifier < 1e-4 and L1 to
    the oracle's iterate within 2 d tol / (1 - d);
  - every score >= (1-d)/n, the FP64 mass matches the scores, mass <= 1."""
import os

import numpy as np
import pytest

import gapgen
import oracle
from gpu_helpers import D, FP32_L1, FP32_REL, FP64_L1
from paper_1508_03619_gb300 import gap, tuning

pytestmark = pytest.mark.gpu

THREADS = max(1, os.cpu_count() or 1)


def oracle_iterates(off, idx, counts, x_t, k_t):
    """The oracle's iterates x_k for the GPU's iteration counts, from its
    tolerance-mode run (x_t after k_t iterations), continued where needed."""
    out = {}
    for k in sorted(set(counts)):
        if k == k_t:
            out[k] = x_t
        elif k > k_t:
            out[k] = oracle.pagerank_from(off, idx, x_t, k - k_t, D)[0]
        else:
            out[k] = oracle.pagerank(off, idx, D, 0.0, k)[0]
    return out


def gpu_run(g, n, **fields):
    import torch
    o = tuning.pagerank_options()
    for k, v in fields.items():
        setattr(o, k, v)
    f64 = fields.get("precision") == gap.GAP_PREC_F64
    x = torch.empty(n, dtype=torch.float64 if f64 else torch.float32, device="cuda:0")
    gap.gap_pr_run_ex(g.handle, D, 1e-4, 100, o, x)
    status, st = gap.gap_pr_stats(g.handle)
    assert status == gap.GAP_OK and st["converged"] and st["final_delta"] < 1e-4
    return x.cpu().numpy().astype(np.float64), st


@pytest.mark.parametrize("kind", ["kron26", "urand26"])
def test_full_size_against_oracle(cuda_device, kind):
    import torch
    n = 1 << 26
    if kind == "kron26":
        hs, hd = gapgen.kron(26, 16, 0x26)
        sym = True
    else:
        hs, hd = gapgen.urand(n, 16 * n, 0x26)
        sym = False
    off, idx = oracle.build_csr(n, hs, hd, symmetrize=sym, threads=THREADS)
    del hs, hd
    if kind == "kron26":
        src, dst = gapgen.kron_device(26, 16, 0x26)
    else:
        src, dst = gapgen.urand_device(n, 16 * n, 0x26)
    g = gap.Graph.from_edges(n, src, dst, symmetrize=sym)
    del src, dst
    torch.cuda.empty_cache()
    try:
        assert g.m == len(idx)
        x32, st32 = gpu_run(g, n)
        assert st32["segments"] >= 2
        if kind == "kron26":
            assert st32["bins"][6]["rows"] > 0  # hub rows, pulled in chunks
        x64, st64 = gpu_run(g, n, precision=gap.GAP_PREC_F64)
        xbf, stbf = gpu_run(g, n, contrib=gap.GAP_CONTRIB_BF16, bf16_until_log2_delta=-10)
        x_t, k_t, _ = oracle.pagerank(off, idx, D, 1e-4, 100)
        # FP32 and FP64 stop within one iteration of the oracle; BF16 rounding
        # slows the early iterations, so that run is held to the verifier
        for st in (st32, st64):
            assert abs(st["iterations"] - k_t) <= 1, (st["iterations"], k_t)
        xo = oracle_iterates(off, idx, [st32["iterations"], st64["iterations"], stbf["iterations"]],
                             x_t, k_t)
        o32 = xo[st32["iterations"]]
        l1 = float(np.abs(x32 - o32).sum())
        rel = float(np.max(np.abs(x32 - o32) / o32))
        assert l1 <= FP32_L1 and rel <= FP32_REL, (l1, rel)
        l1_64 = float(np.abs(x64 - xo[st64["iterations"]]).sum())
        assert l1_64 <= FP64_L1, l1_64
        ob = xo[stbf["iterations"]]
        l1_bf = float(np.abs(xbf - ob).sum())
        rel_bf = float(np.max(np.abs(xbf - ob) / ob))
        v32 = oracle.verify(off, idx, x32, D)
        vbf = oracle.verify(off, idx, xbf, D)
        assert v32 < 1e-4 and vbf < 1e-4, (v32, vbf)
        # the residual algorithm: the paper's criterion, and within twice the
        # contraction bound d*tol/(1-d) of the oracle's own converged iterate
        xdl, stdl = gpu_run(g, n, algorithm=gap.GAP_ALGO_DELTA)
        vdl = oracle.verify(off, idx, xdl, D)
        l1_dl = float(np.abs(xdl - x_t).sum())
        assert vdl < 1e-4 and l1_dl <= 2 * D * 1e-4 / (1 - D), (vdl, l1_dl)
        if kind == "kron26":
            # the CSR handed back from host memory (gap_graph_create_csc: uploaded in
            # 1 GB chunks while checked) is the same graph: out-degrees equal, and
            # the same trial gives the same scores bit for bit
            h_off, h_idx = g.export_csr(1)
            gu = gap.Graph.from_csc(n, h_off, h_idx)
            try:
                assert gu.m == g.m and np.array_equal(gu.export_outdeg(), g.export_outdeg())
                xu, _ = gpu_run(gu, n)
                assert np.array_equal(xu, x32)
            finally:
                gu.close()
            del h_off, h_idx
        base = (1 - D) / n
        assert x32.min() >= base * (1 - 1e-6)
        assert abs(st32["mass"] - x32.sum()) <= 1e-9 and st32["mass"] <= 1 + 1e-5
        print(f"{kind}: m={g.m} iterations fp32/fp64/bf16 {st32['iterations']}/{st64['iterations']}/"
              f"{stbf['iterations']} (oracle {k_t}); vs oracle: fp32 L1 {l1:.3e} rel {rel:.3e}, "
              f"fp64 L1 {l1_64:.3e}, bf16-ladder L1 {l1_bf:.3e} rel {rel_bf:.3e}; "
              f"verifier fp32 {v32:.3e} bf16 {vbf:.3e}; residual algorithm {stdl['iterations']} rounds "
              f"({stdl['sparse_rounds']} sparse), {stdl['arcs_traversed'] / g.m:.2f} m arcs, verifier "
              f"{vdl:.3e}, L1 to the oracle {l1_dl:.3e}")
    finally:
        g.close()


def test_full_size_ppr(cuda_device):
    """Personalized PageRank on the serving graph (Chung-Lu, 2^24 vertices, 5e8
    draws): each query converges, keeps mass <= 1, and meets the one-more-
    iteration criterion estimated on 2^17 rows (plus its seeds) recomputed by
    the oracle (oracle.ppr_rows) from the GPU's scores; a query run through the
    continuous-batching server equals the batch entry point bit for bit."""
    import torch
    n = 1 << 24
    table = gapgen.chung_lu_table(n, 500_000_000, 2.1)
    hs, hd = gapgen.chung_lu(n, 500_000_000, 2.1, 0x5C, table=table)
    in_off, in_idx = oracle.build_csr(n, hd, hs, threads=THREADS)  # the oracle's own CSC
    del hs, hd
    outdeg = np.bincount(in_idx, minlength=n).astype(np.int32)  # arcs leaving each vertex
    src, dst = gapgen.chung_lu_device(n, 500_000_000, 2.1, 0x5C, table=table)
    g = gap.Graph.from_edges(n, src, dst, symmetrize=False)
    del src, dst
    torch.cuda.empty_cache()
    try:
        assert g.m == len(in_idx)
        rng = np.random.default_rng(0x5E)
        cand = np.flatnonzero(outdeg > 0)
        queries = [rng.choice(cand, size=k).astype(np.int32) for k in (1, 17, 64)]
        offs = np.concatenate([[0], np.cumsum([len(q) for q in queries])]).astype(np.int64)
        seeds = np.concatenate(queries).astype(np.int32)
        out = torch.empty(len(queries) * n, dtype=torch.float32, device="cuda:0")
        st = gap.gap_ppr_batch(g.handle, offs, seeds, D, 1e-4, 100, out)
        xs = out.view(len(queries), n)
        rows = rng.choice(n, 1 << 17, replace=False)
        for j, q in enumerate(queries):
            assert st[j]["converged"] and st[j]["final_delta"] < 1e-4
            x = xs[j].cpu().numpy().astype(np.float64)
            assert x.min() >= 0 and x.sum() <= 1 + 1e-5
            y = oracle.ppr_rows(in_off, in_idx, outdeg, x, q, rows, D)
            est = n * float(np.abs(y - x[rows]).mean())
            ys = oracle.ppr_rows(in_off, in_idx, outdeg, x, q, np.unique(q).astype(np.int64), D)
            assert est + float(np.abs(ys - x[np.unique(q)]).sum()) < 1e-4, (j, est)
        srv = gap.PprServer(g.handle, max_cols=8, damping=D, tol=1e-4, max_iters=100)
        try:
            one = torch.empty(n, dtype=torch.float32, device="cuda:0")
            info = srv.wait(srv.submit(queries[1], one))
            assert info["iterations"] == st[1]["iterations"]
            assert torch.equal(one, xs[1])
        finally:
            srv.close()
    finally:
        g.close()
