"""Full-size graphs (2^26 vertices, the bench's workloads) in the bench's
launch configuration.  Too large for a serial oracle run, so they are checked
by properties that hold at any size and by the oracle on sampled rows:
  - every score >= (1-d)/n, the FP64 mass matches the scores, mass <= 1;
  - the §2.1 criterion (one more iteration changes the scores by < 1e-4 in
    L1), estimated from 2^18 uniformly sampled rows recomputed one by one by
    the oracle (oracle.pr_rows) from the GPU's scores;
  - FP32 vs the FP64 GPU path: L1 <= 1e-4 (the paper's tolerance)."""
import numpy as np
import pytest

import gapgen
import oracle
from gpu_helpers import D
from paper_1508_03619_gb300 import gap, tuning

pytestmark = pytest.mark.gpu

SAMPLE = 1 << 18


@pytest.mark.parametrize("kind", ["kron26", "urand26"])
def test_full_size_fp32(cuda_device, kind):
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
        x = torch.empty(n, dtype=torch.float32, device="cuda:0")
        o = tuning.pagerank_options()
        gap.gap_pr_run_ex(g.handle, D, 1e-4, 100, o, x)
        status, st = gap.gap_pr_stats(g.handle)
        assert status == gap.GAP_OK and st["converged"] and st["final_delta"] < 1e-4
        assert 5 <= st["iterations"] <= 40
        xs = x.cpu().numpy().astype(np.float64)
        base = (1 - D) / n
        assert xs.min() >= base * (1 - 1e-6)
        assert abs(st["mass"] - xs.sum()) <= 1e-9 and st["mass"] <= 1 + 1e-5
        # sampled §2.1 criterion, rows recomputed by the oracle
        in_off, in_idx = g.export_csr(1)
        outdeg = g.export_outdeg()
        rows = np.random.default_rng(0x5A).choice(n, SAMPLE, replace=False)
        y = oracle.pr_rows(in_off, in_idx, outdeg, xs, rows, D)
        est = n * float(np.abs(y - xs[rows]).mean())
        assert est < 1e-4, est
        del in_off, in_idx
        # FP64 GPU path on the same graph
        o64 = tuning.pagerank_options()
        o64.precision = gap.GAP_PREC_F64
        x64 = torch.empty(n, dtype=torch.float64, device="cuda:0")
        gap.gap_pr_run_ex(g.handle, D, 1e-4, 100, o64, x64)
        status64, st64 = gap.gap_pr_stats(g.handle)
        assert status64 == gap.GAP_OK and abs(st64["iterations"] - st["iterations"]) <= 1
        assert float((x64 - x.double()).abs().sum().item()) <= 1e-4
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
    src, dst = gapgen.chung_lu_device(n, 500_000_000, 2.1, 0x5C)
    g = gap.Graph.from_edges(n, src, dst, symmetrize=False)
    del src, dst
    torch.cuda.empty_cache()
    try:
        in_off, in_idx = g.export_csr(1)
        outdeg = g.export_outdeg()
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
