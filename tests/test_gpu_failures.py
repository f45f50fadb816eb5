"""Failure detection without a GPU fault.

Faults are injected on the host: an allocator callback that runs out after a
few blocks (every entry point must return GAP_ERR_OOM, free what it took and
leave the library usable), and one that returns blocks off the 256-byte
alignment the kernels need (GAP_ERR_INVALID_ARG, no kernel runs on them).
On the device, the grid barrier's bounded wait is made to run out by design
(a barrier that counts one block more than was launched): it must report
GAP_ERR_TIMEOUT within its bound, and the context must stay usable."""
import numpy as np
import pytest

import gapgen
import oracle
from gpu_helpers import D, assert_fp32_parity, gpu_graph
from paper_1508_03619_gb300 import gap

pytestmark = pytest.mark.gpu


class TorchAllocator:
    """Scratch blocks from torch's caching allocator (on the current stream,
    which the library calls share), with fault injection: fail after
    `budget` blocks, or hand out blocks `shift` bytes past the aligned start."""

    def __init__(self, budget=None, shift=0):
        import torch
        self.torch = torch
        self.budget = budget
        self.shift = shift
        self.live = {}
        self.allocs = self.frees = self.refused = 0
        self._a = gap.gap_allocator.ALLOC(self._alloc)
        self._f = gap.gap_allocator.FREE(self._free)
        self.c = gap.gap_allocator(self._a, self._f, None)

    def _alloc(self, nbytes, stream, ctx):
        if self.budget is not None and self.allocs >= self.budget:
            self.refused += 1
            return None
        t = self.torch.empty(nbytes + self.shift + 256, dtype=self.torch.uint8, device="cuda")
        p = t.data_ptr() + self.shift
        self.live[p] = t
        self.allocs += 1
        return p

    def _free(self, ptr, nbytes, stream, ctx):
        self.live.pop(ptr)
        self.frees += 1

    def __enter__(self):
        gap.gap_set_allocator(self.c)
        return self

    def __exit__(self, *exc):
        gap.gap_set_allocator(None)


def _graph():
    n = 1 << 12
    s, d = gapgen.kron(12, 8, seed=0xF1)
    return n, s, d


def test_custom_allocator_runs_every_entry_point(cuda_device):
    import torch
    n, s, d = _graph()
    off, idx = oracle.build_csr(n, s, d, symmetrize=True)
    with gpu_graph(n, s, d, symmetrize=True) as g:
        with TorchAllocator() as al:
            x = torch.empty(n, dtype=torch.float32, device="cuda")
            gap.gap_pr_run(g.handle, D, 0.0, 20, x)
            gap.gap_pr_stats(g.handle)
            lab = torch.empty(n, dtype=torch.int32, device="cuda")
            gap.gap_cc_run(g.handle, lab)
            gap.gap_cc_stats(g.handle)
            par = torch.empty(n, dtype=torch.int32, device="cuda")
            gap.gap_bfs_run(g.handle, 3, par)
            gap.gap_bfs_stats(g.handle)
            torch.cuda.synchronize()
        assert al.allocs > 5 and al.allocs == al.frees and not al.live
        xo, _, _ = oracle.pagerank(off, idx, D, 0.0, 20)
        assert_fp32_parity(x.cpu().numpy().astype(np.float64), xo)
        assert np.array_equal(lab.cpu().numpy(), oracle.cc(off, idx))
        assert oracle.bfs_verify(off, idx, 3, par.cpu().numpy())


@pytest.mark.parametrize("which,budget", [("pr", 0), ("pr", 1), ("pr", 3), ("pr", 8),
                                          ("cc", 0), ("cc", 1), ("bfs", 0), ("bfs", 3), ("bfs", 8)])
def test_allocator_running_out_gives_oom_and_frees_what_it_took(cuda_device, which, budget):
    """Each budget is below the blocks that entry point takes (a PageRank trial
    about 20, CC with host labels 2, BFS 9), so the run fails part-way."""
    import torch
    n, s, d = _graph()
    with gpu_graph(n, s, d, symmetrize=True) as g:
        run = {
            "pr": lambda: gap.gap_pr_run(g.handle, D, 1e-4, 100, torch.empty(n, dtype=torch.float32, device="cuda")),
            "cc": lambda: gap.gap_cc_run(g.handle, np.empty(n, np.int32)),  # host labels need device scratch
            "bfs": lambda: gap.gap_bfs_run(g.handle, 0, torch.empty(n, dtype=torch.int32, device="cuda")),
        }[which]
        with TorchAllocator(budget=budget) as al:
            with pytest.raises(gap.GapError) as ei:
                run()
            torch.cuda.synchronize()
        assert ei.value.status == gap.GAP_ERR_OOM, ei.value
        assert al.refused >= 1 and al.allocs == al.frees and not al.live
        # the default allocator is back and the library works
        x = torch.empty(n, dtype=torch.float32, device="cuda")
        assert gap.gap_pr_run(g.handle, D, 1e-4, 100, x) == gap.GAP_OK
        status, st = gap.gap_pr_stats(g.handle)
        assert status == gap.GAP_OK and st["converged"]


def test_misaligned_allocator_is_refused(cuda_device):
    import torch
    n, s, d = _graph()
    with gpu_graph(n, s, d, symmetrize=True) as g:
        with TorchAllocator(shift=16) as al:
            with pytest.raises(gap.GapError) as ei:
                gap.gap_pr_run(g.handle, D, 1e-4, 100, torch.empty(n, dtype=torch.float32, device="cuda"))
            torch.cuda.synchronize()
        assert ei.value.status == gap.GAP_ERR_INVALID_ARG and "256" in str(ei.value)
        assert al.allocs == al.frees and not al.live


def test_grid_barrier_wait_runs_out_and_reports_timeout(cuda_device):
    import torch
    for _ in range(2):
        observed, ms = gap.gap_selftest_barrier_timeout()
        assert observed == gap.GAP_ERR_TIMEOUT
        assert 45.0 <= ms < 2000.0  # gave up after its 50 ms bound, not at the 2 s production bound
    # the context is intact: a batch (the kernel that uses this barrier) still runs
    n, s, d = _graph()
    off, idx = oracle.build_csr(n, s, d, symmetrize=True)
    with gpu_graph(n, s, d, symmetrize=True) as g:
        x = [torch.empty(n, dtype=torch.float32, device="cuda")]
        st = gap.gap_pr_run_batch([g.handle], x, D, 0.0, 20)
        xo, _, _ = oracle.pagerank(off, idx, D, 0.0, 20)
        assert st[0]["iterations"] == 20
        assert_fp32_parity(x[0].cpu().numpy().astype(np.float64), xo)


def test_worklist_checks_pass_on_real_trials_and_change_nothing(cuda_device):
    """options.check_worklists validates the trial's device-built work lists
    (bin list, split points, packed small-row arcs, hub chunk tables) before the
    iterations: on real graphs -- whole rows, L2 segments, hubs -- every check
    passes and the scores equal an unchecked run bit for bit."""
    import gapgen
    from gpu_helpers import oracle_graph, run_gpu, seg_bytes_for
    from test_gpu_pagerank import threshold_graph
    n, src, dst = threshold_graph()
    cases = [(n, src, dst, False), (1 << 14, *gapgen.kron(14, 16, 0x14), True)]
    for n, src, dst, sym in cases:
        g = gpu_graph(n, src, dst, sym)
        try:
            for seg in (0, seg_bytes_for(n)):
                x0, st0, _ = run_gpu(g, 0.0, 6, segment_bytes=seg)
                x1, st1, s1 = run_gpu(g, 0.0, 6, segment_bytes=seg, check_worklists=1)
                assert s1 == gap.GAP_OK and np.array_equal(x0, x1)
                assert st1["segments"] == st0["segments"]
            if n == cases[0][0]:
                assert st1["bins"][6]["rows"] > 0  # hub chunk tables were checked too
        finally:
            g.close()


def test_worklist_validators_report_broken_lists(cuda_device):
    """The validators report each kind of broken list (fed to them directly; no
    pull kernel reads these lists): an entry outside [0, n), a vertex listed
    twice, a row in the wrong bin, a packed source outside its segment, a
    packed row outside [0, n) or not a small row; valid lists pass."""
    import torch

    import gapgen
    from gpu_helpers import oracle_graph
    n = 1024
    src, dst = gapgen.kron(10, 16, 0x15)
    off, idx = oracle_graph(n, dst, src, True)  # a CSC (symmetric anyway)
    deg = np.diff(off)
    hi = np.array([64, 64, 64, 64, 256, 512], np.int64)  # bins 0 (<= 64), 4 (<= 256), 5 (<= 512), 6
    bins = np.searchsorted(hi, deg, side="left")         # first bin whose bound is not below the degree
    order = np.argsort(bins, kind="stable").astype(np.int32)
    bin_start = np.searchsorted(bins[order], np.arange(8)).astype(np.int64)
    dev = torch.device("cuda:0")
    t_off = torch.from_numpy(off).to(dev)

    def check_list(lst):
        return gap.gap_selftest_check_bin_list(t_off, torch.from_numpy(lst).to(dev), bin_start, hi)

    assert check_list(order) == (0, 0)
    bad = order.copy()
    bad[5] = n + 7
    assert check_list(bad) == (1, 5)
    bad = order.copy()
    bad[5] = bad[6]                # positions 5 and 6 share bin 0
    assert check_list(bad)[0] == 2
    big = int(np.flatnonzero(bins[order] == bins[order][-1])[0])
    bad = order.copy()
    bad[0], bad[big] = bad[big], bad[0]   # a bin-0 row and a top-bin row trade places
    assert check_list(bad)[0] == 3

    # packed small-row arcs, two segments of 512 sources
    wbits, small_max = 9, 64
    rows, srcs = [], []
    for sg in range(2):
        for v in range(n):
            if deg[v] <= small_max:
                for u in idx[off[v]:off[v + 1]]:
                    if u >> wbits == sg:
                        rows.append(v)
                        srcs.append(u)
    seg_end = np.array([sum(1 for u in srcs if u >> wbits == 0), len(srcs)], np.int64)

    def check_packed(p, r):
        return gap.gap_selftest_check_packed(t_off, torch.tensor(p, dtype=torch.int32, device=dev),
                                             torch.tensor(r, dtype=torch.int32, device=dev),
                                             torch.from_numpy(seg_end).to(dev), wbits, small_max)

    assert check_packed(srcs, rows) == (0, 0)
    p = list(srcs)
    p[0] = 600                     # a segment-1 source among segment 0's arcs
    assert check_packed(p, rows) == (6, 0)
    r = list(rows)
    r[1] = n + 5
    assert check_packed(srcs, r) == (7, 1)
    r = list(rows)
    r[2] = int(np.flatnonzero(deg > small_max)[0])  # a row that is not small
    assert check_packed(srcs, r) == (7, 2)
