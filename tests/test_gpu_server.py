"""Continuous-batching PPR server: queries admitted as columns free up give
exactly the result of the same query run alone (column independence), with
host or device output buffers and staggered arrivals."""
import time

import numpy as np
import pytest

import gapgen
from gpu_helpers import D, gpu_graph, oracle_graph
from paper_1508_03619_gb300 import gap

pytestmark = pytest.mark.gpu


def alone(g, seeds, tol=1e-4, iters=100):
    import torch
    out = torch.empty(g.n, dtype=torch.float32, device="cuda:0")
    st = gap.gap_ppr_batch(g.handle, np.array([0, len(seeds)], np.int64), np.asarray(seeds, np.int32), D,
                           tol, iters, out)
    return out.cpu().numpy(), st[0]


def test_server_mix_equals_alone(cuda_device):
    import torch
    n = 1 << 13
    src, dst = gapgen.kron(13, 16, 0x61)
    off, idx = oracle_graph(n, src, dst, True)
    cand = np.flatnonzero(np.diff(off) > 0)
    rng = np.random.default_rng(4)
    g = gpu_graph(n, src, dst, True)
    srv = gap.PprServer(g.handle, max_cols=8, damping=D, tol=1e-4, max_iters=100)
    try:
        assert srv.info()["columns"] == 8
        queries, outs, tickets = [], [], []
        for i in range(24):
            seeds = rng.choice(cand, size=int(rng.integers(1, 65))).astype(np.int32)
            out = np.zeros(n, np.float32) if i % 2 == 0 else torch.zeros(n, dtype=torch.float32, device="cuda:0")
            queries.append(seeds)
            outs.append(out)
            tickets.append(srv.submit(seeds, out))
            if i in (5, 13):
                time.sleep(0.02)  # arrivals while others are on the GPU
        infos = [srv.wait(t) for t in tickets]
        for seeds, out, info in zip(queries, outs, infos):
            got = out if isinstance(out, np.ndarray) else out.cpu().numpy()
            ref, st = alone(g, seeds)
            assert info["iterations"] == st["iterations"] and info["converged"]
            assert np.array_equal(got, ref)
            assert info["latency_ms"] > 0 and 0 <= info["column"] < 8
        s = srv.info()
        assert s["completed"] == 24 and s["waiting"] == 0 and s["steps"] > 0
    finally:
        srv.close()
        g.close()


def test_server_bad_input_and_destroy_with_pending(cuda_device):
    n = 500
    src, dst = gapgen.urand(n, 4000, 0x62)
    g = gpu_graph(n, src, dst)
    srv = gap.PprServer(g.handle, max_cols=4, damping=D, tol=0.0, max_iters=50)
    try:
        with pytest.raises(gap.GapError) as e:
            srv.submit(np.array([n], np.int32), np.zeros(n, np.float32))
        assert e.value.status == gap.GAP_ERR_INVALID_ARG
        outs = [np.zeros(n, np.float32) for _ in range(10)]
        for o in outs:
            srv.submit(np.array([1, 2], np.int32), o)
    finally:
        srv.close()  # abandons what is still queued; must not hang
        g.close()


def test_server_releases_tickets(cuda_device):
    """A ticket reported done (by wait or poll) is released: asking again is an
    error, so a long-running server holds only queries in flight."""
    n = 1000
    src, dst = gapgen.urand(n, 8000, 0x63)
    g = gpu_graph(n, src, dst)
    srv = gap.PprServer(g.handle, max_cols=4, damping=D, tol=1e-4, max_iters=100)
    try:
        t1 = srv.submit(np.array([1, 2], np.int32), np.zeros(n, np.float32))
        t2 = srv.submit(np.array([3], np.int32), np.zeros(n, np.float32))
        assert srv.wait(t1)["converged"]
        with pytest.raises(gap.GapError) as e:
            srv.wait(t1)
        assert e.value.status == gap.GAP_ERR_INVALID_ARG
        info = None
        while info is None:
            info = srv.poll(t2)
            time.sleep(0.001)
        assert info["converged"]
        with pytest.raises(gap.GapError):
            srv.poll(t2)
        assert not srv._keep
    finally:
        srv.close()
        g.close()


def test_server_width_changes_keep_results(cuda_device):
    """A 16-column server runs a 4-column engine while the load is light, moves
    the running columns to the 16-column engine when a burst queues far beyond
    the narrow width, and back once it drained: every query's scores and
    iteration count equal the same query run alone, bit for bit."""
    import torch
    n = 1 << 12
    src, dst = gapgen.kron(12, 16, 0x64)
    off, idx = oracle_graph(n, src, dst, True)
    cand = np.flatnonzero(np.diff(off) > 0)
    rng = np.random.default_rng(6)
    g = gpu_graph(n, src, dst, True)
    srv = gap.PprServer(g.handle, max_cols=16, damping=D, tol=1e-6, max_iters=100)
    try:
        i0 = srv.info()
        assert i0["columns"] == 16 and i0["narrow_columns"] == 4 and i0["narrow"] == 1
        queries, outs, tickets = [], [], []

        def submit(k):
            for _ in range(k):
                seeds = rng.choice(cand, size=int(rng.integers(1, 20))).astype(np.int32)
                out = torch.zeros(n, dtype=torch.float32, device="cuda:0")
                queries.append(seeds)
                outs.append(out)
                tickets.append(srv.submit(seeds, out))

        submit(2)            # narrow engine
        time.sleep(0.01)
        submit(30)           # a queue far beyond twice the narrow width: the running queries move up
        infos = [srv.wait(t) for t in tickets]
        submit(2)            # drained: back to the narrow engine
        infos += [srv.wait(t) for t in tickets[32:]]
        s = srv.info()
        assert s["switches"] >= 2 and s["completed"] == 34 and s["narrow"] == 1
        for seeds, out, info in zip(queries, outs, infos):
            ref, st = alone(g, seeds, tol=1e-6)
            assert info["iterations"] == st["iterations"] and info["converged"]
            assert np.array_equal(out.cpu().numpy(), ref)
    finally:
        srv.close()
        g.close()


class BudgetAllocator:
    """Scratch blocks from torch's caching allocator within a byte budget the
    test moves while the server runs: a block that would pass the budget is
    refused (NULL), which the library sees as out of memory."""

    def __init__(self):
        import threading

        import torch
        self.torch = torch
        self.lock = threading.Lock()
        self.budget = None
        self.used = 0
        self.live = {}
        self.refused = 0
        self._a = gap.gap_allocator.ALLOC(self._alloc)
        self._f = gap.gap_allocator.FREE(self._free)
        self.c = gap.gap_allocator(self._a, self._f, None)

    def _alloc(self, nbytes, stream, ctx):
        with self.lock:
            if self.budget is not None and self.used + nbytes > self.budget:
                self.refused += 1
                return None
            t = self.torch.empty(nbytes, dtype=self.torch.uint8, device="cuda")
            self.live[t.data_ptr()] = (t, nbytes)
            self.used += nbytes
            return t.data_ptr()

    def _free(self, ptr, nbytes, stream, ctx):
        with self.lock:
            _, nb = self.live.pop(ptr)
            self.used -= nb


def test_server_admission_by_free_memory(cuda_device):
    """The wide engine is allocated only when the load needs it and the memory
    is there at that moment.  With no room for it, a burst far beyond the
    narrow width is served by the narrow engine alone (the growth is refused);
    once room appears, the next burst moves up into a newly allocated wide
    engine; 2 s after the load is gone the wide engine is released and its
    memory returned.  Every query equals the same query run alone bit for bit,
    and a sample matches the oracle within the FP32 bars."""
    import torch

    import oracle
    from gpu_helpers import FP32_L1, FP32_REL
    n = 1 << 12
    src, dst = gapgen.kron(12, 16, 0x65)
    off, idx = oracle_graph(n, src, dst, True)
    cand = np.flatnonzero(np.diff(off) > 0)
    rng = np.random.default_rng(7)
    g = gpu_graph(n, src, dst, True)
    alloc = BudgetAllocator()
    queries, outs, infos = [], [], []
    gap.gap_set_allocator(alloc.c)
    try:
        srv = gap.PprServer(g.handle, max_cols=16, damping=D, tol=1e-4, max_iters=100)
        try:
            i0 = srv.info()
            assert i0["narrow"] == 1 and i0["narrow_columns"] == 4 and i0["wide_ready"] == 0
            narrow_bytes = alloc.used

            def burst(k):
                tickets = []
                for _ in range(k):
                    seeds = rng.choice(cand, size=int(rng.integers(1, 20))).astype(np.int32)
                    out = torch.zeros(n, dtype=torch.float32, device="cuda:0")
                    queries.append(seeds)
                    outs.append(out)
                    tickets.append(srv.submit(seeds, out))
                infos.extend(srv.wait(t) for t in tickets)

            alloc.budget = alloc.used  # no room for the wide engine
            burst(30)
            s1 = srv.info()
            assert s1["completed"] == 30 and s1["grow_refused"] >= 1
            assert s1["wide_ready"] == 0 and s1["wide_allocs"] == 0 and s1["switches"] == 0
            assert alloc.refused >= 1 and alloc.used == narrow_bytes
            alloc.budget = None  # room again
            time.sleep(0.06)
            burst(30)
            s2 = srv.info()
            assert s2["completed"] == 60 and s2["wide_allocs"] == 1 and s2["switches"] >= 1
            assert alloc.used > narrow_bytes or s2["wide_releases"] == 1
            time.sleep(3.0)  # idle: the unused wide engine goes back
            s3 = srv.info()
            assert s3["wide_ready"] == 0 and s3["wide_releases"] == 1 and s3["narrow"] == 1
            assert alloc.used == narrow_bytes
        finally:
            srv.close()
    finally:
        gap.gap_set_allocator(None)
    try:
        for j, (seeds, out, info) in enumerate(zip(queries, outs, infos)):
            ref, st = alone(g, seeds)
            assert info["iterations"] == st["iterations"] and info["converged"]
            assert np.array_equal(out.cpu().numpy(), ref)
            if j % 10 == 0:  # unreachable vertices score exactly 0 on both sides
                xo, _, _ = oracle.ppr(off, idx, seeds, D, 0.0, info["iterations"])
                x = out.cpu().numpy().astype(np.float64)
                reach = xo > 0
                assert np.all(x[~reach] == 0.0)
                assert np.abs(x - xo).sum() <= FP32_L1
                big = xo > 1e-6  # the bar the batch PPR tests apply
                assert np.max(np.abs(x[big] - xo[big]) / xo[big]) <= FP32_REL
    finally:
        g.close()
