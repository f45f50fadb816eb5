"""Host logic of bench.py for N > 1 replicas, run as two gloo ranks on the CPU:
the job's time is the slowest rank's, its arcs are every rank's, and only rank
0 of the reference arm prints."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, arcs = bench.combine_ranks(10.0 * (rank + 1), 1000 * (rank + 1), dist, "cpu")
        out.put((rank, ms, arcs))
    finally:
        dist.destroy_process_group()


def test_two_replicas_combine_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 20.0, 3000.0), (1, 20.0, 3000.0)]


def test_single_process_keeps_local_figures():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(5.0, 123, None, "cpu") == (5.0, 123)


def test_reference_arm_other_ranks_print_nothing(capsys):
    sys.path.insert(0, ROOT)
    import bench
    argv = sys.argv
    sys.argv = ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"]
    try:
        a = bench.parse()
    finally:
        sys.argv = argv
    bench.run_reference(a, 2, 1)
    assert capsys.readouterr().out == ""
