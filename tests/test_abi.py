"""Host-side checks of the C ABI (no GPU compute): the library builds and loads,
exports every symbol include/*.h declares, its structs match the C layout,
and argument validation rejects bad input before touching the device."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1508_03619_gb300 import gap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_symbols():
    names = set()
    for fn in os.listdir(INCLUDE):
        if fn.endswith(".h"):
            text = open(os.path.join(INCLUDE, fn)).read()
            names |= set(re.findall(r"GAP_API\s+[\w\s\*]*?\b(gap_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = gap.load()
    declared = declared_symbols()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", gap.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (gap_\w+)", out))
    assert declared <= exported, declared - exported
    assert set(gap.EXPORTED) == declared
    for name in declared:
        assert hasattr(lib, name)


def test_struct_layout_matches_c(tmp_path):
    """Every struct the binding shares with C has the same size and field offsets."""
    fields = [("gap_pr_options", gap.gap_pr_options), ("gap_pr_stats_t", gap.gap_pr_stats_t),
              ("gap_batch_tuning", gap.gap_batch_tuning),
              ("gap_ppr_query_info_t", gap.gap_ppr_query_info_t),
              ("gap_ppr_server_info_t", gap.gap_ppr_server_info_t),
              ("gap_cc_stats_t", gap.gap_cc_stats_t),
              ("gap_bfs_stats_t", gap.gap_bfs_stats_t)]
    lines, want = [], []
    for cname, py in fields:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        want.append(ctypes.sizeof(py))
        for f, _ in py._fields_:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
            want.append(getattr(py, f).offset)
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gap.h"\nint main(){'
                   + "".join(lines) + "}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", f"-I{INCLUDE}", str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    assert got == want


def test_status_strings_and_defaults():
    assert gap.status_string(gap.GAP_OK) == "GAP_OK"
    assert gap.status_string(gap.GAP_WARN_NOT_CONVERGED) == "GAP_WARN_NOT_CONVERGED"
    assert gap.status_string(12345) == "GAP_STATUS_UNKNOWN"
    o = gap.gap_pr_options_default()
    assert (o.precision, o.contrib, o.kahan_hubs, o.hub_threshold, o.deterministic, o.loop) == \
        (gap.GAP_PREC_F32, gap.GAP_CONTRIB_F32, 1, 10000, 0, gap.GAP_LOOP_GRAPH)
    assert o.bf16_until_log2_delta == gap.GAP_NO_LADDER
    assert o.algorithm == gap.GAP_ALGO_PULL and o.l2_window == 0


@pytest.mark.parametrize("n,m", [(0, 0), (-1, 0), (2 ** 31, 0)])
def test_create_rejects_bad_sizes(n, m):
    src = np.zeros(max(m, 1), np.int32)
    with pytest.raises(gap.GapError) as e:
        out = ctypes.c_void_p()
        gap._check(gap.load().gap_graph_create_from_edges(n, m, gap._ptr(src), gap._ptr(src), 0,
                                                          None, ctypes.byref(out)), "create")
    assert e.value.status == gap.GAP_ERR_INVALID_ARG
    assert "n =" in str(e.value)


def test_create_rejects_null_arrays():
    out = ctypes.c_void_p()
    s = gap.load().gap_graph_create_from_edges(4, 3, None, None, 0, None, ctypes.byref(out))
    assert s == gap.GAP_ERR_INVALID_ARG
    s = gap.load().gap_graph_create_from_edges(4, 0, None, None, 0, None, None)
    assert s == gap.GAP_ERR_INVALID_ARG


def test_run_rejects_null_graph():
    x = np.zeros(4, np.float32)
    assert gap.load().gap_pr_run(None, 0.85, 1e-4, 10, gap._ptr(x), None) == gap.GAP_ERR_INVALID_ARG
    assert "graph is NULL" in gap.last_error_message()
    st = gap.gap_pr_stats_t()
    assert gap.load().gap_pr_stats(None, ctypes.byref(st)) == gap.GAP_ERR_INVALID_ARG


def test_server_create_rejects_null_graph():
    out = ctypes.c_void_p()
    assert gap.load().gap_ppr_server_create(None, 8, 0, 0.85, 1e-4, 100, ctypes.byref(out)) == \
        gap.GAP_ERR_INVALID_ARG
    assert gap.load().gap_ppr_batch(None, 1, None, None, 0.85, 1e-4, 10, None, None, None) == \
        gap.GAP_ERR_INVALID_ARG


def test_new_entry_points_reject_null_arguments_before_any_device_work():
    lib = gap.load()
    bad = gap.GAP_ERR_INVALID_ARG
    x = np.zeros(4, np.int32)
    assert lib.gap_cc_run(None, gap._ptr(x), None) == bad
    assert lib.gap_cc_stats(None, ctypes.byref(gap.gap_cc_stats_t())) == bad
    assert lib.gap_bfs_run(None, 0, gap._ptr(x), None) == bad
    assert lib.gap_bfs_stats(None, ctypes.byref(gap.gap_bfs_stats_t())) == bad
    assert lib.gap_selftest_barrier_timeout(None, None, None) == bad
    assert lib.gap_graph_save(None, b"/nonexistent/x.gcsc", None) == bad
    assert lib.gap_graph_load(None, 0, 0, None, None) == bad
    assert lib.gap_edge_list_read(None, 0, None) == bad
    assert lib.gap_edge_list_info(None, None, None, None) == bad
    assert lib.gap_edge_list_arrays(None, None, None) == bad
    f = ctypes.c_uint32()
    assert lib.gap_graph_build_flags(None, ctypes.byref(f)) == bad
    lib.gap_edge_list_destroy(None)  # a no-op
    assert gap.last_error_message()


def test_allocator_hook_validation():
    lib = gap.load()
    assert lib.gap_set_allocator(None) == gap.GAP_OK


def test_binding_rejects_wrong_score_buffers():
    """The binding checks tensor/array dtype and length against the graph before
    any device work (a float32 buffer for an FP64 run would be overrun)."""
    class FakeHandle:
        pass
    import paper_1508_03619_gb300.gap as g
    orig = g.gap_graph_info
    g.gap_graph_info = lambda h: (100, 0, 0)
    try:
        with pytest.raises(ValueError, match="float64"):
            g._check_scores(FakeHandle(), np.zeros(100, np.float32), 8, "run")
        with pytest.raises(ValueError, match="100 vertices"):
            g._check_scores(FakeHandle(), np.zeros(99, np.float32), 4, "run")
        with pytest.raises(ValueError, match="float32"):
            g._check_scores(FakeHandle(), np.zeros(100, np.int32), 4, "run")
        g._check_scores(FakeHandle(), np.zeros(100, np.float32), 4, "run")
    finally:
        g.gap_graph_info = orig
