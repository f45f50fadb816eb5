"""Thin ctypes binding of libgap.so (include/gap.h), same names as the C ABI.

Argument marshalling only: every step of PageRank runs in the library's CUDA
kernels.  Array arguments may be torch tensors (host or CUDA) or numpy
arrays; their raw addresses are passed through.  ``stream`` defaults to
torch's current CUDA stream.  If the library is missing this module raises —
there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

GAP_OK = 0
GAP_ERR_INVALID_ARG = -1
GAP_ERR_OOM = -2
GAP_ERR_CUDA = -3
GAP_ERR_TIMEOUT = -4
GAP_ERR_BOUNDS = -5
GAP_ERR_UNSUPPORTED = -6
GAP_WARN_NOT_CONVERGED = 1

GAP_SYMMETRIZE = 0x1
GAP_DEDUP = 0x2
GAP_DROP_SELF_LOOPS = 0x4
GAP_INPUT_ON_DEVICE = 0x8

GAP_FMT_AUTO = 0
GAP_FMT_EDGE_LIST = 1
GAP_FMT_MATRIX_MARKET = 2
GAP_FMT_METIS = 3
GAP_FMT_SERIALIZED = 4

GAP_PREC_F32 = 0
GAP_PREC_F64 = 1
GAP_CONTRIB_F32 = 0
GAP_CONTRIB_BF16 = 1
GAP_LOOP_GRAPH = 0
GAP_LOOP_HOST = 1
GAP_NO_LADDER = -(2 ** 31)
GAP_PR_HIST = 256
GAP_PR_PHASES = 13
GAP_PR_BINS = 7
PHASE_NAMES = ("bin", "init", "pull0", "pull1", "pull2", "pull3", "pull4", "pull5", "pull6",
               "hub_fixup", "finalize", "output", "prep")
PULL_PHASES = PHASE_NAMES[2:9]

# every symbol include/gap.h declares (checked by the ABI test)
EXPORTED = (
    "gap_status_string", "gap_last_error_message", "gap_version", "gap_set_allocator",
    "gap_graph_create_from_edges", "gap_graph_create", "gap_graph_create_csc", "gap_graph_info",
    "gap_graph_export_csr",
    "gap_graph_export_outdeg", "gap_graph_destroy", "gap_pr_run", "gap_pr_run_f64",
    "gap_pr_options_default", "gap_pr_run_ex", "gap_pr_stats", "gap_pr_run_noalloc",
    "gap_batch_tuning_default", "gap_pr_run_batch", "gap_pr_run_batch_ex", "gap_ppr_batch",
    "gap_ppr_server_create", "gap_ppr_submit", "gap_ppr_poll", "gap_ppr_wait",
    "gap_ppr_server_info", "gap_ppr_server_info_ex", "gap_ppr_server_destroy",
    "gap_edge_list_read", "gap_edge_list_info", "gap_edge_list_arrays", "gap_edge_list_destroy",
    "gap_graph_load", "gap_graph_save", "gap_graph_build_flags",
    "gap_cc_run", "gap_cc_stats", "gap_bfs_run", "gap_bfs_stats", "gap_selftest_barrier_timeout",
    "gap_selftest_check_bin_list", "gap_selftest_check_packed",
)
GAP_NOALLOC_MAX_VERTICES = 1 << 20
GAP_BATCH_MAX_GRAPHS = 65536
GAP_ALGO_PULL = 0
GAP_ALGO_BINNED = 1
GAP_ALGO_DELTA = 2


class gap_batch_tuning(ctypes.Structure):
    _fields_ = [("heavy_min_degree", ctypes.c_int32), ("chunk_arcs", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gap_pr_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_uint32), ("contrib", ctypes.c_uint32),
                ("bf16_until_log2_delta", ctypes.c_int32), ("kahan_hubs", ctypes.c_uint32),
                ("hub_threshold", ctypes.c_int64), ("deterministic", ctypes.c_uint32),
                ("l2_window", ctypes.c_uint32), ("loop", ctypes.c_uint32),
                ("timing", ctypes.c_uint32), ("segment_bytes", ctypes.c_int64),
                ("small_max_degree", ctypes.c_int64), ("algorithm", ctypes.c_uint32),
                ("group_lanes", ctypes.c_uint32), ("group_max_degree", ctypes.c_int64),
                ("cta_max_degree", ctypes.c_int64), ("hub_chunk_arcs", ctypes.c_int64),
                ("check_worklists", ctypes.c_uint32), ("reserved1", ctypes.c_uint32)]


class gap_pr_stats_t(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("final_delta", ctypes.c_double), ("mass", ctypes.c_double),
                ("bf16_iters", ctypes.c_int32), ("device_error", ctypes.c_int32),
                ("delta_hist", ctypes.c_double * GAP_PR_HIST),
                ("bin_rows", ctypes.c_int64 * GAP_PR_BINS), ("bin_arcs", ctypes.c_int64 * GAP_PR_BINS),
                ("bin_max_degree", ctypes.c_int64 * GAP_PR_BINS),
                ("bin_lanes", ctypes.c_int32 * GAP_PR_BINS),
                ("bin_segmented", ctypes.c_int32 * GAP_PR_BINS), ("segments", ctypes.c_int32),
                ("phase_ms", ctypes.c_double * GAP_PR_PHASES),
                ("phase_launches", ctypes.c_int32 * GAP_PR_PHASES),
                ("kernel_launches", ctypes.c_int32), ("pad0", ctypes.c_int32),
                ("l2_window_bytes", ctypes.c_int64), ("arcs_traversed", ctypes.c_int64),
                ("sparse_rounds", ctypes.c_int32), ("pad1", ctypes.c_int32)]

    def to_dict(self):
        k = min(self.iterations, GAP_PR_HIST)
        return {"iterations": self.iterations, "converged": bool(self.converged),
                "final_delta": self.final_delta, "mass": self.mass, "bf16_iters": self.bf16_iters,
                "device_error": self.device_error, "deltas": list(self.delta_hist[:k]),
                "bins": [{"rows": self.bin_rows[q], "arcs": self.bin_arcs[q],
                          "max_degree": self.bin_max_degree[q], "lanes": self.bin_lanes[q],
                          "segmented": bool(self.bin_segmented[q])} for q in range(GAP_PR_BINS)],
                "segments": self.segments,
                "phase_ms": dict(zip(PHASE_NAMES, self.phase_ms)),
                "phase_launches": dict(zip(PHASE_NAMES, self.phase_launches)),
                "kernel_launches": self.kernel_launches,
                "l2_window_bytes": self.l2_window_bytes, "arcs_traversed": self.arcs_traversed,
                "sparse_rounds": self.sparse_rounds}


class gap_ppr_query_info_t(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("final_delta", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("column", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def to_dict(self):
        return {"iterations": self.iterations, "converged": bool(self.converged),
                "final_delta": self.final_delta, "latency_ms": self.latency_ms, "column": self.column}


class gap_ppr_server_info_t(ctypes.Structure):
    _fields_ = [("columns", ctypes.c_int32), ("narrow_columns", ctypes.c_int32), ("narrow", ctypes.c_int32),
                ("live", ctypes.c_int32), ("waiting", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("switches", ctypes.c_int64), ("completed", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("wide_ready", ctypes.c_int32), ("pad2", ctypes.c_int32), ("grow_refused", ctypes.c_int64),
                ("wide_allocs", ctypes.c_int64), ("wide_releases", ctypes.c_int64)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("pad")}


class gap_cc_stats_t(ctypes.Structure):
    _fields_ = [("components", ctypes.c_int64), ("giant_size", ctypes.c_int64),
                ("giant_label", ctypes.c_int32), ("sample_rounds", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32), ("device_error", ctypes.c_int32)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gap_bfs_stats_t(ctypes.Structure):
    _fields_ = [("reached", ctypes.c_int64), ("levels", ctypes.c_int32),
                ("top_down_steps", ctypes.c_int32), ("bottom_up_steps", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int32)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GapError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {status_string(status)} ({status}): {msg}")
        self.status = status


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libgap.so (building it in-tree first if asked).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"{_build.LIB} is not built")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    i64, i32, u32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p
    st = ctypes.c_int32
    sig = {
        "gap_status_string": ([st], ctypes.c_char_p),
        "gap_last_error_message": ([], ctypes.c_char_p),
        "gap_version": ([], i32),
        "gap_set_allocator": ([vp], st),
        "gap_graph_create_from_edges": ([i64, i64, vp, vp, u32, vp, ctypes.POINTER(vp)], st),
        "gap_graph_create": ([i64, i64, vp, vp, u32, vp, ctypes.POINTER(vp)], st),
        "gap_graph_create_csc": ([i64, i64, vp, vp, vp, ctypes.POINTER(vp)], st),
        "gap_graph_info": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)], st),
        "gap_graph_export_csr": ([vp, ctypes.c_int, vp, vp, vp], st),
        "gap_graph_export_outdeg": ([vp, vp, vp], st),
        "gap_graph_destroy": ([vp], None),
        "gap_pr_run": ([vp, dbl, dbl, i32, vp, vp], st),
        "gap_pr_run_f64": ([vp, dbl, dbl, i32, vp, vp], st),
        "gap_pr_options_default": ([ctypes.POINTER(gap_pr_options)], None),
        "gap_pr_run_ex": ([vp, dbl, dbl, i32, ctypes.POINTER(gap_pr_options), vp, vp], st),
        "gap_pr_stats": ([vp, ctypes.POINTER(gap_pr_stats_t)], st),
        "gap_pr_run_noalloc": ([vp, dbl, dbl, i32, vp, vp], st),
        "gap_batch_tuning_default": ([ctypes.POINTER(gap_batch_tuning)], None),
        "gap_pr_run_batch": ([vp, i32, dbl, dbl, i32, vp, vp, vp], st),
        "gap_pr_run_batch_ex": ([vp, i32, dbl, dbl, i32, ctypes.POINTER(gap_batch_tuning), vp, vp, vp],
                                st),
        "gap_ppr_batch": ([vp, i32, vp, vp, dbl, dbl, i32, vp, vp, vp], st),
        "gap_ppr_server_create": ([vp, i32, ctypes.c_size_t, dbl, dbl, i32, ctypes.POINTER(vp)], st),
        "gap_ppr_submit": ([vp, vp, i32, vp, ctypes.POINTER(i64)], st),
        "gap_ppr_poll": ([vp, i64, ctypes.POINTER(i32), ctypes.POINTER(gap_ppr_query_info_t)], st),
        "gap_ppr_wait": ([vp, i64, ctypes.POINTER(gap_ppr_query_info_t)], st),
        "gap_ppr_server_info": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i64),
                                 ctypes.POINTER(i32)], st),
        "gap_ppr_server_info_ex": ([vp, ctypes.POINTER(gap_ppr_server_info_t)], st),
        "gap_ppr_server_destroy": ([vp], None),
        "gap_edge_list_read": ([ctypes.c_char_p, i32, ctypes.POINTER(vp)], st),
        "gap_edge_list_info": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(u32)], st),
        "gap_edge_list_arrays": ([vp, ctypes.POINTER(vp), ctypes.POINTER(vp)], st),
        "gap_edge_list_destroy": ([vp], None),
        "gap_graph_load": ([ctypes.c_char_p, i32, u32, vp, ctypes.POINTER(vp)], st),
        "gap_graph_save": ([vp, ctypes.c_char_p, vp], st),
        "gap_graph_build_flags": ([vp, ctypes.POINTER(u32)], st),
        "gap_cc_run": ([vp, vp, vp], st),
        "gap_cc_stats": ([vp, ctypes.POINTER(gap_cc_stats_t)], st),
        "gap_bfs_run": ([vp, i32, vp, vp], st),
        "gap_bfs_stats": ([vp, ctypes.POINTER(gap_bfs_stats_t)], st),
        "gap_selftest_barrier_timeout": ([ctypes.POINTER(i32), ctypes.POINTER(dbl), vp], st),
        "gap_selftest_check_bin_list": ([i64, vp, vp, vp, vp, ctypes.POINTER(i32), ctypes.POINTER(i64), vp], st),
        "gap_selftest_check_packed": ([i64, vp, vp, vp, vp, i32, i32, i64, ctypes.POINTER(i32),
                                       ctypes.POINTER(i64), vp], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def status_string(s: int) -> str:
    return load().gap_status_string(s).decode()


def last_error_message() -> str:
    return load().gap_last_error_message().decode()


def _check(status: int, where: str, ok=(GAP_OK,)):
    if status not in ok:
        raise GapError(status, where, last_error_message())
    return status


def _ptr(a):
    """Raw address of a torch tensor / numpy array / int / None."""
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"cannot pass {type(a)} as a pointer")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _on_device(a) -> bool:
    return bool(getattr(a, "is_cuda", False))


# ------------------------------------------------------------------ graph ---

def gap_graph_create_from_edges(n: int, src, dst, flags: int, stream=None):
    if len(src) != len(dst):
        raise ValueError("src and dst differ in length")
    if _on_device(src) != _on_device(dst):
        raise ValueError("src and dst must both be host or both device arrays")
    if _on_device(src):
        flags |= GAP_INPUT_ON_DEVICE
    out = ctypes.c_void_p()
    _check(load().gap_graph_create_from_edges(n, len(src), _ptr(src), _ptr(dst), flags,
                                              _stream(stream), ctypes.byref(out)),
           "gap_graph_create_from_edges")
    return out


def gap_graph_create_csc(n: int, in_offsets, in_idx, stream=None):
    """A graph from a prebuilt in-direction CSR (host or device arrays; int64
    offsets of n+1 entries, int32 sources); copied and checked, not rebuilt."""
    for a, size, count, name in ((in_offsets, 8, n + 1, "in_offsets"), (in_idx, 4, None, "in_idx")):
        esz = a.element_size() if hasattr(a, "element_size") else a.itemsize
        cnt = a.numel() if hasattr(a, "numel") else a.size
        if esz != size or (count is not None and cnt != count):
            raise ValueError(f"gap_graph_create_csc: {name} needs {size}-byte integers"
                             + (f", {count} of them" if count is not None else ""))
    m = int(in_idx.numel() if hasattr(in_idx, "numel") else in_idx.size)
    out = ctypes.c_void_p()
    _check(load().gap_graph_create_csc(n, m, _ptr(in_offsets), _ptr(in_idx), _stream(stream), ctypes.byref(out)),
           "gap_graph_create_csc")
    return out


def gap_graph_create(n: int, row_offsets, col_idx, flags: int, stream=None):
    if _on_device(row_offsets):
        flags |= GAP_INPUT_ON_DEVICE
    out = ctypes.c_void_p()
    _check(load().gap_graph_create(n, len(col_idx), _ptr(row_offsets), _ptr(col_idx), flags,
                                   _stream(stream), ctypes.byref(out)), "gap_graph_create")
    return out


def gap_graph_info(h):
    n, m, nd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().gap_graph_info(h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nd)),
           "gap_graph_info")
    return n.value, m.value, nd.value


def gap_graph_export_csr(h, direction: int, offsets, idx, stream=None):
    _check(load().gap_graph_export_csr(h, direction, _ptr(offsets), _ptr(idx), _stream(stream)),
           "gap_graph_export_csr")


def gap_graph_export_outdeg(h, outdeg, stream=None):
    _check(load().gap_graph_export_outdeg(h, _ptr(outdeg), _stream(stream)),
           "gap_graph_export_outdeg")


def gap_graph_destroy(h):
    if h is not None and h.value:
        load().gap_graph_destroy(h)


# ------------------------------------------------------------ graph files ---

def _path(path) -> bytes:
    return os.fsencode(path)


def gap_edge_list_read(path, fmt: int = GAP_FMT_AUTO):
    """Parse a text graph file on the host.  Returns (n, src, dst, implied_flags)
    with src/dst int32 numpy arrays (copies; the library's list is released)."""
    import numpy as np
    lib = load()
    h = ctypes.c_void_p()
    _check(lib.gap_edge_list_read(_path(path), fmt, ctypes.byref(h)), "gap_edge_list_read")
    try:
        n, m, fl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint32()
        _check(lib.gap_edge_list_info(h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(fl)), "gap_edge_list_info")
        ps, pd = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib.gap_edge_list_arrays(h, ctypes.byref(ps), ctypes.byref(pd)), "gap_edge_list_arrays")
        src = np.empty(m.value, dtype=np.int32)
        dst = np.empty(m.value, dtype=np.int32)
        if m.value:
            ctypes.memmove(src.ctypes.data, ps.value, 4 * m.value)
            ctypes.memmove(dst.ctypes.data, pd.value, 4 * m.value)
        return n.value, src, dst, fl.value
    finally:
        lib.gap_edge_list_destroy(h)


def gap_graph_load(path, fmt: int = GAP_FMT_AUTO, flags: int = 0, stream=None):
    out = ctypes.c_void_p()
    _check(load().gap_graph_load(_path(path), fmt, flags, _stream(stream), ctypes.byref(out)), "gap_graph_load")
    return out


def gap_graph_save(h, path, stream=None):
    _check(load().gap_graph_save(h, _path(path), _stream(stream)), "gap_graph_save")


def gap_graph_build_flags(h) -> int:
    f = ctypes.c_uint32()
    _check(load().gap_graph_build_flags(h, ctypes.byref(f)), "gap_graph_build_flags")
    return f.value


# --------------------------------------------------------------- PageRank ---

def gap_pr_options_default() -> gap_pr_options:
    o = gap_pr_options()
    load().gap_pr_options_default(ctypes.byref(o))
    return o


def _check_scores(h, scores, itemsize: int, where: str, n=None):
    """The C ABI cannot see buffer sizes: for tensors and arrays, check here that
    the output holds n elements of the run's precision (raw integer addresses
    are passed through unchecked).  `n` may be given when the caller knows it."""
    if scores is None or isinstance(scores, int):
        return
    if n is None:
        n = gap_graph_info(h)[0]
    if hasattr(scores, "element_size"):
        size, numel = scores.element_size(), scores.numel()
        floating = scores.is_floating_point()
    elif hasattr(scores, "itemsize"):
        size, numel = scores.itemsize, scores.size
        floating = scores.dtype.kind == "f"
    else:
        return
    if not floating or size != itemsize:
        raise ValueError(f"{where}: scores must be float{8 * itemsize}")
    if numel < n:
        raise ValueError(f"{where}: scores holds {numel} elements, the graph has {n} vertices")


def gap_pr_run(h, damping: float, tol: float, max_iters: int, scores, stream=None):
    _check_scores(h, scores, 4, "gap_pr_run")
    return _check(load().gap_pr_run(h, damping, tol, max_iters, _ptr(scores), _stream(stream)),
                  "gap_pr_run")


def gap_pr_run_f64(h, damping: float, tol: float, max_iters: int, scores, stream=None):
    _check_scores(h, scores, 8, "gap_pr_run_f64")
    return _check(load().gap_pr_run_f64(h, damping, tol, max_iters, _ptr(scores), _stream(stream)),
                  "gap_pr_run_f64")


def gap_pr_run_ex(h, damping: float, tol: float, max_iters: int, options: gap_pr_options, scores,
                  stream=None):
    _check_scores(h, scores, 8 if options.precision == GAP_PREC_F64 else 4, "gap_pr_run_ex")
    return _check(load().gap_pr_run_ex(h, damping, tol, max_iters, ctypes.byref(options),
                                       _ptr(scores), _stream(stream)), "gap_pr_run_ex")


def gap_pr_run_noalloc(h, damping: float, tol: float, max_iters: int, scores, stream=None):
    """No-allocation FP32 trial (scratch in a static device array); see gap.h."""
    _check_scores(h, scores, 4, "gap_pr_run_noalloc")
    return _check(load().gap_pr_run_noalloc(h, damping, tol, max_iters, _ptr(scores),
                                            _stream(stream)), "gap_pr_run_noalloc")


def gap_batch_tuning_default():
    t = gap_batch_tuning()
    load().gap_batch_tuning_default(ctypes.byref(t))
    return t


def gap_pr_run_batch(handles, scores, damping: float, tol: float, max_iters: int, stats=True,
                     stream=None, tuning=None):
    """PageRank on len(handles) graphs in one persistent launch (see gap.h);
    handles are gap_graph_t handles or Graph objects, scores[i] a float32
    device tensor of graph i's n floats.  `tuning` is a gap_batch_tuning or a
    dict of its fields (None = built-in).  Returns the per-graph stats dicts
    when `stats`."""
    count = len(handles)
    if len(scores) != count:
        raise ValueError(f"gap_pr_run_batch: {count} graphs but {len(scores)} score arrays")
    raw = []
    for i, (h, sc) in enumerate(zip(handles, scores)):
        if isinstance(h, Graph):  # n is known: no library call per graph
            _check_scores(h.handle, sc, 4, "gap_pr_run_batch", n=h.n)
            raw.append(h.handle)
        else:
            _check_scores(h, sc, 4, "gap_pr_run_batch")
            raw.append(h)
    hs = (ctypes.c_void_p * max(count, 1))(*[h if isinstance(h, ctypes.c_void_p) else _ptr(h) for h in raw])
    ps = (ctypes.c_void_p * max(count, 1))(*[_ptr(sc) for sc in scores])
    st = (gap_pr_stats_t * max(count, 1))() if stats else None
    if tuning is None:
        rc = load().gap_pr_run_batch(hs, count, damping, tol, max_iters, ps, st, _stream(stream))
    else:
        if isinstance(tuning, dict):
            t = gap_batch_tuning_default()
            for k, v in tuning.items():
                setattr(t, k, int(v))
            tuning = t
        rc = load().gap_pr_run_batch_ex(hs, count, damping, tol, max_iters, ctypes.byref(tuning), ps,
                                        st, _stream(stream))
    _check(rc, "gap_pr_run_batch")
    return [st[i].to_dict() for i in range(count)] if stats else None


def gap_ppr_batch(h, seed_offsets, seeds, damping: float, tol: float, max_iters: int, scores,
                  stats=True, stream=None):
    """Personalized PageRank for q = len(seed_offsets)-1 queries (see gap.h).
    Returns the list of per-query stats dicts when `stats`."""
    q = len(seed_offsets) - 1
    n = gap_graph_info(h)[0]
    _check_scores(h, scores, 4, "gap_ppr_batch")
    numel = scores.numel() if hasattr(scores, "numel") else getattr(scores, "size", None)
    if numel is not None and numel < q * n:
        raise ValueError(f"gap_ppr_batch: scores holds {numel} floats, need {q * n}")
    st = (gap_pr_stats_t * max(q, 1))() if stats else None
    _check(load().gap_ppr_batch(h, q, _ptr(seed_offsets), _ptr(seeds), damping, tol, max_iters,
                                _ptr(scores), st, _stream(stream)), "gap_ppr_batch")
    return [st[i].to_dict() for i in range(q)] if stats else None


class PprServer:
    """Continuous-batching PPR server (gap_ppr_server_*)."""

    def __init__(self, graph_handle, max_cols=128, hbm_reserve=0, damping=0.85, tol=1e-4,
                 max_iters=100):
        self.handle = ctypes.c_void_p()
        _check(load().gap_ppr_server_create(graph_handle, max_cols, hbm_reserve, damping, tol,
                                            max_iters, ctypes.byref(self.handle)),
               "gap_ppr_server_create")
        self._keep = {}

    def submit(self, seeds, out):
        import numpy as np
        seeds = np.ascontiguousarray(seeds, dtype=np.int32)
        t = ctypes.c_int64()
        _check(load().gap_ppr_submit(self.handle, _ptr(seeds), len(seeds), _ptr(out), ctypes.byref(t)),
               "gap_ppr_submit")
        self._keep[t.value] = out  # the output buffer must outlive the query
        return t.value

    def poll(self, ticket):
        done = ctypes.c_int32()
        info = gap_ppr_query_info_t()
        _check(load().gap_ppr_poll(self.handle, ticket, ctypes.byref(done), ctypes.byref(info)),
               "gap_ppr_poll")
        if done.value:  # the ticket is released once reported done
            self._keep.pop(ticket, None)
            return info.to_dict()
        return None

    def wait(self, ticket):
        info = gap_ppr_query_info_t()
        _check(load().gap_ppr_wait(self.handle, ticket, ctypes.byref(info)), "gap_ppr_wait")
        self._keep.pop(ticket, None)
        return info.to_dict()

    def info(self):
        i = gap_ppr_server_info_t()
        _check(load().gap_ppr_server_info_ex(self.handle, ctypes.byref(i)), "gap_ppr_server_info_ex")
        return i.to_dict()

    def close(self):
        if self.handle is not None and self.handle.value:
            load().gap_ppr_server_destroy(self.handle)
        self.handle = None
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gap_pr_stats(h):
    """Synchronize the last run on h; returns (status, stats dict).  Raises on
    errors; GAP_WARN_NOT_CONVERGED is returned, not raised."""
    st = gap_pr_stats_t()
    s = _check(load().gap_pr_stats(h, ctypes.byref(st)), "gap_pr_stats",
               ok=(GAP_OK, GAP_WARN_NOT_CONVERGED))
    return s, st.to_dict()


# --------------------------------------------------- connected components ---

def gap_cc_run(h, labels, stream=None, n=None):
    """One CC trial into `labels` (int32, n elements, host or device)."""
    if labels is not None and not isinstance(labels, int):
        if n is None:
            n = gap_graph_info(h)[0]
        if hasattr(labels, "element_size"):
            ok = labels.element_size() == 4 and not labels.is_floating_point() and labels.numel() >= n
        else:
            ok = labels.itemsize == 4 and labels.dtype.kind == "i" and labels.size >= n
        if not ok:
            raise ValueError(f"gap_cc_run: labels must be int32 with at least {n} elements")
    return _check(load().gap_cc_run(h, _ptr(labels), _stream(stream)), "gap_cc_run")


def gap_cc_stats(h):
    st = gap_cc_stats_t()
    status = load().gap_cc_stats(h, ctypes.byref(st))
    _check(status, "gap_cc_stats")
    return status, st.to_dict()


# --------------------------------------------------- breadth-first search ---

def gap_bfs_run(h, source: int, parent, stream=None, n=None):
    """One BFS trial from `source` into `parent` (int32, n elements, host or device)."""
    if parent is not None and not isinstance(parent, int):
        if n is None:
            n = gap_graph_info(h)[0]
        if hasattr(parent, "element_size"):
            ok = parent.element_size() == 4 and not parent.is_floating_point() and parent.numel() >= n
        else:
            ok = parent.itemsize == 4 and parent.dtype.kind == "i" and parent.size >= n
        if not ok:
            raise ValueError(f"gap_bfs_run: parent must be int32 with at least {n} elements")
    return _check(load().gap_bfs_run(h, int(source), _ptr(parent), _stream(stream)), "gap_bfs_run")


def gap_bfs_stats(h):
    st = gap_bfs_stats_t()
    _check(load().gap_bfs_stats(h, ctypes.byref(st)), "gap_bfs_stats")
    return st.to_dict()


def bfs_sources(outdeg, count: int = 64, seed: int = 0x5EED):
    """`count` source vertices of non-zero out-degree (§2.3), drawn by a
    splitmix64 sequence from `seed`: deterministic for a graph and seed."""
    import numpy as np
    outdeg = np.asarray(outdeg)
    n = len(outdeg)
    if not (outdeg > 0).any():
        raise ValueError("the graph has no vertex with out-arcs")
    out, i = [], 0
    mask = (1 << 64) - 1
    while len(out) < count:
        z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        z ^= z >> 31
        v = z % n
        if outdeg[v] > 0:
            out.append(int(v))
        i += 1
    return out


# ------------------------------------------------------- failure detection ---

def _device_i(t, dtype_size, count, name):
    """A contiguous CUDA integer tensor of `count` elements of `dtype_size` bytes."""
    if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous() and t.element_size() == dtype_size
            and not t.is_floating_point() and t.numel() >= count):
        raise ValueError(f"{name}: needs a contiguous CUDA integer tensor of {count} x {dtype_size}-byte elements")
    return _ptr(t)


def gap_selftest_check_bin_list(off, lst, bin_start, bin_hi, stream=None):
    """Run the bin-list validator on caller lists; returns (code, where)."""
    import numpy as np
    n = int(lst.numel())
    bs = np.ascontiguousarray(bin_start, np.int64)
    hi = np.ascontiguousarray(bin_hi, np.int64)
    if len(bs) != GAP_PR_BINS + 1 or len(hi) != GAP_PR_BINS - 1:
        raise ValueError("bin_start needs GAP_PR_BINS + 1 entries and bin_hi GAP_PR_BINS - 1")
    code, where = ctypes.c_int32(), ctypes.c_int64()
    _check(load().gap_selftest_check_bin_list(n, _device_i(off, 8, n + 1, "off"), _device_i(lst, 4, n, "list"),
                                              _ptr(bs), _ptr(hi), ctypes.byref(code), ctypes.byref(where),
                                              _stream(stream)), "gap_selftest_check_bin_list")
    return code.value, where.value


def gap_selftest_check_packed(off, packed, prow, seg_end, wbits, small_max, stream=None):
    """Run the packed-arc validator on caller lists; returns (code, where)."""
    n = int(off.numel()) - 1
    S = int(seg_end.numel())
    total = int(seg_end[-1].item()) if S else 0
    code, where = ctypes.c_int32(), ctypes.c_int64()
    _check(load().gap_selftest_check_packed(n, _device_i(off, 8, n + 1, "off"), _device_i(packed, 4, total, "packed"),
                                            _device_i(prow, 4, total, "prow"), _device_i(seg_end, 8, S, "seg_end"),
                                            S, wbits, small_max, ctypes.byref(code), ctypes.byref(where),
                                            _stream(stream)), "gap_selftest_check_packed")
    return code.value, where.value


def gap_selftest_barrier_timeout(stream=None):
    """Run the grid barrier's bounded-wait self-test; returns (observed status,
    waited ms).  The status is GAP_ERR_TIMEOUT when detection works."""
    obs, ms = ctypes.c_int32(), ctypes.c_double()
    _check(load().gap_selftest_barrier_timeout(ctypes.byref(obs), ctypes.byref(ms), _stream(stream)),
           "gap_selftest_barrier_timeout")
    return obs.value, ms.value


class gap_allocator(ctypes.Structure):
    """The C gap_allocator: alloc(bytes, stream, ctx) / free(ptr, bytes, stream, ctx)."""
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    _fields_ = [("alloc", ALLOC), ("free", FREE), ("ctx", ctypes.c_void_p)]


def gap_set_allocator(allocator):
    """Install a gap_allocator (keep the object and its callbacks alive while
    it is installed), or None for the default stream-ordered pool."""
    lib = load()
    return _check(lib.gap_set_allocator(None if allocator is None else ctypes.byref(allocator)),
                  "gap_set_allocator")


# -------------------------------------------------------- convenience ---

class Graph:
    """Owning wrapper around a gap_graph_t handle."""

    def __init__(self, handle):
        self.handle = handle
        self.n, self.m, self.n_dangling = gap_graph_info(handle)

    @classmethod
    def from_edges(cls, n, src, dst, symmetrize=False, dedup=True, drop_self_loops=True,
                   stream=None):
        flags = ((GAP_SYMMETRIZE if symmetrize else 0) | (GAP_DEDUP if dedup else 0)
                 | (GAP_DROP_SELF_LOOPS if drop_self_loops else 0))
        return cls(gap_graph_create_from_edges(n, src, dst, flags, stream))

    @classmethod
    def from_csr(cls, n, row_offsets, col_idx, symmetrize=False, dedup=True, drop_self_loops=True,
                 stream=None):
        flags = ((GAP_SYMMETRIZE if symmetrize else 0) | (GAP_DEDUP if dedup else 0)
                 | (GAP_DROP_SELF_LOOPS if drop_self_loops else 0))
        return cls(gap_graph_create(n, row_offsets, col_idx, flags, stream))

    @classmethod
    def from_csc(cls, n, in_offsets, in_idx, stream=None):
        """A graph from a prebuilt in-direction CSR (copied and checked, not rebuilt)."""
        return cls(gap_graph_create_csc(n, in_offsets, in_idx, stream))

    @classmethod
    def load(cls, path, fmt: int = GAP_FMT_AUTO, symmetrize=False, dedup=True, drop_self_loops=True,
             stream=None):
        """A graph from a file (edge list, Matrix Market, METIS or serialized);
        the cleaning flags apply to text formats only."""
        flags = ((GAP_SYMMETRIZE if symmetrize else 0) | (GAP_DEDUP if dedup else 0)
                 | (GAP_DROP_SELF_LOOPS if drop_self_loops else 0))
        return cls(gap_graph_load(path, fmt, flags, stream))

    def save(self, path, stream=None):
        gap_graph_save(self.handle, path, stream)

    @property
    def build_flags(self) -> int:
        return gap_graph_build_flags(self.handle)

    def export_csr(self, direction: int = 1):
        import numpy as np
        off = np.empty(self.n + 1, np.int64)
        idx = np.empty(max(self.m, 1), np.int32)
        gap_graph_export_csr(self.handle, direction, off, idx)
        return off, idx[: self.m]

    def export_outdeg(self):
        import numpy as np
        out = np.empty(self.n, np.int32)
        gap_graph_export_outdeg(self.handle, out)
        return out

    def close(self):
        if self.handle is not None:
            gap_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
