"""CPU oracle for the GAP PageRank kernel — TEST INFRASTRUCTURE ONLY.

Plain, slow, single-threaded FP64 code (``gap_oracle.c``, built with
``-ffp-contract=off``) that states what the CUDA path computes:

* :func:`build_csr` / :func:`build_csc` — CSR construction with the cleaning
  steps paper §2.3 allows (drop self-loops and duplicates, sort neighbours).
* :func:`pagerank` — the §2.1 PageRank equation iterated in the push
  direction from x0 = 1/n until the summed change drops below tol (§2.1
  tolerance equation), or for a fixed count with tol = 0.
* :func:`verify` — the §3 verifier: one extra serial push iteration, returning
  the summed absolute change (correct when below 1e-4).
* :func:`ppr` — personalized PageRank (not in the paper): teleport (1-d)/|S|
  on a seed set S instead of (1-d)/n.
* :func:`bfs_depths` — §3 serial BFS depths; :func:`bfs_verify` — the §3 BFS
  verifier of a parent array (§2.1 BFS definition).
* :func:`cc` — §2.1 Connected Components (weak), labelled by each component's
  smallest vertex id (union-find); :func:`cc_verify` — the §3 CC verifier
  (one traversal per label).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.
Every function here is pinned by ``tests/test_oracle_pins.py`` against
closed forms, dense linear solves and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gap_oracle.c")
_SRC_MT = os.path.join(_HERE, "csr_threaded.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None
_OMP_SRC = os.path.join(_HERE, "cpu_pull_omp.c")
_OMP_LIB = os.path.join(_LIBDIR, "libcpupull.so")
_omp = None

DAMPING = 0.85
TOL = 1e-4


def build(force: bool = False) -> str:
    """Compile liboracle.so in-tree (gcc -O2 -ffp-contract=off, single-threaded)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f)
                                                 for f in (_SRC, _SRC_MT)):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-pthread", _SRC, _SRC_MT, "-o", tmp])
        os.replace(tmp, _LIB)
    if force or not os.path.exists(_OMP_LIB) or os.path.getmtime(_OMP_LIB) < os.path.getmtime(_OMP_SRC):
        tmp = _OMP_LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", _OMP_SRC, "-o", tmp]
        try:  # the multi-core baseline; one thread where OpenMP is missing
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _OMP_LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
        lib.oracle_build_csr.argtypes = [i64, i64, vp, vp, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, vp, vp, ctypes.POINTER(i64)]
        lib.oracle_pagerank.argtypes = [i64, vp, vp, dbl, dbl, i32, vp, vp]
        lib.oracle_pagerank_from.argtypes = [i64, vp, vp, dbl, dbl, i32, vp, vp]
        lib.oracle_build_csr_threaded.argtypes = [i64, i64, vp, vp, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, vp, vp, ctypes.POINTER(i64), ctypes.c_int]
        lib.oracle_pr_verify.argtypes = [i64, vp, vp, dbl, vp, ctypes.POINTER(dbl)]
        lib.oracle_ppr.argtypes = [i64, vp, vp, dbl, dbl, i32, vp, i32, vp, vp]
        lib.oracle_pr_rows.argtypes = [i64, vp, vp, vp, dbl, vp, i64, vp, vp]
        lib.oracle_ppr_rows.argtypes = [i64, vp, vp, vp, dbl, vp, vp, i32, i64, vp, vp]
        lib.oracle_cc.argtypes = [i64, vp, vp, vp]
        lib.oracle_bfs_depths.argtypes = [i64, vp, vp, i32, vp]
        lib.oracle_bfs_depths.restype = i64
        lib.oracle_bfs_verify.argtypes = [i64, vp, vp, i32, vp]
        lib.oracle_bfs_verify.restype = ctypes.c_int
        lib.oracle_cc_verify.argtypes = [i64, vp, vp, vp]
        for f in (lib.oracle_build_csr, lib.oracle_build_csr_threaded, lib.oracle_pagerank_from,
                  lib.oracle_pagerank, lib.oracle_pr_verify, lib.oracle_ppr,
                  lib.oracle_pr_rows, lib.oracle_ppr_rows, lib.oracle_cc, lib.oracle_cc_verify):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def build_csr(n: int, src, dst, symmetrize: bool = False, dedup: bool = True,
              drop_self_loops: bool = True, threads: int = 1):
    """Out-direction CSR (row u lists v for arcs u->v, ascending).  Returns
    (offsets int64[n+1], idx int32[m]).  threads > 1 runs the row-partitioned
    twin of the builder (csr_threaded.c), whose output is identical."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = len(src)
    if len(dst) != m:
        raise ValueError("src and dst differ in length")
    cap = 2 * m if symmetrize else m
    offsets = np.zeros(n + 1, np.int64)
    idx = np.empty(max(cap, 1), np.int32)
    m_out = ctypes.c_int64(0)
    if threads > 1:
        rc = _load().oracle_build_csr_threaded(n, m, _ptr(src), _ptr(dst), int(symmetrize), int(dedup),
                                               int(drop_self_loops), _ptr(offsets), _ptr(idx),
                                               ctypes.byref(m_out), int(threads))
    else:
        rc = _load().oracle_build_csr(n, m, _ptr(src), _ptr(dst), int(symmetrize), int(dedup),
                                      int(drop_self_loops), _ptr(offsets), _ptr(idx),
                                      ctypes.byref(m_out))
    if rc != 0:
        raise ValueError(f"oracle_build_csr failed ({rc})")
    if threads > 1:  # large graphs: a view, not a second copy of the heads
        return offsets, idx[: m_out.value]
    return offsets, idx[: m_out.value].copy()


def build_csc(n: int, src, dst, symmetrize: bool = False, dedup: bool = True,
              drop_self_loops: bool = True):
    """In-direction CSR (row v lists u for arcs u->v, ascending): the CSR of
    the reversed draws."""
    return build_csr(n, dst, src, symmetrize, dedup, drop_self_loops)


def pagerank(offsets, idx, d: float = DAMPING, tol: float = TOL, max_iters: int = 100):
    """Push-direction FP64 PageRank on an out-CSR.  Returns (x, iterations, deltas)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n = len(offsets) - 1
    x = np.empty(n, np.float64)
    hist = np.zeros(max(max_iters, 1), np.float64)
    k = _load().oracle_pagerank(n, _ptr(offsets), _ptr(idx), d, tol, max_iters, _ptr(x),
                                _ptr(hist))
    if k < 0:
        raise ValueError(f"oracle_pagerank failed ({k})")
    return x, int(k), hist[:k].copy()


def pagerank_from(offsets, idx, x, iters: int, d: float = DAMPING, tol: float = 0.0):
    """Continue the push iteration from the iterate x (FP64) for up to iters
    more iterations (oracle_pagerank's steps and stop test).  Returns (x', k,
    deltas); continuing x_k for j iterations gives pagerank's x_{k+j}."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.array(x, dtype=np.float64, copy=True)
    n = len(offsets) - 1
    hist = np.zeros(max(iters, 1), np.float64)
    k = _load().oracle_pagerank_from(n, _ptr(offsets), _ptr(idx), d, tol, iters, _ptr(out), _ptr(hist))
    if k < 0:
        raise ValueError(f"oracle_pagerank_from failed ({k})")
    return out, int(k), hist[:k].copy()


def verify(offsets, idx, y, d: float = DAMPING) -> float:
    """§3 verifier: summed absolute change of one extra push iteration from y."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.float64)
    n = len(offsets) - 1
    out = ctypes.c_double(0.0)
    rc = _load().oracle_pr_verify(n, _ptr(offsets), _ptr(idx), d, _ptr(y), ctypes.byref(out))
    if rc != 0:
        raise ValueError(f"oracle_pr_verify failed ({rc})")
    return float(out.value)


def pr_rows(in_offsets, in_idx, outdeg, x, rows, d: float = DAMPING):
    """The §2.1 update evaluated for the listed rows only (pull over the CSC):
    returns y'[rows] for the score vector x (FP64)."""
    in_offsets = np.ascontiguousarray(in_offsets, dtype=np.int64)
    in_idx = np.ascontiguousarray(in_idx, dtype=np.int32)
    outdeg = np.ascontiguousarray(outdeg, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    n = len(in_offsets) - 1
    out = np.empty(len(rows), np.float64)
    rc = _load().oracle_pr_rows(n, _ptr(in_offsets), _ptr(in_idx), _ptr(outdeg), d, _ptr(x), len(rows),
                                _ptr(rows), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_pr_rows failed ({rc})")
    return out


def ppr_rows(in_offsets, in_idx, outdeg, x, seeds, rows, d: float = DAMPING):
    """The personalized update evaluated for the listed rows only (pull over
    the CSC): returns y'[rows] for the score vector x (FP64)."""
    in_offsets = np.ascontiguousarray(in_offsets, dtype=np.int64)
    in_idx = np.ascontiguousarray(in_idx, dtype=np.int32)
    outdeg = np.ascontiguousarray(outdeg, dtype=np.int32)
    x = np.ascontiguousarray(x, dtype=np.float64)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    n = len(in_offsets) - 1
    out = np.empty(len(rows), np.float64)
    rc = _load().oracle_ppr_rows(n, _ptr(in_offsets), _ptr(in_idx), _ptr(outdeg), d, _ptr(x), _ptr(seeds),
                                 len(seeds), len(rows), _ptr(rows), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_ppr_rows failed ({rc})")
    return out


def cpu_pagerank_pull(in_offsets, in_idx, outdeg, d: float = DAMPING, tol: float = TOL, max_iters: int = 100):
    """Multi-core CPU baseline (not the oracle): pull PageRank over the CSC
    with OpenMP threads, FP64.  Returns (x, iterations, threads)."""
    global _omp
    if _omp is None:
        build()
        lib = ctypes.CDLL(_OMP_LIB)
        lib.cpu_pagerank_pull.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p]
        lib.cpu_pagerank_pull.restype = ctypes.c_int
        lib.cpu_pull_threads.restype = ctypes.c_int
        _omp = lib
    in_offsets = np.ascontiguousarray(in_offsets, dtype=np.int64)
    in_idx = np.ascontiguousarray(in_idx, dtype=np.int32)
    outdeg = np.ascontiguousarray(outdeg, dtype=np.int32)
    n = len(in_offsets) - 1
    x = np.empty(n, np.float64)
    k = _omp.cpu_pagerank_pull(n, _ptr(in_offsets), _ptr(in_idx), _ptr(outdeg), d, tol, max_iters, _ptr(x))
    if k < 0:
        raise ValueError(f"cpu_pagerank_pull failed ({k})")
    return x, int(k), int(_omp.cpu_pull_threads())


def ppr(offsets, idx, seeds, d: float = DAMPING, tol: float = TOL, max_iters: int = 100):
    """Personalized PageRank with teleport uniform over the distinct seeds.
    Returns (x, iterations, deltas)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    n = len(offsets) - 1
    x = np.empty(n, np.float64)
    hist = np.zeros(max(max_iters, 1), np.float64)
    k = _load().oracle_ppr(n, _ptr(offsets), _ptr(idx), d, tol, max_iters, _ptr(seeds),
                           len(seeds), _ptr(x), _ptr(hist))
    if k < 0:
        raise ValueError(f"oracle_ppr failed ({k})")
    return x, int(k), hist[:k].copy()


def cc(offsets, idx):
    """Weakly connected components of the graph in CSR (either direction):
    int32 labels, each the smallest vertex id of its component (§2.1)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n = len(offsets) - 1
    labels = np.empty(max(n, 1), np.int32)
    rc = _load().oracle_cc(n, _ptr(offsets), _ptr(idx), _ptr(labels))
    if rc != 0:
        raise ValueError(f"oracle_cc failed ({rc})")
    return labels[:n]


def cc_verify(offsets, idx, labels) -> bool:
    """The §3 CC verifier: one traversal per label over the undirected graph;
    True when labels name exactly the weakly connected components."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    n = len(offsets) - 1
    if len(labels) != n:
        raise ValueError("labels must have n entries")
    rc = _load().oracle_cc_verify(n, _ptr(offsets), _ptr(idx), _ptr(labels))
    if rc < 0:
        raise ValueError(f"oracle_cc_verify failed ({rc})")
    return rc == 1


def bfs_depths(offsets, idx, source: int):
    """Depths (int32, -1 unreachable) from `source` over the out-arcs of the CSR."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n = len(offsets) - 1
    depth = np.empty(max(n, 1), np.int32)
    rc = _load().oracle_bfs_depths(n, _ptr(offsets), _ptr(idx), int(source), _ptr(depth))
    if rc < 0:
        raise ValueError(f"oracle_bfs_depths failed ({rc})")
    return depth[:n]


def bfs_verify(offsets, idx, source: int, parent) -> bool:
    """The §3 BFS verifier: True when `parent` is a valid BFS parent array from
    `source` (rows of the CSR sorted, as build_csr makes them)."""
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    n = len(offsets) - 1
    if len(parent) != n:
        raise ValueError("parent must have n entries")
    rc = _load().oracle_bfs_verify(n, _ptr(offsets), _ptr(idx), int(source), _ptr(parent))
    if rc < 0:
        raise ValueError(f"oracle_bfs_verify failed ({rc})")
    return rc == 1
