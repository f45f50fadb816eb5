"""Seeded synthetic graph inputs shaped like the GAP benchmark graphs (paper §2.2).

This module only draws edge lists; it holds none of PageRank's arithmetic and
is the one piece of code that both the CPU oracle and the CUDA path consume.
Every edge is a pure function of (seed, stream, edge index) via a
counter-based splitmix64, so graphs are identical for any thread count (paper
§3 asks the same of its generators).

Generators (all return ``(src, dst)`` int32 numpy arrays of draws; the graph
builder removes self-loops and duplicates and symmetrizes where asked):

* :func:`urand`   — Erdos-Renyi style uniform draws (paper's "Urand", §2.2).
* :func:`kron`    — Kronecker / R-MAT with Graph 500 parameters
  A=0.57, B=C=0.19 and a seeded random relabelling (paper's "Kron", §2.2).
* :func:`grid`    — road-like 2D lattice with random edge deletions, standing
  in for the paper's "Road" graph shape (high diameter, low degree).
* :func:`chung_lu`— power-law digraph with expected-degree exponent gamma.
* :func:`batch_specs` — the 256-graph uneven batch (half R-MAT, half grids).
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import sys
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libgapgen.so")
_SRC = os.path.join(_HERE, "gapgen.c")
_CORE = os.path.join(_HERE, "gapgen_core.h")
_CUSRC = os.path.join(_HERE, "gapgen_cuda.cu")
_CULIB = os.path.join(_LIBDIR, "libgapgen_cuda.so")
_NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
_lib = None
_culib = None

KRON_A, KRON_B, KRON_C = 0.57, 0.19, 0.19


def _stale(out: str, srcs) -> bool:
    return not os.path.exists(out) or any(os.path.getmtime(out) < os.path.getmtime(x) for x in srcs)


def build(force: bool = False, cuda: bool = True) -> str:
    """Compile libgapgen.so (gcc, no FMA contraction) and, where nvcc exists,
    libgapgen_cuda.so (sm_103a) in-tree."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or _stale(_LIB, [_SRC, _CORE]):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
               _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    if cuda and shutil.which(_NVCC) and (force or _stale(_CULIB, [_CUSRC, _CORE])):
        tmp = _CULIB + f".tmp{os.getpid()}"
        cmd = [_NVCC, "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
               "-lineinfo", "-Xcompiler", "-fPIC", "-shared", _CUSRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _CULIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i64, u64, i32, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        p32 = ctypes.POINTER(ctypes.c_int32)
        lib.gapgen_splitmix64_at.argtypes = [u64, u64]
        lib.gapgen_splitmix64_at.restype = u64
        lib.gapgen_perm_apply.argtypes = [i32, u64, u64]
        lib.gapgen_perm_apply.restype = u64
        lib.gapgen_urand.argtypes = [i64, i64, u64, p32, p32, i32]
        lib.gapgen_kron.argtypes = [i32, i64, dbl, dbl, dbl, u64, i32, p32, p32, i32]
        lib.gapgen_grid.argtypes = [i64, i64, dbl, u64, p32, p32, ctypes.POINTER(i64)]
        pu32 = ctypes.POINTER(ctypes.c_uint32)
        lib.gapgen_chunglu_table.argtypes = [i64, i64, dbl, dbl, pu32, pu32]
        lib.gapgen_chunglu_draw.argtypes = [i64, i64, u64, pu32, pu32, p32, p32, i32]
        lib.gapgen_prob_threshold.argtypes = [dbl]
        lib.gapgen_prob_threshold.restype = ctypes.c_uint32
        for f in (lib.gapgen_urand, lib.gapgen_kron, lib.gapgen_grid, lib.gapgen_chunglu_table,
                  lib.gapgen_chunglu_draw):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _threads() -> int:
    """Generator threads: GAPGEN_THREADS if set, else every core (at most 64);
    the draws do not depend on it."""
    env = os.environ.get("GAPGEN_THREADS")
    if env:
        return max(1, min(64, int(env)))
    return max(1, min(64, os.cpu_count() or 1))


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def splitmix64_at(seed: int, i: int) -> int:
    return int(_load().gapgen_splitmix64_at(seed & (2**64 - 1), i))


def perm_apply(bits: int, seed: int, x: int) -> int:
    return int(_load().gapgen_perm_apply(bits, seed & (2**64 - 1), x))


def urand(n: int, m: int, seed: int):
    """m draws (u, v), each endpoint uniform on [0, n)."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    rc = _load().gapgen_urand(n, m, seed & (2**64 - 1), _p32(src), _p32(dst), _threads())
    if rc != 0:
        raise ValueError(f"gapgen_urand({n}, {m}) failed: {rc}")
    return src, dst


def kron(scale: int, edge_factor: int, seed: int, A: float = KRON_A, B: float = KRON_B,
         C: float = KRON_C, permute: bool = True):
    """edge_factor * 2^scale R-MAT draws on 2^scale vertices (Graph 500 parameters)."""
    m = edge_factor << scale
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    rc = _load().gapgen_kron(scale, m, A, B, C, seed & (2**64 - 1), int(permute), _p32(src),
                             _p32(dst), _threads())
    if rc != 0:
        raise ValueError(f"gapgen_kron(scale={scale}) failed: {rc}")
    return src, dst


def grid(rows: int, cols: int, p_del: float, seed: int):
    """4-neighbour lattice edges (each listed once) with each edge deleted w.p. p_del."""
    cap = 2 * rows * cols
    src = np.empty(cap, np.int32)
    dst = np.empty(cap, np.int32)
    m = ctypes.c_int64(0)
    rc = _load().gapgen_grid(rows, cols, p_del, seed & (2**64 - 1), _p32(src), _p32(dst),
                             ctypes.byref(m))
    if rc != 0:
        raise ValueError(f"gapgen_grid({rows}x{cols}) failed: {rc}")
    return src[: m.value].copy(), dst[: m.value].copy()


def chung_lu_table(n: int, m: int, gamma: float, cap: float | None = None):
    """Alias table (thresh, alias) for Chung-Lu draws with expected degrees
    proportional to (i+1)^(-1/(gamma-1)), capped at `cap` (default sqrt(m))."""
    if cap is None:
        cap = float(np.sqrt(m))
    thresh = np.empty(n, np.uint32)
    alias = np.empty(n, np.uint32)
    pu32 = ctypes.POINTER(ctypes.c_uint32)
    rc = _load().gapgen_chunglu_table(n, m, gamma, cap, thresh.ctypes.data_as(pu32),
                                      alias.ctypes.data_as(pu32))
    if rc != 0:
        raise ValueError(f"gapgen_chunglu_table(n={n}, m={m}) failed: {rc}")
    return thresh, alias


def chung_lu(n: int, m: int, gamma: float, seed: int, cap: float | None = None, table=None):
    """m Chung-Lu draws on n (power of two) vertices, expected-degree exponent gamma."""
    thresh, alias = table if table is not None else chung_lu_table(n, m, gamma, cap)
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    pu32 = ctypes.POINTER(ctypes.c_uint32)
    rc = _load().gapgen_chunglu_draw(n, m, seed & (2**64 - 1), thresh.ctypes.data_as(pu32),
                                     alias.ctypes.data_as(pu32), _p32(src), _p32(dst), _threads())
    if rc != 0:
        raise ValueError(f"gapgen_chunglu_draw(n={n}, m={m}) failed: {rc}")
    return src, dst


# ---- device twins (same draws, written straight into HBM) ----

def _load_cuda():
    global _culib
    if _culib is None:
        build()
        if not os.path.exists(_CULIB):
            raise RuntimeError("libgapgen_cuda.so is not built (nvcc missing?)")
        lib = ctypes.CDLL(_CULIB)
        i64, u64, i32, u32, vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32,
                                  ctypes.c_void_p)
        lib.gapgen_cuda_urand.argtypes = [i64, i64, u64, vp, vp, vp]
        lib.gapgen_cuda_kron.argtypes = [i32, i64, u32, u32, u32, u64, i32, vp, vp, vp]
        lib.gapgen_cuda_chunglu.argtypes = [i64, i64, u64, vp, vp, vp, vp, vp]
        for f in (lib.gapgen_cuda_urand, lib.gapgen_cuda_kron, lib.gapgen_cuda_chunglu):
            f.restype = ctypes.c_int
        _culib = lib
    return _culib


def _dev_pair(m: int, device):
    import torch
    return (torch.empty(m, dtype=torch.int32, device=device),
            torch.empty(m, dtype=torch.int32, device=device))


def _stream_ptr(device):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def urand_device(n: int, m: int, seed: int, device="cuda"):
    """Device twin of :func:`urand`; returns two int32 CUDA tensors."""
    src, dst = _dev_pair(m, device)
    rc = _load_cuda().gapgen_cuda_urand(n, m, seed & (2**64 - 1), src.data_ptr(), dst.data_ptr(),
                                        _stream_ptr(src.device))
    if rc != 0:
        raise RuntimeError(f"gapgen_cuda_urand failed: {rc}")
    return src, dst


def kron_device(scale: int, edge_factor: int, seed: int, A: float = KRON_A, B: float = KRON_B,
                C: float = KRON_C, permute: bool = True, device="cuda"):
    """Device twin of :func:`kron`; returns two int32 CUDA tensors."""
    m = edge_factor << scale
    lib = _load()
    tA, tAB, tABC = (lib.gapgen_prob_threshold(A), lib.gapgen_prob_threshold(A + B),
                     lib.gapgen_prob_threshold(A + B + C))
    src, dst = _dev_pair(m, device)
    rc = _load_cuda().gapgen_cuda_kron(scale, m, tA, tAB, tABC, seed & (2**64 - 1), int(permute),
                                       src.data_ptr(), dst.data_ptr(), _stream_ptr(src.device))
    if rc != 0:
        raise RuntimeError(f"gapgen_cuda_kron failed: {rc}")
    return src, dst


def chung_lu_device(n: int, m: int, gamma: float, seed: int, cap: float | None = None,
                    table=None, device="cuda"):
    """Device twin of :func:`chung_lu` (alias table built on the host)."""
    import torch
    thresh, alias = table if table is not None else chung_lu_table(n, m, gamma, cap)
    t_thr = torch.from_numpy(thresh.view(np.int32)).to(device)
    t_ali = torch.from_numpy(alias.view(np.int32)).to(device)
    src, dst = _dev_pair(m, device)
    rc = _load_cuda().gapgen_cuda_chunglu(n, m, seed & (2**64 - 1), t_thr.data_ptr(),
                                          t_ali.data_ptr(), src.data_ptr(), dst.data_ptr(),
                                          _stream_ptr(src.device))
    if rc != 0:
        raise RuntimeError(f"gapgen_cuda_chunglu failed: {rc}")
    torch.cuda.current_stream(src.device).synchronize()
    return src, dst


@dataclass(frozen=True)
class GraphSpec:
    """One member of the uneven batch: kind 'rmat' or 'grid'."""
    kind: str
    n: int
    seed: int
    edge_factor: int = 0  # rmat only
    rows: int = 0         # grid only
    cols: int = 0         # grid only
    p_del: float = 0.05   # grid only

    def edges(self):
        if self.kind == "rmat":
            scale = self.n.bit_length() - 1
            return kron(scale, self.edge_factor, self.seed)
        return grid(self.rows, self.cols, self.p_del, self.seed)


def batch_specs(count: int = 256, seed: int = 0x4, min_exp: int = 10, max_exp: int = 18):
    """The uneven batch: count/2 R-MAT graphs with n = 2^U(min_exp..max_exp) and edge
    factor U(8..32), then count/2 grids with n = 2^U(min_exp..max_exp) vertices laid out
    as a x b (a = 2^floor(e/2), b = 2^ceil(e/2)) and 5% edge deletions.  All choices
    come from the counter-based generator keyed by `seed`."""
    specs = []
    span = max_exp - min_exp + 1
    for i in range(count):
        r = splitmix64_at(seed, 3 * i)
        e = min_exp + (r >> 32) % span
        gseed = splitmix64_at(seed, 3 * i + 1)
        if i < count // 2:
            ef = 8 + (splitmix64_at(seed, 3 * i + 2) >> 32) % 25
            specs.append(GraphSpec("rmat", 1 << e, gseed, edge_factor=int(ef)))
        else:
            a, b = 1 << (e // 2), 1 << (e - e // 2)
            specs.append(GraphSpec("grid", a * b, gseed, rows=a, cols=b, p_del=0.05))
    return specs


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
    print(_LIB)
