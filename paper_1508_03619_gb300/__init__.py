"""GB300-native pull PageRank of the GAP Benchmark Suite (arXiv:1508.03619).

The compute lives in ``libgap.so`` (hand-written CUDA for sm_103a behind the
C ABI of ``include/gap.h``); :mod:`.gap` is the thin ctypes binding with the
same names.  PyTorch is used only for device memory and streams.
"""
from . import gap  # noqa: F401
from .gap import Graph, GapError  # noqa: F401

__all__ = ["gap", "Graph", "GapError"]
