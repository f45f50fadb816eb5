"""Host logic of bench.py that turns measurements into the reported figures:
the roofline entry of the dominant kernel and the clock record."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _stats(segments, lanes0, dom_ms, launches):
    """A trial's stats as the binding reports them: bin 0 dominant."""
    names = ["bin", "init", "pull0", "pull1", "pull2", "pull3", "pull4", "pull5", "pull6",
             "hub_fixup", "finalize", "output", "prep"]
    phase_ms = {k: 0.0 for k in names}
    phase_ms["pull0"] = dom_ms
    phase_ms["pull5"] = dom_ms / 2
    launches_d = {k: 0 for k in names}
    launches_d["pull0"] = launches
    launches_d["pull5"] = launches
    bins = [{"rows": 1000, "arcs": 10000, "max_degree": 255, "lanes": lanes0, "segmented": False}]
    bins += [{"rows": 0, "arcs": 0, "max_degree": 255, "lanes": 1, "segmented": False}] * 3
    bins += [{"rows": 10, "arcs": 2000, "max_degree": 1024, "lanes": 8, "segmented": segments > 1},
             {"rows": 5, "arcs": 5000, "max_degree": 32768, "lanes": 32, "segmented": segments > 1},
             {"rows": 1, "arcs": 100000, "max_degree": 2 ** 63 - 1, "lanes": 0, "segmented": segments > 1}]
    return {"phase_ms": phase_ms, "phase_launches": launches_d, "bins": bins, "iterations": 7}


def test_scaled_traffic_rescales_the_streamed_bytes_only(monkeypatch):
    """Small-case capture C bytes at a arcs, s streamed bytes per arc: a launch
    of A arcs moves C + s (A - a) bytes (the rest is per launch)."""
    monkeypatch.setattr(bench, "NCU_SMALL", {"k": (1.0e6, 1000, 8)})
    assert bench.scaled_traffic("k", 1000) == pytest.approx(1.0e6)
    assert bench.scaled_traffic("k", 5000) == pytest.approx(1.0e6 + 8 * 4000)
    assert bench.scaled_traffic("other", 5000) is None


def test_roofline_entry_of_the_packed_small_row_pass(monkeypatch):
    monkeypatch.setattr(bench, "NCU_SMALL", {"k_pull_small_coo<float,8,32>": (2.0e5, 1000, 8)})
    st = _stats(segments=8, lanes0=-1, dom_ms=5.6, launches=56)
    r = bench.roofline_entry(st, m=117000, n=1016, segments=8)
    assert r["kernel"].startswith("k_pull_small_coo<float,8,32> (bin 0")
    alg = (8 * 10000 + 24 * 1000) * 7 / 56          # per launch
    assert r["alg_bytes_per_launch"] == pytest.approx(alg)
    assert r["launch_ms"] == pytest.approx(0.1)
    assert r["achieved"] == pytest.approx(alg / 1e-4 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["traffic"] == pytest.approx(2.0e5 + 8 * (10000 * 7 / 56 - 1000))
    assert r["useful_byte_efficiency"] == pytest.approx(alg / r["traffic"])
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_roofline_entry_names_the_unsegmented_kernel():
    st = _stats(segments=1, lanes0=-1, dom_ms=1.0, launches=7)
    r = bench.roofline_entry(st, m=117000, n=1016, segments=1)
    assert r["kernel"].startswith("k_pull_small<float,4>") and "whole rows" in r["kernel"]
    assert r["traffic"] is None and r["useful_byte_efficiency"] is None


def test_clock_record():
    rows = ["0, 2070, 2070, 480.1, 0x0, Not Active, Not Active, Not Active, Not Active\n",
            "0, 2065, 2070, 500.0, 0x4, Not Active, Not Active, Not Active, Active\n",
            "0, 2070, 2070, 510.2, 0x0, Not Active, Not Active, Not Active, Not Active\n",
            "garbage\n"]
    c = bench.parse_clock_samples(rows)
    assert c["sm_mhz"] == 2070 and c["sm_max_mhz"] == 2070 and c["samples"] == 3
    assert c["reasons"] == ["sw_power_cap"]
    assert bench.parse_clock_samples([])["reasons"] == ["no samples"]

