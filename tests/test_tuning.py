"""Host logic of the per-GPU tuning table and the autotuner's search."""
import json

from paper_1508_03619_gb300 import autotune, tuning


def test_coordinate_search_finds_separable_minimum():
    space = {"a": [1, 2, 3, 4, 5], "b": [10, 20, 30], "c": [0, 1]}
    target = {"a": 4, "b": 20, "c": 1}
    calls = []

    def cost(p):
        calls.append(dict(p))
        return sum((p[k] - target[k]) ** 2 for k in p) + 1.0

    best, c = autotune.coordinate_search(space, {"a": 1, "b": 10, "c": 0}, cost, log=lambda s: None)
    assert best == target and c == 1.0
    assert len(calls) < 2 * sum(len(v) for v in space.values()) + 2


def test_coordinate_search_keeps_start_within_noise():
    # a candidate must beat the incumbent by more than 0.5% to replace it
    best, _ = autotune.coordinate_search({"a": [1, 2]}, {"a": 1},
                                         lambda p: 100.0 if p["a"] == 1 else 99.8, log=lambda s: None)
    assert best == {"a": 1}


def test_table_lookup_by_model(tmp_path, monkeypatch):
    monkeypatch.setattr(tuning, "TABLE_DIR", str(tmp_path))
    (tmp_path / "a.json").write_text(json.dumps({"device": "GPU A", "sms": 152,
                                                 "batch": {"chunk_arcs": 1024}}))
    (tmp_path / "b.json").write_text(json.dumps({"device": "GPU A", "sms": 148,
                                                 "batch": {"chunk_arcs": 4096}}))
    assert tuning.load_table("GPU A", 152)["batch"]["chunk_arcs"] == 1024
    assert tuning.load_table("GPU A", 148)["batch"]["chunk_arcs"] == 4096
    assert tuning.load_table("GPU B", 152) is None


def test_committed_tables_are_well_formed():
    import glob
    import os
    for path in glob.glob(os.path.join(tuning.TABLE_DIR, "*.json")):
        t = json.load(open(path))
        assert isinstance(t["device"], str) and t["sms"] > 0
        if "batch" in t:
            b = t["batch"]
            assert b["heavy_min_degree"] >= 32 and 32 <= b["chunk_arcs"] <= 1 << 24
            assert b["block_threads"] in (128, 256, 512) and b["blocks_per_sm"] >= 0
        if "pagerank" in t:
            assert set(t["pagerank"]) <= {"segment_bytes", "small_max_degree", "group_max_degree",
                                          "cta_max_degree", "hub_chunk_arcs", "group_lanes"}
        assert "tuning_set" in t
