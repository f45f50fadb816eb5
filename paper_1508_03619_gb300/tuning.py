"""Per-GPU tuning table.

The autotuner (``python -m paper_1508_03619_gb300.autotune``) measures the
launch and split parameters once per GPU model on a tuning set of synthetic
graphs that is disjoint from the evaluation graphs, and writes one fixed JSON
table per model under ``tuning/``.  The table holds hardware-specific values
only (§2.3 allows tuning to the platform, not to an input graph): the same
values are used for every graph on that GPU model, and the per-graph choices
(degree bins, heavy rows) stay run-time decisions inside each trial.

Table layout::

    {"device": "<CUDA device name>", "sms": <SM count>,
     "batch": {gap_batch_tuning fields},
     "pagerank": {"segment_bytes": .., "small_max_degree": ..},
     "tuning_set": "...", "measured": {...}}
"""
from __future__ import annotations

import glob
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE_DIR = os.path.join(HERE, "tuning")


def device_key(device=0):
    """(name, SM count) of a CUDA device."""
    import torch
    p = torch.cuda.get_device_properties(device)
    return p.name, int(p.multi_processor_count)


def load_table(name: str, sms: int):
    """The table entry for this GPU model, or None."""
    for path in sorted(glob.glob(os.path.join(TABLE_DIR, "*.json"))):
        with open(path) as f:
            t = json.load(f)
        if t.get("device") == name and int(t.get("sms", -1)) == sms:
            return t
    return None


def table_for_device(device=0):
    return load_table(*device_key(device))


def batch_tuning_for_device(device=0):
    """gap_batch_tuning fields for this GPU model (dict), or None for the
    library's built-in values."""
    t = table_for_device(device)
    return dict(t["batch"]) if t and "batch" in t else None


def pagerank_options(device=0):
    """gap_pr_options with this GPU model's tuned fields applied."""
    from . import gap
    o = gap.gap_pr_options_default()
    t = table_for_device(device)
    if t and "pagerank" in t:
        for k, v in t["pagerank"].items():
            setattr(o, k, int(v))
    return o
