"""Writes tests/golden/urand4096_oracle.json from the oracle alone.

The fixture fingerprints the oracle's FP64 PageRank on the 4,096-vertex
uniform-random digraph (65,536 draws, seed 0x1, self-loops and duplicates
removed): the tolerance-mode run (d = 0.85, tol = 1e-4) and a 20-iteration
fixed run, the §2.1 connected-components labels (smallest member id per weak
component) and the §3 serial BFS depths from vertex 0.  It is regenerated only by this script, which calls nothing but
``oracle`` and the input generator; the test that reads it checks that the
oracle (and the generator) give the same bits on every machine.
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gapgen  # noqa: E402
import oracle  # noqa: E402


def fingerprint():
    n, m, seed = 4096, 65536, 0x1
    src, dst = gapgen.urand(n, m, seed)
    off, idx = oracle.build_csr(n, src, dst)
    out = {"graph": {"n": n, "draws": m, "seed": seed, "arcs": int(off[-1]),
                     "csr_sha256": hashlib.sha256(off.tobytes() + idx.tobytes()).hexdigest()}}
    for name, tol, iters in (("tolerance", 1e-4, 100), ("fixed20", 0.0, 20)):
        x, k, deltas = oracle.pagerank(off, idx, 0.85, tol, iters)
        out[name] = {"iterations": k, "deltas": [float(d).hex() for d in deltas],
                     "x_sha256": hashlib.sha256(x.tobytes()).hexdigest(),
                     "sum_x": float(x.sum()).hex()}
    lab = oracle.cc(off, idx)
    out["cc"] = {"components": int(len(set(lab.tolist()))),
                 "labels_sha256": hashlib.sha256(lab.tobytes()).hexdigest()}
    depth = oracle.bfs_depths(off, idx, 0)
    out["bfs_from_0"] = {"reached": int((depth >= 0).sum()), "max_depth": int(depth.max()),
                         "depths_sha256": hashlib.sha256(depth.tobytes()).hexdigest()}
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "urand4096_oracle.json"), "w") as f:
        json.dump(fingerprint(), f, indent=1)
        f.write("\n")
