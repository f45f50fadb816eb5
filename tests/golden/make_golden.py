"""Writes tests/golden/urand4096_oracle.json from the oracle alone.

The fixture fingerprints the oracle's FP64 PageRank on the 4,096-vertex
uniform-random digraph (65,536 draws, seed 0x1, self-loops and duplicates
removed): the tolerance-mode run (d = 0.85, tol = 1e-4) and a 20-iteration
fixed run.  It is regenerated only by this script, which calls nothing but
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
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "urand4096_oracle.json"), "w") as f:
        json.dump(fingerprint(), f, indent=1)
        f.write("\n")
