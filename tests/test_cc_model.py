"""Host model of the connected-components schedule the CUDA path runs (CPU).

The GPU kernels link in an order nobody controls, sample only some vertices
in the second round, skip the vertices already in one chosen component in the
final pass and start that pass at position 1 of every in-row.  Whether that
schedule always finds every component does not depend on the GPU: it is a
property of which arcs get linked.  This model replays the same schedule with
a sequential union-find in random orders, with any choice of the skipped
component (not only the largest), on many small symmetric and directed
graphs, and compares the labels with the oracle's union-find."""
import numpy as np
import pytest

import oracle


def _csr(n, src, dst):
    order = np.lexsort((src, dst))  # in-rows: arcs grouped by head, sources ascending
    in_src, in_dst = src[order], dst[order]
    in_off = np.zeros(n + 1, np.int64)
    np.add.at(in_off, in_dst + 1, 1)
    in_off = np.cumsum(in_off)
    order = np.lexsort((dst, src))
    out_dst, out_src = dst[order], src[order]
    out_off = np.zeros(n + 1, np.int64)
    np.add.at(out_off, out_src + 1, 1)
    return in_off, in_src, np.cumsum(out_off), out_dst


def _model_cc(n, in_off, in_idx, out_off, out_idx, directed, rng, participate, pick_giant):
    comp = list(range(n))

    def link(u, v):  # hook the larger root under the smaller
        while comp[u] != u:
            u = comp[u]
        while comp[v] != v:
            v = comp[v]
        if u != v:
            hi, lo = max(u, v), min(u, v)
            comp[hi] = lo

    def compress():
        for v in range(n):
            r = v
            while comp[r] != r:
                r = comp[r]
            comp[v] = r

    for v in rng.permutation(n):  # round 0: every vertex, its first in-neighbour
        if in_off[v + 1] > in_off[v]:
            link(v, int(in_idx[in_off[v]]))
    compress()
    for v in rng.permutation(n):  # round 1: the sampled vertices, their second in-neighbour
        if in_off[v + 1] - in_off[v] > 1 and participate(v):
            link(v, int(in_idx[in_off[v] + 1]))
    compress()
    giant = pick_giant(comp)
    jobs = [("in", v) for v in range(n)] + ([("out", v) for v in range(n)] if directed else [])
    for k in rng.permutation(len(jobs)):
        kind, v = jobs[k]
        if comp[v] == giant:  # skipped: checked when the row is reached, as on the GPU
            continue
        if kind == "in":
            for j in range(in_off[v] + 1, in_off[v + 1]):
                link(v, int(in_idx[j]))
        else:
            for j in range(out_off[v], out_off[v + 1]):
                link(v, int(out_idx[j]))
    compress()
    return np.array(comp, np.int32)


def _hash_participate(bits):
    return lambda v: ((int(v) * 0x9E3779B97F4A7C15) & ((1 << 64) - 1)) >> (64 - bits) == 0


@pytest.mark.parametrize("directed", [False, True])
def test_schedule_finds_every_component_for_any_skipped_component(directed):
    rng = np.random.default_rng(0xCC0 + directed)
    for case in range(250):
        n = int(rng.integers(1, 90))
        m = int(rng.integers(0, 3 * n))
        src = rng.integers(0, n, m).astype(np.int32)
        dst = rng.integers(0, n, m).astype(np.int32)
        if not directed:
            src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
        keep = src != dst
        pairs = np.unique(np.stack([src[keep], dst[keep]], 1), axis=0) if keep.any() else np.zeros((0, 2), np.int32)
        src, dst = pairs[:, 0].astype(np.int32), pairs[:, 1].astype(np.int32)
        in_off, in_idx, out_off, out_idx = _csr(n, src, dst)
        want = oracle.cc(out_off, out_idx)
        for trial in range(3):
            bits = int(rng.integers(0, 5))  # 1, 2, 4, 8 or 16 share of vertices in round 1
            # skip the most frequent root, a random root, or a non-root label nobody has
            choice = trial % 3

            def pick(comp, choice=choice):
                roots = [v for v in range(n) if comp[v] == v]
                if choice == 0:
                    vals, cnt = np.unique(comp, return_counts=True)
                    return int(vals[np.argmax(cnt)])
                if choice == 1:
                    return int(rng.choice(roots))
                return -1

            got = _model_cc(n, in_off, in_idx, out_off, out_idx, directed, rng, _hash_participate(bits),
                            pick)
            assert np.array_equal(got, want), (case, trial, n, m)


def test_the_final_pass_must_start_at_position_1_when_round_1_is_sparse():
    """The final pass starts at position 1 because round 1 links only some
    vertices' second in-neighbour; starting at position 2 (right when round 1
    is full) loses arcs.  Symmetric edges 0-2, 1-3, 2-3: round 0 joins {0, 2}
    and {1, 3}; if vertex 3 does not take part in round 1 and {0, 2} is the
    skipped component, only position 1 of vertex 3's in-row (vertex 2) joins
    the two."""
    n = 4
    src = np.array([0, 2, 1, 3, 2, 3], np.int32)
    dst = np.array([2, 0, 3, 1, 3, 2], np.int32)
    in_off, in_idx, out_off, out_idx = _csr(n, src, dst)
    assert in_idx[in_off[3]:in_off[4]].tolist() == [1, 2]

    def run(start):
        comp = list(range(n))

        def root(x):
            while comp[x] != x:
                x = comp[x]
            return x

        def link(u, v):
            u, v = root(u), root(v)
            if u != v:
                comp[max(u, v)] = min(u, v)

        for v in range(n):
            if in_off[v + 1] > in_off[v]:
                link(v, int(in_idx[in_off[v]]))
        giant = root(0)  # round 1: nobody takes part
        for v in range(n):
            if root(v) != giant:
                for j in range(in_off[v] + start, in_off[v + 1]):
                    link(v, int(in_idx[j]))
        return [root(v) for v in range(n)]

    want = oracle.cc(out_off, out_idx).tolist()
    assert run(1) == want == [0, 0, 0, 0]
    assert run(2) == [0, 1, 0, 1]
