"""Graph files on the host (paper §3: the reference loads METIS, Matrix Market
and a plain edge list, and serializes built graphs).  Parsing needs no GPU:
each format is checked against hand-written expectations, against the
oracle's CSR builder on seeded graphs written out as text, and on malformed
input.  Header checks of serialized files also run before any device call."""
import numpy as np
import pytest

import gapgen
import oracle
from paper_1508_03619_gb300 import gap

import gcsc_format


def _read(tmp_path, name, text, fmt=gap.GAP_FMT_AUTO):
    p = tmp_path / name
    p.write_bytes(text.encode() if isinstance(text, str) else text)
    return gap.gap_edge_list_read(p, fmt)


def _arcs(src, dst):
    return list(zip(src.tolist(), dst.tolist()))


# ---------------------------------------------------------------- formats ---

def test_edge_list_comments_weights_blank_lines_crlf(tmp_path):
    text = "# a comment\n0 1\n\n  2\t3  \r\n% another\n3 0 7\n1 1 0.25\n5 2"  # no final newline
    n, src, dst, fl = _read(tmp_path, "g.el", text)
    assert n == 6 and fl == 0
    assert _arcs(src, dst) == [(0, 1), (2, 3), (3, 0), (1, 1), (5, 2)]


def test_edge_list_long_file_spans_buffer_refills(tmp_path):
    src0, dst0 = gapgen.urand(1 << 12, 1 << 20, seed=0x77)  # ~11 MB of text, one refill
    text = "".join(f"{u} {v}\n" for u, v in zip(src0.tolist(), dst0.tolist()))
    n, src, dst, _ = _read(tmp_path, "big.txt", text)
    assert np.array_equal(src, src0) and np.array_equal(dst, dst0)
    assert n == max(src0.max(), dst0.max()) + 1


def test_matrix_market_general_and_symmetric(tmp_path):
    gen = ("%%MatrixMarket matrix coordinate pattern general\n% c\n\n4 5 3\n1 2\n3 4\n4 1\n")
    n, src, dst, fl = _read(tmp_path, "a.mtx", gen)
    assert (n, fl) == (5, 0) and _arcs(src, dst) == [(0, 1), (2, 3), (3, 0)]
    sym = ("%%matrixmarket MATRIX Coordinate real Symmetric\n3 3 2\n2 1 0.5\n3 3 -1e3\n")
    n, src, dst, fl = _read(tmp_path, "b.mtx", sym)
    assert (n, fl) == (3, gap.GAP_SYMMETRIZE) and _arcs(src, dst) == [(1, 0), (2, 2)]
    n, src, dst, fl = _read(tmp_path, "c.txt", "%%MatrixMarket matrix coordinate integer hermitian\n2 2 1\n2 1 4\n",
                            gap.GAP_FMT_MATRIX_MARKET)
    assert (n, fl) == (2, gap.GAP_SYMMETRIZE) and _arcs(src, dst) == [(1, 0)]


def test_metis_plain_weighted_and_blank_vertices(tmp_path):
    # path 1-2-3 plus isolated vertex 4 (blank line), 1-based neighbours
    plain = "% comment\n4 2\n2\n1 3\n2\n\n"
    n, src, dst, fl = _read(tmp_path, "p.graph", plain)
    assert (n, fl) == (4, 0) and _arcs(src, dst) == [(0, 1), (1, 0), (1, 2), (2, 1)]
    # fmt 011: one vertex weight first, then (neighbour, edge weight) pairs
    weighted = "3 2 011\n5 2 9\n6 1 9 3 4\n7 2 4\n"
    n, src, dst, _ = _read(tmp_path, "w.metis", weighted)
    assert n == 3 and _arcs(src, dst) == [(0, 1), (1, 0), (1, 2), (2, 1)]
    # fmt 110 with ncon = 2: a vertex size and two vertex weights, no edge weights
    sized = "2 1 110 2\n1 5 5 2\n1 6 6 1\n"
    n, src, dst, _ = _read(tmp_path, "s.graph", sized)
    assert n == 2 and _arcs(src, dst) == [(0, 1), (1, 0)]


@pytest.mark.parametrize("name,text,msg", [
    ("a.el", "0\n", "two integer"),
    ("b.el", "0 -1\n", "outside"),
    ("c.el", "0 2147483647\n", "outside"),
    ("d.el", "1.5 2\n", "two integer"),
    ("e.mtx", "%%MatrixMarket matrix array real general\n2 2\n1\n2\n3\n4\n", "coordinate"),
    ("f.mtx", "%MatrixMarket matrix coordinate pattern general\n2 2 1\n1 2\n", "MatrixMarket"),
    ("g.mtx", "%%MatrixMarket matrix coordinate pattern general\n2 2 1\n3 1\n", "outside the matrix"),
    ("h.mtx", "%%MatrixMarket matrix coordinate pattern general\n2 2 2\n1 2\n", "fewer entries"),
    ("i.mtx", "%%MatrixMarket matrix coordinate pattern general\n2 2 1\n1 2\n2 1\n", "more entries"),
    ("j.mtx", "%%MatrixMarket matrix coordinate pattern skewed\n2 2 1\n1 2\n", "symmetry"),
    ("k.graph", "3 2\n2\n1\n", "fewer vertex lines"),
    ("l.graph", "2 1\n2\n1\n1\n", "more vertex lines"),
    ("m.graph", "2 1\n3\n1\n", "outside [1, n]"),
    ("n.graph", "3 2\n2\n1\n\n", "2m"),
    ("o.graph", "2 1 1\n2\n1 1\n", "edge weight"),
    ("p.graph", "2 1 2\n2\n1\n", "3-digit"),
])
def test_malformed_text_is_rejected_with_the_line(tmp_path, name, text, msg):
    with pytest.raises(gap.GapError) as ei:
        _read(tmp_path, name, text)
    assert ei.value.status == gap.GAP_ERR_INVALID_ARG
    assert msg in str(ei.value) and name in str(ei.value)


def test_unknown_suffix_and_missing_file(tmp_path):
    with pytest.raises(gap.GapError, match="not a text graph format"):
        _read(tmp_path, "g.bin", "0 1\n")
    with pytest.raises(gap.GapError, match="cannot open"):
        gap.gap_edge_list_read(tmp_path / "missing.el")
    with pytest.raises(gap.GapError, match="not a text graph format"):
        _read(tmp_path, "g.gcsc", "0 1\n")


# ------------------------------------- text round trips through the oracle ---

def _oracle_csr(n, src, dst, symmetrize):
    return oracle.build_csr(n, src, dst, symmetrize, True, True)


def test_seeded_graphs_written_as_text_rebuild_the_same_csr(tmp_path):
    """A seeded R-MAT graph written out in each format and parsed back gives
    the oracle builder the same CSR as the generator's own draws."""
    scale = 10
    n = 1 << scale
    src0, dst0 = gapgen.kron(scale, 8, seed=0x31)
    want_dir = _oracle_csr(n, src0, dst0, False)
    want_sym = _oracle_csr(n, src0, dst0, True)

    (tmp_path / "k.el").write_text("".join(f"{u} {v}\n" for u, v in zip(src0.tolist(), dst0.tolist())))
    m_n, s, d, fl = gap.gap_edge_list_read(tmp_path / "k.el")
    got = _oracle_csr(n, s, d, False)
    assert fl == 0 and m_n <= n
    assert all(np.array_equal(a, b) for a, b in zip(got, want_dir))

    # Matrix Market, symmetric: the lower triangle of the symmetrized graph
    off, idx = want_sym
    rows = np.repeat(np.arange(n), np.diff(off))
    low = rows >= idx
    body = "".join(f"{r + 1} {c + 1}\n" for r, c in zip(rows[low].tolist(), idx[low].tolist()))
    (tmp_path / "k.mtx").write_text(f"%%MatrixMarket matrix coordinate pattern symmetric\n{n} {n} {low.sum()}\n"
                                    + body)
    m_n, s, d, fl = gap.gap_edge_list_read(tmp_path / "k.mtx")
    assert m_n == n and fl == gap.GAP_SYMMETRIZE
    got = _oracle_csr(n, s, d, True)
    assert all(np.array_equal(a, b) for a, b in zip(got, want_sym))

    # METIS: every vertex's neighbour list of the symmetrized graph
    lines = [f"{n} {len(idx) // 2}"]
    lines += [" ".join(str(j + 1) for j in idx[off[v]:off[v + 1]].tolist()) for v in range(n)]
    (tmp_path / "k.graph").write_text("\n".join(lines) + "\n")
    m_n, s, d, fl = gap.gap_edge_list_read(tmp_path / "k.graph")
    assert m_n == n and fl == 0 and len(s) == len(idx)
    got = _oracle_csr(n, s, d, False)
    assert all(np.array_equal(a, b) for a, b in zip(got, want_sym))


# ------------------------------------------ serialized headers (host side) ---

def _good(tmp_path, name="g.gcsc"):
    p = tmp_path / name
    gcsc_format.write(p, 3, [0, 1, 2, 2], [1, 0])
    return p


@pytest.mark.parametrize("damage,msg", [
    (lambda b: b"XAPCSC\x00\x01" + b[8:], "bad magic"),
    (lambda b: b[:8] + (2).to_bytes(4, "little") + b[12:], "unsupported version"),
    (lambda b: b[:36] + (0x04030201).to_bytes(4, "little") + b[40:], "byte order"),
    (lambda b: b[:-1], "the header implies"),
    (lambda b: b + b"\x00" * 4, "the header implies"),
    (lambda b: b[:16] + (0).to_bytes(8, "little") + b[24:], "out of range"),
    (lambda b: b[:20], "shorter than"),
])
def test_serialized_header_damage_is_rejected_before_any_device_work(tmp_path, damage, msg):
    p = _good(tmp_path)
    p.write_bytes(damage(p.read_bytes()))
    with pytest.raises(gap.GapError) as ei:
        gap.gap_graph_load(p)
    assert ei.value.status == gap.GAP_ERR_INVALID_ARG and msg in str(ei.value)


def test_checksum_definition_pins():
    """The checksum of the documented definition on hand-checkable payloads:
    empty payload sums nothing; one zero word is mix(golden); word order matters."""
    assert gcsc_format.checksum(b"") == 0
    g = 0x9E3779B97F4A7C15
    z = g
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) % 2 ** 64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) % 2 ** 64
    z ^= z >> 31
    assert gcsc_format.checksum(b"\x00" * 8) == z
    assert gcsc_format.checksum(b"\x00" * 3) == z  # zero-padded tail
    a = (1).to_bytes(8, "little") + (2).to_bytes(8, "little")
    b = (2).to_bytes(8, "little") + (1).to_bytes(8, "little")
    assert gcsc_format.checksum(a) != gcsc_format.checksum(b)


def test_load_flags_and_formats_checked_before_device_work(tmp_path):
    p = tmp_path / "g.el"
    p.write_text("0 1\n")
    with pytest.raises(gap.GapError, match="GAP_INPUT_ON_DEVICE"):
        gap.gap_graph_load(p, gap.GAP_FMT_AUTO, gap.GAP_INPUT_ON_DEVICE)
    q = tmp_path / "g.unknown"
    q.write_text("0 1\n")
    with pytest.raises(gap.GapError, match="unknown graph format"):
        gap.gap_graph_load(q)
    e = tmp_path / "empty.el"
    e.write_text("# nothing\n")
    with pytest.raises(gap.GapError, match="no vertex"):
        gap.gap_graph_load(e)


def test_bfs_source_selector_is_deterministic_and_picks_vertices_with_out_arcs():
    """§2.3: sources are random vertices of non-zero degree, drawn by a
    deterministic selector (same graph and seed, same sources)."""
    rng = np.random.default_rng(5)
    outdeg = rng.integers(0, 3, 5000)
    a = gap.bfs_sources(outdeg, 64)
    assert a == gap.bfs_sources(outdeg, 64) and len(a) == 64
    assert all(outdeg[v] > 0 for v in a)
    assert gap.bfs_sources(outdeg, 64, seed=7) != a
    assert len(set(a)) > 50  # spread over the graph, not one vertex repeated
    with pytest.raises(ValueError):
        gap.bfs_sources(np.zeros(10, np.int64), 4)


def test_line_longer_than_the_read_buffer(tmp_path):
    """A METIS vertex line of ~27 MB (a hub with 3.5M neighbours) is longer
    than the reader's 16 MB buffer, which must grow to hold it."""
    n = 3_500_001
    hub_line = " ".join(map(str, range(2, n + 1)))
    assert len(hub_line) > (16 << 20)
    text = f"{n} {n - 1}\n" + hub_line + "\n" + "1\n" * (n - 1)
    p = tmp_path / "hub.graph"
    p.write_text(text)
    m_n, src, dst, _ = gap.gap_edge_list_read(p)
    assert m_n == n and len(src) == 2 * (n - 1)
    assert (src[: n - 1] == 0).all() and np.array_equal(dst[: n - 1], np.arange(1, n))
    assert np.array_equal(src[n - 1:], np.arange(1, n)) and (dst[n - 1:] == 0).all()
