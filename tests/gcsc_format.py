"""Independent numpy reading of the serialized graph format that
include/gap.h documents (GAP_FMT_SERIALIZED): used by the tests to read files
the library wrote and to write files (valid or deliberately inconsistent)
for the library to load."""
import numpy as np

MAGIC = b"GAPCSC\x00\x01"
ORDER_TAG = 0x01020304
GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _mix(z):
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def checksum(payload: bytes) -> int:
    """Sum over the 64-bit little-endian words w_i (i from 1, last word
    zero-padded) of splitmix64-finalizer(w_i + i * golden), modulo 2^64."""
    pad = (-len(payload)) % 8
    w = np.frombuffer(payload + b"\x00" * pad, dtype="<u8")
    with np.errstate(over="ignore"):
        i = np.arange(1, len(w) + 1, dtype=np.uint64)
        return int(np.sum(_mix(w + i * GOLDEN), dtype=np.uint64))


def write(path, n, off, idx, flags=0, version=1, order_tag=ORDER_TAG, checksum_value=None):
    off = np.ascontiguousarray(off, dtype="<i8")
    idx = np.ascontiguousarray(idx, dtype="<i4")
    payload = off.tobytes() + idx.tobytes()
    ck = checksum(payload) if checksum_value is None else checksum_value
    hdr = (MAGIC + np.array([version, 64], "<u4").tobytes() + np.array([n, len(idx)], "<i8").tobytes()
           + np.array([flags, order_tag], "<u4").tobytes() + np.array([ck], "<u8").tobytes() + b"\x00" * 16)
    assert len(hdr) == 64
    with open(path, "wb") as f:
        f.write(hdr + payload)


def read(path):
    """(n, m, flags, checksum, off, idx) of a serialized file."""
    raw = open(path, "rb").read()
    assert raw[:8] == MAGIC
    version, hbytes = np.frombuffer(raw[8:16], "<u4")
    n, m = (int(v) for v in np.frombuffer(raw[16:32], "<i8"))
    flags, tag = (int(v) for v in np.frombuffer(raw[32:40], "<u4"))
    ck = int(np.frombuffer(raw[40:48], "<u8")[0])
    assert version == 1 and hbytes == 64 and tag == ORDER_TAG and raw[48:64] == b"\x00" * 16
    off = np.frombuffer(raw[64:64 + 8 * (n + 1)], "<i8")
    idx = np.frombuffer(raw[64 + 8 * (n + 1):], "<i4")
    assert len(idx) == m
    assert checksum(raw[64:]) == ck
    return n, m, flags, ck, off, idx
