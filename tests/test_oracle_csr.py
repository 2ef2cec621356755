"""Pins for the oracle's delta-compressed LEB128 CSR (Sec. 3.2).

Pinned against the LEB128 encodings printed in the DWARF standard
(tests/golden/leb128.txt), round trips, the malformed-stream rules, and the
paper's own size accounting for a representative node (Sec. 3.2: ~13,800
one-byte deltas plus ~133 two-byte row jumps of ~1200 give ~14 KB compressed
against ~56 KB as 32-bit ids, about 4x).
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _leb_vectors():
    out = []
    for line in open(os.path.join(GOLDEN, "leb128.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            parts = line.split()
            out.append((int(parts[0]), bytes(int(h, 16) for h in parts[1:])))
    return out


@pytest.mark.parametrize("value,encoded", _leb_vectors())
def test_leb128_standard_vectors(value, encoded):
    assert oracle.leb128(value) == encoded


def test_first_absolute_then_deltas():
    row_ptr = np.array([0, 3, 3, 5], np.uint64)
    col = np.array([1, 2, 300, 0, 128], np.uint32)
    offsets, b = oracle.csr_encode(row_ptr, col)
    # node 0: 1 (abs), +1, +298 (2 bytes); node 1: empty; node 2: 0 (abs), +128 (2 bytes)
    assert offsets.tolist() == [0, 4, 4, 7]
    assert bytes(b) == bytes([0x01, 0x01, 0xAA, 0x02, 0x00, 0x80, 0x01])


@pytest.mark.parametrize("seed", range(5))
def test_round_trip_random_lists(seed):
    rng = np.random.default_rng(seed)
    n = 50
    rows = []
    for v in range(n):
        k = int(rng.integers(0, 40))
        ids = np.unique(rng.integers(0, 2**32 - 1, size=k, dtype=np.uint64) if seed % 2 else rng.integers(0, n, size=k))
        rows.append(ids.astype(np.uint64))
    row_ptr = np.zeros(n + 1, np.uint64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.uint32)
    offsets, b = oracle.csr_encode(row_ptr, col)
    big_n = 2**32 if seed % 2 else n
    for v in range(n):
        got = oracle.decode_list(b, int(offsets[v]), int(offsets[v + 1]), big_n)
        assert got.tolist() == rows[v].tolist()


def test_paper_size_accounting():
    # Sec. 3.2: a node with ~13,800 within-row neighbours (delta < 128) and
    # ~133 row jumps of ~1200 compresses to ~14 KB vs ~56 KB uncompressed.
    # 134 runs of 104 consecutive ids (103 one-byte deltas each) joined by 133
    # row jumps of 1201 (two bytes each), after a one-byte absolute first id.
    ids, cur = [], 5
    for r in range(134):
        for k in range(104):
            ids.append(cur)
            cur += 1
        cur += 1200
    row_ptr = np.array([0, len(ids)], np.uint64)
    offsets, b = oracle.csr_encode(row_ptr, np.array(ids, np.uint32))
    compressed = int(offsets[-1])
    raw = 4 * len(ids)
    assert 13_900 <= compressed <= 14_300          # ~14 KB
    assert 55_000 <= raw <= 56_500                  # ~56 KB
    assert 3.8 <= raw / compressed <= 4.1           # ~4x


@pytest.mark.parametrize("stream,n", [
    (bytes([0x80]), 10),                           # varint runs past the end
    (bytes([0x80, 0x80, 0x80, 0x80, 0x80, 0x01]), 2**40),  # six bytes: over the u32 limit
    (bytes([0x03, 0x00]), 10),                     # zero delta: duplicate neighbour
    (bytes([0x0A]), 10),                           # id 10 >= n
    (bytes([0x05, 0x05]), 10),                     # 5 + 5 = 10 >= n
])
def test_malformed_lists_rejected(stream, n):
    assert oracle.decode_list(np.frombuffer(stream, np.uint8), 0, len(stream), n) is None


def test_graph_bytes_per_edge_near_one():
    import workloads
    offsets, b, cells = oracle.build_graph(workloads.tiny(2))
    row_ptr, _ = oracle.decode_csr(offsets, b)
    # raster-ordered visibility lists are dominated by deltas of 1 (one byte each)
    assert 1.0 <= len(b) / int(row_ptr[-1]) < 1.3
