"""GPU parity on synthetic CSRs built to stress the LEB128 handling of the
run-aware path: validation (run counting), the lookup write pass and the
scatter pass 1 all read the byte stream directly.

  - wide ids: 2.2 million nodes with sparse lists, so deltas and first ids take
    one to four bytes, with runs pinned to id 0 and to id n - 1;
  - long lists: runs of up to 600 ids, so that a list spans many 128-byte
    windows and runs cross window and lane boundaries at every offset.

Each is run for two passes at p = 4 with both table schemes and both first-pass
methods, and compared with the oracle bit for bit after every pass.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vga():
    from paper_2604_08374_gb300 import build
    build.build()
    import paper_2604_08374_gb300 as v
    return v


def _csr(n, frac, runs_max, lengths, seed):
    """Lists of up to runs_max runs (lengths drawn from `lengths`, starts uniform,
    2 % of them at id 0 and 2 % ending at id n - 1) for a `frac` share of the
    nodes; self ids removed, duplicates merged."""
    rng = np.random.default_rng(seed)
    k = rng.integers(0, runs_max + 1, size=n) * (rng.random(n) < frac)
    node = np.repeat(np.arange(n, dtype=np.int64), k)
    m = len(node)
    length = rng.choice(np.asarray(lengths), size=m)
    start = rng.integers(0, n, size=m)
    pick = rng.random(m)
    start[pick < 0.02] = 0
    tail = (pick >= 0.02) & (pick < 0.04)
    start[tail] = n - length[tail]
    start = np.clip(start, 0, n - length)
    rep = np.repeat(np.arange(m), length)
    ids = start[rep] + (np.arange(len(rep)) - np.repeat(np.cumsum(length) - length, length))
    owner = node[rep]
    keep = ids != owner
    key = np.unique(owner[keep] * n + ids[keep])
    owner = key // n
    row_ptr = np.zeros(n + 1, np.uint64)
    row_ptr[1:] = np.cumsum(np.bincount(owner, minlength=n))
    return oracle.csr_encode(row_ptr, (key % n).astype(np.uint32))


_cache = {}


def graph(name):
    if name not in _cache:
        if name == "wide_ids":
            _cache[name] = _csr(2_200_000, 0.04, 6, [1, 2, 3, 4, 5, 7, 15, 16, 17, 31, 33, 64, 150], seed=5)
        else:
            _cache[name] = _csr(60_000, 0.03, 6, [1, 3, 16, 17, 100, 255, 256, 257, 600], seed=9)
    return _cache[name]


@pytest.mark.parametrize("name", ["wide_ids", "long_lists"])
def test_stress_csr_bit_exact(vga, name):
    off, b = graph(name)
    # the stream really holds multi-byte varints
    assert np.count_nonzero(b >= 0x80) > 0
    ref = oracle.hyperball(off, b, 4, 2, seed=11, trace=2)
    with vga.vga_graph_load(off, b) as g:
        for levels in (3, 5):
            for first in (2, 1):
                got = vga.hyperball_run_trace(g, 4, 2, seed=11, max_trace=2, union_mode=2, table_levels=levels,
                                              first_pass=first, slice_bytes=16)
                assert got["iterations"] == ref["iterations"]
                for t in range(got["iterations"] + 1):
                    assert np.array_equal(got["regs"][t], ref["regs"][t]), (levels, first, t)
                assert np.array_equal(got["mean_depth"], ref["mean_depth"], equal_nan=True)
