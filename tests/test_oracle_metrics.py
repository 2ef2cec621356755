"""Pins for the oracle's closed-form VGA metrics (Sec. 3.3, "Metric derivation").

- The RRA normaliser D_k is checked against its definition: the relative
  asymmetry of the root of a diamond-shaped graph (1, 2, 4, ..., 2^h, ..., 2, 1
  nodes per level) with k = 3 * 2^h - 2 nodes, computed by exact BFS.
- Complete graphs (exact MD = 1) and end nodes of paths (exact MD = k / 2)
  give the textbook values: Tekl 0, P-value 1, HH infinite; RA = 1, P-value 0,
  HH = D_k.
- Degenerate components (k <= 2) leave RA undefined.
"""
import math

import numpy as np
import pytest

import oracle


def diamond_graph(h):
    levels = [2 ** i for i in range(h + 1)] + [2 ** i for i in range(h - 1, -1, -1)]
    ids, start = [], 0
    for w in levels:
        ids.append(list(range(start, start + w)))
        start += w
    n = start
    adj = [set() for _ in range(n)]
    for a, b in zip(ids[:-1], ids[1:]):
        if len(b) > len(a):      # widening: node i feeds children 2i, 2i+1
            for i, u in enumerate(a):
                for w in b[2 * i:2 * i + 2]:
                    adj[u].add(w), adj[w].add(u)
        else:                    # narrowing: children 2i, 2i+1 merge into i
            for i, w in enumerate(b):
                for u in a[2 * i:2 * i + 2]:
                    adj[u].add(w), adj[w].add(u)
    row_ptr = np.zeros(n + 1, np.uint64)
    row_ptr[1:] = np.cumsum([len(a) for a in adj])
    col = np.concatenate([sorted(a) for a in adj]).astype(np.uint32)
    return n, oracle.csr_encode(row_ptr, col)


@pytest.mark.parametrize("h", [1, 2, 3, 4, 5, 6])
def test_dvalue_is_the_diamond_root_relative_asymmetry(h):
    n, (off, b) = diamond_graph(h)
    assert n == 3 * 2 ** h - 2
    dist, ecc = oracle.bfs(off, b, 0)
    assert ecc == 2 * h
    md = dist.sum() / (n - 1)
    ra = 2 * (md - 1) / (n - 2)
    assert oracle.dvalue(n) == pytest.approx(ra, rel=1e-13)


def test_complete_graph_values():
    n = 50
    deg = np.full(n, n - 1, np.uint32)
    m = oracle.metrics(np.ones(n), deg)
    assert np.all(np.isinf(m[:, 0]))          # HH = D / 0
    assert np.all(m[:, 1] == 0.0)             # Tekl = log2(3/3)
    assert np.all(m[:, 2] == 1.0)             # P-value = 1 - 0
    assert np.all(m[:, 3] == n - 1)           # PFM = 1 x deg


@pytest.mark.parametrize("k", [5, 12, 101])
def test_path_end_values(k):
    md = np.array([k / 2.0])
    m = oracle.metrics(md, np.array([1], np.uint32), comp_size=np.array([k], np.uint32))
    assert m[0, 2] == 0.0                                   # RA = 1 exactly
    assert m[0, 0] == pytest.approx(oracle.dvalue(k), rel=1e-15)
    assert m[0, 1] == pytest.approx(math.log2((k / 2 + 2) / 3), rel=1e-15)
    assert m[0, 3] == k / 2.0


def test_pvalue_clamps_and_degenerate_components():
    m = oracle.metrics(np.array([30.0, 1.5, 1.0]), np.array([3, 3, 1], np.uint32),
                       comp_size=np.array([20, 2, 1], np.uint32))
    assert m[0, 2] == 0.0                     # RA > 1 clamps at 0
    assert np.isnan(m[1, 0]) and np.isnan(m[1, 2])
    assert np.isnan(m[2, 0]) and np.isnan(m[2, 2])
    assert m[1, 1] == pytest.approx(math.log2(3.5 / 3))
