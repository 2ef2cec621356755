"""Pins for the oracle's Hilbert numbering (Sec. 3.2, optional Hilbert
reordering): the curve visits every cell of the 2^k square exactly once, and
consecutive cells along it are 4-neighbours (the defining property of the
Hilbert curve); the first-order curve is the U through (0,0), (0,1), (1,1),
(1,0).  A Hilbert-numbered graph has the same edges as the raster one, up to
the renumbering, and compresses to within 1 % of it, as the paper reports."""
import numpy as np
import pytest

import oracle
import workloads


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_hilbert_is_a_continuous_bijection(k):
    n = 1 << k
    pos = {}
    for x in range(n):
        for y in range(n):
            pos[oracle.hilbert_index(k, x, y)] = (x, y)
    assert sorted(pos) == list(range(n * n))
    for d in range(n * n - 1):
        (x0, y0), (x1, y1) = pos[d], pos[d + 1]
        assert abs(x0 - x1) + abs(y0 - y1) == 1, (k, d)
    assert pos[0] == (0, 0)


def test_first_order_curve():
    assert [oracle.hilbert_index(1, x, y) for (x, y) in [(0, 0), (0, 1), (1, 1), (1, 0)]] == [0, 1, 2, 3]


def test_hilbert_graph_is_a_renumbering():
    obst = workloads.tiny(2)
    off_r, b_r, cells_r = oracle.build_graph(obst)
    off_h, b_h, cells_h = oracle.build_graph(obst, order="hilbert")
    assert sorted(cells_h.tolist()) == cells_r.tolist()
    rp_r, col_r = oracle.decode_csr(off_r, b_r)
    rp_h, col_h = oracle.decode_csr(off_h, b_h)
    raster_id = {int(c): i for i, c in enumerate(cells_r)}
    to_r = np.array([raster_id[int(c)] for c in cells_h])
    edges_r = {(u, int(w)) for u in range(len(cells_r)) for w in col_r[rp_r[u]:rp_r[u + 1]]}
    edges_h = {(int(to_r[u]), int(to_r[w])) for u in range(len(cells_h)) for w in col_h[rp_h[u]:rp_h[u + 1]]}
    assert edges_r == edges_h
    assert abs(len(b_h) / len(b_r) - 1) < 0.01   # "within 1 %" (Sec. 3.2)
