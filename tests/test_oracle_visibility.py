"""Pins for the oracle's visibility builder (Sec. 3.1) and node numbering.

The supercover traversal is pinned against (a) a brute-force separating-axis
test over every cell of the segment's bounding box, (b) hand-derived graphs in
tests/golden/visibility_hand.txt, and (c) geometric invariants: symmetry, the
complete graph of an open grid, and 4-neighbours always seeing each other.
"""
import os

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_hand_cases():
    cases, cur = {}, None
    for line in open(os.path.join(GOLDEN, "visibility_hand.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        if key == "case":
            cur = cases.setdefault(rest, {"grid": [], "edges": set()})
        elif key == "grid":
            cur["grid"].append([1 if ch == "#" else 0 for ch in rest])
        elif key == "edge":
            a, b = map(int, rest.split())
            cur["edges"].add((min(a, b), max(a, b)))
    return cases


@pytest.mark.parametrize("name", sorted(_load_hand_cases()))
def test_hand_derived_graphs(name):
    case = _load_hand_cases()[name]
    obst = np.array(case["grid"], np.uint8)
    offsets, bytes_, _ = oracle.build_graph(obst, nthreads=1)
    row_ptr, col = oracle.decode_csr(offsets, bytes_)
    edges = set()
    for v in range(len(offsets) - 1):
        for w in col[row_ptr[v]:row_ptr[v + 1]]:
            edges.add((min(v, int(w)), max(v, int(w))))
    assert edges == case["edges"]


def test_segment_cell_cases():
    # straight row: passes through the interior of the cells between, never the rows above/below
    assert oracle.segment_meets_cell(0, 0, 3, 0, 1, 0)
    assert not oracle.segment_meets_cell(0, 0, 3, 0, 1, 1)
    # diagonal passes through grid corners and touches the four cells around each
    assert oracle.segment_meets_cell(0, 0, 2, 2, 1, 0)
    assert oracle.segment_meets_cell(0, 0, 2, 2, 0, 1)
    assert not oracle.segment_meets_cell(0, 0, 2, 2, 2, 0)
    # a shallow line clears a cell it only approaches
    assert not oracle.segment_meets_cell(0, 0, 4, 1, 0, 1)
    assert oracle.segment_meets_cell(0, 0, 4, 1, 2, 1)


@pytest.mark.parametrize("seed", range(6))
def test_dda_matches_bruteforce_all_pairs(seed):
    obst = workloads.random_rectangles(14, 11, 5, (1, 4), seed)
    H, W = obst.shape
    cells = [(x, y) for y in range(H) for x in range(W) if not obst[y, x]]
    for i, a in enumerate(cells):
        for b in cells[i + 1:]:
            fwd = oracle.visible_dda(obst, a, b)
            assert fwd == oracle.visible_bruteforce(obst, a, b), (a, b)
            assert fwd == oracle.visible_dda(obst, b, a), (a, b)  # symmetry


def test_dda_matches_bruteforce_random_pairs_tiny():
    obst = workloads.tiny(1)
    H, W = obst.shape
    rng = np.random.default_rng(0)
    free = np.argwhere(obst == 0)
    for _ in range(4000):
        (ya, xa), (yb, xb) = free[rng.integers(len(free), size=2)]
        assert oracle.visible_dda(obst, (xa, ya), (xb, yb)) == oracle.visible_bruteforce(obst, (xa, ya), (xb, yb))


def test_open_grid_is_complete():
    obst = workloads.open_grid(7, 5)
    offsets, bytes_, cells = oracle.build_graph(obst, nthreads=2)
    n = len(cells)
    assert n == 35
    row_ptr, col = oracle.decode_csr(offsets, bytes_)
    assert int(row_ptr[-1]) == n * (n - 1)


def test_adjacency_symmetric_and_four_neighbours_visible():
    obst = workloads.tiny(3)
    offsets, bytes_, cells = oracle.build_graph(obst, nthreads=4)
    n = len(cells)
    row_ptr, col = oracle.decode_csr(offsets, bytes_)
    adj = [set(col[row_ptr[v]:row_ptr[v + 1]].tolist()) for v in range(n)]
    for v in range(n):
        assert v not in adj[v]
        for w in adj[v]:
            assert v in adj[w]
    W = obst.shape[1]
    node = {int(c): i for i, c in enumerate(cells)}
    for i, c in enumerate(cells):
        c = int(c)
        if c % W + 1 < W and (c + 1) in node:
            assert node[c + 1] in adj[i]
        if (c + W) in node:
            assert node[c + W] in adj[i]


def test_main_component_raster_numbering():
    obst = np.array([[0, 1, 0, 0],
                     [0, 1, 0, 0],
                     [1, 1, 0, 1]], np.uint8)
    node_of_cell, cells = oracle.main_component(obst)
    # right component has 5 cells, left 2: right wins; ids follow raster order
    assert cells.tolist() == [2, 3, 6, 7, 10]
    assert node_of_cell.tolist() == [-1, -1, 0, 1, -1, -1, 2, 3, -1, -1, 4, -1]


def test_tiny_config_sizes():
    # 32x32, 8 rectangles with sides 2..6: a few hundred thousand directed edges
    for seed in (1, 2, 3):
        offsets, bytes_, cells = oracle.build_graph(workloads.tiny(seed))
        n = len(cells)
        assert 700 < n < 1024
        row_ptr, _ = oracle.decode_csr(offsets, bytes_)
        assert 1e5 < int(row_ptr[-1]) < 1e6
