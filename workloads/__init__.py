"""Seeded synthetic obstacle grids: the inputs of every test and benchmark.

This module serves both the CPU oracle and the CUDA library.  It holds none of
the method's arithmetic: it only decides which grid cells are obstacles.
Visibility, node numbering, the compressed CSR and HyperBall are computed by
each side on its own.

The paper measures on OpenStreetMap building footprints of Valdivia, Chile,
rasterised at 3-20 m spacing (Sec. 4.1); that data is not available here.
These generators stand in for it with axis-aligned rectangular obstacles whose
sizes and densities follow the paper's workloads (cell counts and edge counts
of the edge-density table in Sec. 4.3):

  tiny    32 x 32 grid, 8 rectangles with sides uniform in 2..6 cells;
  medium  220 x 220 grid, sides uniform in 2..20, added until the main
          component is about 42,700 cells (about 12 % cover);
  city    520 x 520 grid of urban blocks with sides uniform in 8..40 cells on a
          jittered street lattice, some slots left open as plazas, about
          236,000 free cells and 4-5e9 directed visibility edges;
  batch   256 grids of 1,000-30,000 free cells (log-uniform), mixed p and d;
  serve   a pool of 64 grids of 1,000-236,000 free cells and a Poisson stream
          of (graph, p, d) requests.

All randomness comes from numpy's PCG64 ``default_rng(seed)``; a rectangle's
top-left corner is uniform over the positions that keep it inside the grid,
and rectangles may overlap.  The grid is an ``uint8`` array of shape (H, W),
row-major (row = y), 1 = obstacle.
"""
from __future__ import annotations

import numpy as np

TINY = dict(W=32, H=32, n_rect=8, side=(2, 6))
MEDIUM = dict(W=220, H=220, side=(2, 20), target_free=42_700)
CITY = dict(W=520, H=520, side=(8, 40), pitch=56, street=6, block_free=239_500, n_small=700, small_side=(1, 3))


def _place(rng, grid, w, h, x0_range, y0_range):
    x0 = int(rng.integers(x0_range[0], x0_range[1] + 1))
    y0 = int(rng.integers(y0_range[0], y0_range[1] + 1))
    grid[y0:y0 + h, x0:x0 + w] = 1


def random_rectangles(W: int, H: int, n_rect: int, side=(2, 6), seed: int = 0) -> np.ndarray:
    """n_rect rectangles with integer sides uniform in [side[0], side[1]]."""
    rng = np.random.default_rng(seed)
    grid = np.zeros((H, W), np.uint8)
    for _ in range(n_rect):
        w = int(rng.integers(side[0], min(side[1], W) + 1))
        h = int(rng.integers(side[0], min(side[1], H) + 1))
        _place(rng, grid, w, h, (0, W - w), (0, H - h))
    return grid


def rectangles_until(W: int, H: int, side, target_free: int, seed: int = 0) -> np.ndarray:
    """Add rectangles until at most target_free cells remain free."""
    rng = np.random.default_rng(seed)
    grid = np.zeros((H, W), np.uint8)
    free = W * H
    while free > target_free:
        w = int(rng.integers(side[0], min(side[1], W) + 1))
        h = int(rng.integers(side[0], min(side[1], H) + 1))
        _place(rng, grid, w, h, (0, W - w), (0, H - h))
        free = W * H - int(grid.sum())
    return grid


def tiny(seed: int = 1) -> np.ndarray:
    """32 x 32 grid, 8 rectangles with sides 2..6 (expect N ~ 850)."""
    return random_rectangles(TINY["W"], TINY["H"], TINY["n_rect"], TINY["side"], seed)


def medium(seed: int = 0) -> np.ndarray:
    """220 x 220 grid, sides 2..20, rectangles added until <= 42,700 free cells."""
    return rectangles_until(MEDIUM["W"], MEDIUM["H"], MEDIUM["side"], MEDIUM["target_free"], seed)


def city(seed: int = 0, W: int = CITY["W"], H: int = CITY["H"], pitch: int = CITY["pitch"],
         street: int = CITY["street"], side=CITY["side"], block_free: int = CITY["block_free"],
         n_small: int = CITY["n_small"], small_side=CITY["small_side"]) -> np.ndarray:
    """Urban blocks on a jittered street lattice, plus small street obstacles.

    The grid is cut into square slots of `pitch` cells; a slot receives at most
    one block with sides uniform in `side` (capped at pitch - street, so a
    street of at least `street` cells separates neighbouring slots' blocks),
    placed uniformly inside the slot.  Slots are visited in a seeded random
    order and filled until at most `block_free` cells remain free; the slots
    left empty are the open plazas.  Then `n_small` small obstacles (sides
    uniform in `small_side`: kiosks, trees, street furniture) are dropped
    uniformly over the grid.  Blocks alone leave sight lines long enough for
    about 1e10 directed edges at this cover; the small obstacles bring the
    graph to the 4-5e9 edges of the paper's 235,983-cell workload while
    adding under 1 % cover."""
    rng = np.random.default_rng(seed)
    grid = np.zeros((H, W), np.uint8)
    nx, ny = W // pitch, H // pitch
    ox, oy = (W - nx * pitch) // 2, (H - ny * pitch) // 2
    order = rng.permutation(nx * ny)
    cap = pitch - street
    free = W * H
    for s in order:
        if free <= block_free:
            break
        sx, sy = int(s % nx), int(s // nx)
        w = int(rng.integers(side[0], min(side[1], cap) + 1))
        h = int(rng.integers(side[0], min(side[1], cap) + 1))
        x_lo = ox + sx * pitch + street // 2
        y_lo = oy + sy * pitch + street // 2
        _place(rng, grid, w, h, (x_lo, x_lo + cap - w), (y_lo, y_lo + cap - h))
        free = W * H - int(grid.sum())
    for _ in range(n_small):
        w = int(rng.integers(small_side[0], small_side[1] + 1))
        h = int(rng.integers(small_side[0], small_side[1] + 1))
        _place(rng, grid, w, h, (0, W - w), (0, H - h))
    return grid


def open_grid(W: int, H: int) -> np.ndarray:
    """No obstacles: the visibility graph is complete."""
    return np.zeros((H, W), np.uint8)


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int = 0) -> np.ndarray:
    """Free-cell targets log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=count)).astype(np.int64)


def grid_for_free_cells(target_free: int, seed: int = 0, cover: float = 0.12, side=(2, 20)) -> np.ndarray:
    """Square grid sized so that about `target_free` cells stay free at the
    given cover, filled like the medium workload (sides 2..20)."""
    side_len = int(np.ceil(np.sqrt(target_free / (1.0 - cover))))
    return rectangles_until(side_len, side_len, side, target_free, seed)


def batch(count: int = 256, seed: int = 0):
    """Batched workload: `count` grids with free cells log-uniform in 1,000-30,000
    (medium-style generator, per-graph seed = seed + i), each with p uniform
    over {8, 10, 12} and d uniform over {3, unlimited (0)}.  Returns a list of
    dicts (grid, p, d)."""
    sizes = log_uniform_sizes(count, 1_000, 30_000, seed)
    rng = np.random.default_rng(seed + 1)
    return [dict(grid=grid_for_free_cells(int(n), seed=seed + i), p=int(rng.choice([8, 10, 12])),
                 d=int(rng.choice([3, 0]))) for i, n in enumerate(sizes)]


def serve_pool(count: int = 64, seed: int = 0):
    """Serving pool: `count` grids with free cells log-uniform in 1,000-236,000
    (medium-style generator, per-graph seed = seed + 1000 + i)."""
    sizes = log_uniform_sizes(count, 1_000, 236_000, seed)
    return [grid_for_free_cells(int(n), seed=seed + 1000 + i) for i, n in enumerate(sizes)]


def serve_requests(count: int, pool_size: int, rate: float, seed: int = 0):
    """Poisson arrivals at `rate` per second: (arrival_s, graph index, p, d)
    with graph uniform over the pool, p uniform over {8, 10, 12}, d uniform
    over {3, 5, unlimited (0)}."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    return [(float(t[k]), int(rng.integers(pool_size)), int(rng.choice([8, 10, 12])), int(rng.choice([3, 5, 0])))
            for k in range(count)]
