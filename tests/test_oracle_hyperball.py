"""Pins for the oracle's HyperBall (Eq. hll-union, Eq. hbidentity, Eq. sumD,
Alg. 1) against exact BFS on small graphs.

- Closed form: after t passes node v's registers equal the register-wise max of
  the initial counters of every u in the exact ball B(v, t).
- Registers never decrease; each node's counter dominates its own initial one.
- At convergence every node of the (single) component holds the same registers.
- Iteration count: with no depth limit the run stops at the first pass that
  changes nothing, never later than eccentricity + 1; with a limit d it runs
  min(d, that) passes.
- Eq. sumD fed with exact ball sizes reproduces the exact distance sums of
  Eq. hbidentity (integers, so exactly).
- HLL ball estimates against exact |B(v,t)|: RMS relative error within 1.5x
  the standard error 1.04/sqrt(m) (Sec. 2.3).
- Mean depth against exact BFS mean depth: median relative error of a few
  percent at p = 10 (the paper reports 1.7 % against depthmapX, Sec. 4.2).
"""
import math

import numpy as np
import pytest

import oracle
import workloads


def _graph(seed=1, grid=None):
    obst = workloads.tiny(seed) if grid is None else grid
    offsets, b, cells = oracle.build_graph(obst)
    return offsets, b, len(cells)


def _all_dist(offsets, b, n):
    return np.stack([oracle.bfs(offsets, b, s)[0] for s in range(n)])


@pytest.fixture(scope="module")
def tiny1():
    offsets, b, n = _graph(1)
    return offsets, b, n, _all_dist(offsets, b, n)


@pytest.mark.parametrize("p", [4, 8, 10])
def test_registers_closed_form_every_pass(tiny1, p):
    offsets, b, n, dist = tiny1
    out = oracle.hyperball(offsets, b, p, d=0, seed=3, trace=12)
    regs = out["regs"]
    R0 = oracle.hll_init(n, p, 3)
    assert np.array_equal(regs[0], R0)
    for t in range(1, out["iterations"] + 1):
        for v in range(0, n, 7):
            ball = np.flatnonzero((dist[v] >= 0) & (dist[v] <= t))
            assert np.array_equal(regs[t][v], R0[ball].max(axis=0)), (t, v)


def test_monotone_and_fixed_point(tiny1):
    offsets, b, n, dist = tiny1
    p = 8
    out = oracle.hyperball(offsets, b, p, d=0, seed=0, trace=12)
    regs = out["regs"]
    T = out["iterations"]
    for t in range(1, T + 1):
        assert np.all(regs[t] >= regs[t - 1])
    assert np.all(regs[T] == regs[T][0])
    assert np.array_equal(regs[T][0], regs[0].max(axis=0))
    ecc_max = int(dist.max())
    # first pass that changes nothing, at most one past the largest eccentricity
    first_still = next(t for t in range(1, T + 1) if np.array_equal(regs[t], regs[t - 1]))
    assert T == first_still <= ecc_max + 1


@pytest.mark.parametrize("d", [1, 2, 3, 50])
def test_depth_limit(tiny1, d):
    offsets, b, n, _ = tiny1
    full = oracle.hyperball(offsets, b, 10, d=0)["iterations"]
    assert oracle.hyperball(offsets, b, 10, d=d)["iterations"] == min(d, full)


def test_paper_convergence_rule_stops_no_later(tiny1):
    offsets, b, n, _ = tiny1
    a = oracle.hyperball(offsets, b, 10, d=0, conv_mode=0, trace=12)
    c = oracle.hyperball(offsets, b, 10, d=0, conv_mode=1, trace=12)
    assert c["iterations"] <= a["iterations"]
    T = c["iterations"]
    inc = c["c"][T] - c["c"][T - 1]
    assert inc.max() <= 0.5
    for t in range(1, T):
        assert (c["c"][t] - c["c"][t - 1]).max() > 0.5


def test_sumd_with_exact_balls_gives_exact_distance_sums(tiny1):
    offsets, b, n, dist = tiny1
    D = int(dist.max())
    for v in range(0, n, 5):
        sum_d = 0.0
        prev = 1.0
        for t in range(1, D + 1):
            ball = float(np.count_nonzero((dist[v] >= 0) & (dist[v] <= t)))
            sum_d = oracle.accumulate(sum_d, t, ball, prev)
            prev = ball
        assert sum_d == float(dist[v][dist[v] > 0].sum())


@pytest.mark.parametrize("seed", [1, 2, 4])
def test_ball_estimates_within_standard_error(seed):
    offsets, b, n = _graph(seed)
    dist = _all_dist(offsets, b, n)
    p = 10
    out = oracle.hyperball(offsets, b, p, d=3, trace=3)
    errs = []
    for t in range(1, out["iterations"] + 1):
        exact = ((dist >= 0) & (dist <= t)).sum(axis=1)
        errs.append(out["c"][t] / exact - 1)
    errs = np.concatenate(errs)
    assert math.sqrt(np.mean(errs ** 2)) < 1.5 * 1.04 / math.sqrt(1 << p)


def test_mean_depth_against_exact_bfs(tiny1):
    offsets, b, n, dist = tiny1
    out = oracle.hyperball(offsets, b, 10, d=0)
    exact_md = dist.sum(axis=1) / (n - 1)
    rel = np.abs(out["mean_depth"] / exact_md - 1)
    assert np.median(rel) < 0.05
    # ball size at convergence estimates the component size
    assert abs(np.median(out["ball"]) / n - 1) < 3 * 1.04 / 32


def test_mean_depth_denominator_uses_component_size(tiny1):
    offsets, b, n, _ = tiny1
    a = oracle.hyperball(offsets, b, 8, d=2)
    cs = np.full(n, 2 * n, np.uint32)
    c = oracle.hyperball(offsets, b, 8, d=2, comp_size=cs)
    assert np.allclose(a["mean_depth"] * (n - 1), c["mean_depth"] * (2 * n - 1), rtol=1e-12)


def test_degenerate_graphs():
    # single node: no neighbours, mean depth undefined
    offsets = np.array([0, 0], np.uint64)
    out = oracle.hyperball(offsets, np.zeros(0, np.uint8), 10, d=0)
    assert out["iterations"] == 1
    assert math.isnan(out["mean_depth"][0])
    # two nodes: mean depth 1 exactly in the linear-counting regime is not exact,
    # but the ball estimate after one pass is m ln(m/(m-2)) when the two hashes
    # land in different registers
    offsets, b, cells = oracle.build_graph(np.zeros((1, 2), np.uint8))
    out = oracle.hyperball(offsets, b, 10, d=0)
    m = 1024
    j0, _ = oracle.hll_hash(0, 0, 10)
    j1, _ = oracle.hll_hash(1, 0, 10)
    assert j0 != j1
    assert out["ball"][0] == pytest.approx(m * math.log(m / (m - 2)), rel=1e-15)
    assert out["iterations"] == 2
    # empty graph
    out = oracle.hyperball(np.zeros(1, np.uint64), np.zeros(0, np.uint8), 10, d=3)
    assert out["iterations"] == 0 and len(out["mean_depth"]) == 0


@pytest.mark.parametrize("p", [5, 8, 10])
def test_four_bit_registers_are_the_clamped_eight_bit_ones(tiny1, p):
    # The 4-bit format (Sec. 3.3) clamps rho to 15.  Clamping commutes with
    # the register-wise max, so after every pass the 4-bit registers must be
    # the 8-bit ones clamped to 15 -- as long as the clamp never changes
    # whether a pass changed anything, which the pass counts also check.
    offsets, b, n, dist = tiny1
    seed = 11
    r8 = oracle.hyperball(offsets, b, p, 3, seed=seed, trace=3)
    r4 = oracle.hyperball(offsets, b, p, 3, seed=seed, trace=3, reg_bits=4)
    for t in range(r4["iterations"] + 1):
        assert np.array_equal(r4["regs"][t], np.minimum(r8["regs"][t], 15))
        assert r4["regs"][t].max() <= 15
    # BFS closed form with clamped initial counters
    R0 = oracle.hll_init(n, p, seed, reg_bits=4)
    for v in range(0, n, 11):
        ball = np.flatnonzero((dist[v] >= 0) & (dist[v] <= 2))
        assert np.array_equal(r4["regs"][2][v], R0[ball].max(axis=0))


def test_four_bit_clamp_is_hit_with_large_ids():
    # a node whose rho exceeds 15 must come out as 15
    import itertools
    p = 10
    for v in itertools.count():
        j, rho = oracle.hll_hash(v, 0, p)
        if rho > 15:
            break
    regs = oracle.hll_init(v + 1, p, 0, reg_bits=4)
    assert regs[v, j] == 15
    assert oracle.hll_init(v + 1, p, 0)[v, j] == rho
