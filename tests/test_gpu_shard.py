"""GPU tests of register-range shards (vga_shard_*): one analysis split over
2-16 shards, run in lockstep in one process on one GPU (the arithmetic every
rank of a multi-GPU run does, with the all-gather done by placing the partial
blocks side by side), must give the unsharded run's iterations, mean depth
and ball sizes bit for bit -- for both union variants, 8- and 4-bit
registers, split hubs, both convergence rules and depth limits.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vga():
    from paper_2604_08374_gb300 import build
    build.build()
    import paper_2604_08374_gb300 as v
    return v


@pytest.fixture(scope="module")
def graphs(vga):
    out = {}
    for name, obst in (("tiny1", workloads.tiny(1)), ("tiny3", workloads.tiny(3)),
                       ("rect60", workloads.rectangles_until(60, 45, (2, 9), int(60 * 45 * 0.85), seed=9))):
        off, b, _ = oracle.build_graph(obst)
        out[name] = (vga.vga_graph_load(off, b), off, b)
    yield out
    for g, _, _ in out.values():
        g.free()


def _alone(vga, torch, g, p, d, seed, conv, **tuning):
    md = torch.empty(g.n_nodes, dtype=torch.float64, device="cuda")
    ball = torch.empty_like(md)
    it = vga.hyperball_run_dev(g, p, d, seed, md, ball, conv_mode=conv, **tuning)
    return it, md.cpu().numpy(), ball.cpu().numpy()


CASES = [
    ("tiny1", 8, 0, 2, 0, dict(slice_bytes=16)),
    ("tiny1", 8, 3, 5, 0, dict(slice_bytes=16, union_mode=1)),
    ("tiny3", 10, 0, 3, 1, dict(slice_bytes=64)),
    ("tiny3", 10, 0, 16, 0, dict(slice_bytes=64)),
    ("rect60", 6, 0, 4, 0, dict(slice_bytes=16)),
    ("rect60", 8, 0, 2, 0, dict(slice_bytes=16, register_bits=4)),
    ("tiny1", 10, 2, 4, 0, dict(slice_bytes=32, hub_lookups=3)),
    ("tiny3", 12, 3, 2, 0, dict()),
    # change tracking over each shard's own slices (forced in every pass from the second)
    ("tiny1", 8, 0, 3, 0, dict(slice_bytes=16, track_changes=2)),
    ("rect60", 8, 0, 2, 0, dict(slice_bytes=32, union_mode=1, track_changes=2)),
    ("tiny3", 10, 0, 4, 1, dict(slice_bytes=64, track_changes=2, hub_lookups=5)),
]


@pytest.mark.parametrize("name,p,d,shards,conv,tuning", CASES)
def test_sharded_equals_unsharded(vga, graphs, name, p, d, shards, conv, tuning):
    torch = pytest.importorskip("torch")
    from paper_2604_08374_gb300.sharded import hyperball_run_sharded_local
    g, off, b = graphs[name]
    seed = 1234567 + p
    it0, md0, ball0 = _alone(vga, torch, g, p, d, seed, conv, **tuning)
    md = torch.full((g.n_nodes,), -1.0, dtype=torch.float64, device="cuda")
    ball = torch.full_like(md, -1.0)
    it = hyperball_run_sharded_local(g, p, d, seed, shards, md, ball, conv_mode=conv, **tuning)
    assert it == it0
    assert np.array_equal(md.cpu().numpy(), md0, equal_nan=True)
    assert np.array_equal(ball.cpu().numpy(), ball0)


def test_sharded_against_oracle(vga, graphs):
    torch = pytest.importorskip("torch")
    from paper_2604_08374_gb300.sharded import hyperball_run_sharded_local
    g, off, b = graphs["tiny1"]
    md = torch.empty(g.n_nodes, dtype=torch.float64, device="cuda")
    ball = torch.empty_like(md)
    it = hyperball_run_sharded_local(g, 8, 0, 9, 3, md, ball, slice_bytes=16)
    ref = oracle.hyperball(off, b, 8, 0, seed=9)
    assert it == ref["iterations"]
    assert np.array_equal(md.cpu().numpy(), ref["mean_depth"], equal_nan=True)
    np.testing.assert_allclose(md.cpu().numpy(), ref["mean_depth"], rtol=1e-6)


def test_shard_layout_and_errors(vga, graphs):
    g, _, _ = graphs["tiny1"]
    shards = [vga.vga_shard_create(g, 8, 0, k, 3, slice_bytes=16) for k in range(3)]
    assert [s.slice_first for s in shards] == [0, 5, 10]
    assert [s.slice_count for s in shards] == [5, 5, 6]
    assert all(s.partial_bytes % 256 == 0 and s.partial_bytes >= 12 * g.n_nodes for s in shards)
    for s in shards:
        s.free()
    for args in ((0, 1), (2, 2), (-1, 2), (0, 17)):
        with pytest.raises(vga.VgaError) as e:
            vga.vga_shard_create(g, 8, 0, args[0], args[1], slice_bytes=16)
        assert e.value.status == vga.VGA_EINVAL


def test_sharded_automatic_tracking_medium(vga):
    # on the ~42.7k-cell workload the fifth pass is tracked by every shard and
    # the sharded run equals the unsharded one bit for bit
    torch = pytest.importorskip("torch")
    from paper_2604_08374_gb300.sharded import hyperball_run_sharded_local
    g = vga.vga_visibility_build(workloads.medium(seed=3))
    try:
        it0, md0, ball0 = _alone(vga, torch, g, 10, 0, 5, 0, slice_bytes=128)
        md = torch.empty(g.n_nodes, dtype=torch.float64, device="cuda")
        ball = torch.empty_like(md)
        vga.vga_profile_reset()
        vga.vga_profile_enable(True)
        try:
            it = hyperball_run_sharded_local(g, 10, 0, 5, 2, md, ball, slice_bytes=128)
            prof = vga.vga_profile_read()
        finally:
            vga.vga_profile_enable(False)
    finally:
        g.free()
    assert it == it0 >= 4
    assert prof["tracked_launches"] > 0
    assert np.array_equal(md.cpu().numpy(), md0, equal_nan=True)
    assert np.array_equal(ball.cpu().numpy(), ball0)
