"""GPU parity of change-tracked passes (vga_tuning.track_changes).

A tracked pass recomputes node v in slice s only if one of v's neighbours
changed slice s in the previous pass; every other node keeps its registers.
Forcing tracking in every pass from the second (track_changes = 2) must still
give the oracle's registers bit for bit after every pass, across both union
variants, both table schemes, slice widths, 8- and 4-bit registers, both
first-pass methods and split hubs; the automatic rule must track the late passes of unlimited-depth
runs and give the same results.
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


_cache = {}


def graph(name):
    if name not in _cache:
        if name.startswith("tiny"):
            obst = workloads.tiny(int(name[4:]))
        elif name == "rect96":
            obst = workloads.rectangles_until(96, 96, (2, 12), int(96 * 96 * 0.88), seed=4)
        elif name == "comb":
            obst = workloads.open_grid(33, 21)
            obst[2:19:2, 3:30] = 1
        elif name == "open40x30":
            obst = workloads.open_grid(40, 30)
        else:
            raise KeyError(name)
        off, b, _ = oracle.build_graph(obst)
        _cache[name] = (off, b)
    return _cache[name]


def assert_same_run(got, ref):
    assert got["iterations"] == ref["iterations"]
    for t in range(got["iterations"] + 1):
        assert np.array_equal(got["regs"][t], ref["regs"][t]), f"registers differ after pass {t}"
        assert np.array_equal(got["c"][t], ref["c"][t]), f"estimates differ after pass {t}"
    assert np.array_equal(got["mean_depth"], ref["mean_depth"], equal_nan=True)
    assert np.array_equal(got["ball"], ref["ball"])


CASES = [
    # graph, p, d, register bits, slice bytes, table levels, hub lookups, first pass
    ("tiny1", 10, 0, 8, 0, 0, 0, 0),
    ("tiny2", 10, 0, 8, 128, 3, 0, 1),
    ("tiny3", 8, 0, 8, 16, 5, 0, 2),
    ("tiny4", 12, 0, 8, 128, 3, 0, 0),
    ("tiny5", 9, 4, 4, 32, 5, 0, 0),
    ("tiny1", 8, 0, 8, 64, 3, 5, 2),
    ("tiny2", 10, 0, 4, 16, 3, 2, 1),
    ("comb", 8, 0, 8, 16, 3, 0, 0),
    ("open40x30", 8, 0, 8, 32, 5, 0, 2),
    ("rect96", 10, 0, 8, 128, 0, 0, 0),
]


@pytest.mark.parametrize("name,p,d,bits,S,levels,hub,first", CASES)
def test_tracked_every_pass_bit_exact(vga, name, p, d, bits, S, levels, hub, first):
    off, b = graph(name)
    T = 16
    ref = oracle.hyperball(off, b, p, d, seed=4242, trace=T, reg_bits=bits)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, p, d, seed=4242, max_trace=T, slice_bytes=S, union_mode=2,
                                      register_bits=0 if bits == 8 else bits, hub_lookups=hub, table_levels=levels,
                                      first_pass=first, track_changes=2)
    assert got["iterations"] <= T
    assert_same_run(got, ref)


@pytest.mark.parametrize("name,p,bits,S,first", [("tiny1", 10, 8, 0, 0), ("tiny3", 8, 8, 16, 1), ("comb", 8, 8, 32, 2),
                                                  ("tiny2", 10, 4, 16, 0), ("rect96", 10, 8, 128, 0)])
def test_tracked_per_neighbour(vga, name, p, bits, S, first):
    # the per-neighbour variant finds the nodes to recompute by decoding the CSR
    off, b = graph(name)
    ref = oracle.hyperball(off, b, p, 0, seed=99, trace=16, reg_bits=bits)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, p, 0, seed=99, max_trace=16, slice_bytes=S, union_mode=1,
                                      register_bits=0 if bits == 8 else bits, first_pass=first, track_changes=2)
    assert_same_run(got, ref)


def test_automatic_tracking_on_unlimited_depth(vga):
    # On the ~42.7k-cell workload the fourth pass changes about 0.3 % of the
    # (node, slice) pairs, so the automatic rule tracks the fifth; the run must
    # equal the untracked one bit for bit (which the other tests pin to the
    # oracle, as they pin forced tracking on small graphs).
    torch = pytest.importorskip("torch")
    g = vga.vga_visibility_build(workloads.medium(seed=3))
    try:
        n = g.n_nodes
        out = {}
        for track in (0, 1):
            md = torch.empty(n, dtype=torch.float64, device="cuda")
            ball = torch.empty_like(md)
            vga.vga_profile_reset()
            vga.vga_profile_enable(True)
            try:
                it = vga.hyperball_run_dev(g, 10, 0, 17, md, ball, union_mode=2, track_changes=track)
                prof = vga.vga_profile_read()
            finally:
                vga.vga_profile_enable(False)
            out[track] = (it, md.cpu().numpy(), ball.cpu().numpy(), prof)
    finally:
        g.free()
    (it0, md0, ball0, prof0), (it1, md1, ball1, prof1) = out[0], out[1]
    assert it0 == it1 >= 4
    assert prof0["tracked_launches"] > 0 and prof1["tracked_launches"] == 0
    assert np.array_equal(md0, md1, equal_nan=True)
    assert np.array_equal(ball0, ball1)


def test_tracking_off_when_not_possible_and_errors(vga):
    off, b = graph("tiny1")
    ref = oracle.hyperball(off, b, 12, 0, seed=3, trace=12)
    with vga.vga_graph_load(off, b) as g:
        # 256 slices of 16 bytes: more than the 32 a change mask holds; automatic
        # tracking stays off and the run is unchanged
        assert_same_run(vga.hyperball_run_trace(g, 12, 0, seed=3, max_trace=12, slice_bytes=16, union_mode=2), ref)
        for kw in (dict(p=12, slice_bytes=16, union_mode=2, track_changes=2),
                   dict(p=12, slice_bytes=16, union_mode=1, track_changes=2),
                   dict(p=10, union_mode=2, track_changes=3),
                   dict(p=10, union_mode=2, track_changes=-1)):
            p = kw.pop("p")
            with pytest.raises(vga.VgaError) as e:
                vga.hyperball_run_trace(g, p, 1, max_trace=1, **kw)
            assert e.value.status == vga.VGA_EINVAL


def _skewed_csr(n=9000, seed=8):
    rng = np.random.default_rng(seed)
    lists = []
    hubs = {0: 2, 4500: 3, 8999: 2}
    for v in range(n):
        if v in hubs:
            ids = np.arange(1 if v == 0 else 0, n, hubs[v])
        else:
            starts = rng.integers(0, n - 20, size=3)
            ids = np.unique(np.concatenate([np.arange(s, s + rng.integers(1, 20)) for s in starts]))
        ids = ids[ids != v]
        lists.append(ids.astype(np.uint32))
    row_ptr = np.zeros(n + 1, np.uint64)
    row_ptr[1:] = np.cumsum([len(x) for x in lists])
    return oracle.csr_encode(row_ptr, np.concatenate(lists))


@pytest.mark.parametrize("hub", [0, 700])
def test_tracked_split_hubs(vga, hub):
    # hub chunks that keep their registers merge cur[v] by atomic max beside
    # chunks of the same hub that recompute
    off, b = _skewed_csr()
    ref = oracle.hyperball(off, b, 8, 0, seed=5, trace=20)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, 8, 0, seed=5, max_trace=20, slice_bytes=16, union_mode=2, hub_lookups=hub,
                                      track_changes=2)
    assert got["iterations"] <= 20
    assert_same_run(got, ref)
