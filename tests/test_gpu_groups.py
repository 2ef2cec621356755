"""GPU parity of the grouped run-aware union (vga_tuning.group_nodes).

Groups of 2, 4 or 8 consecutive nodes gather each distinct table row of their
merged lookup lists once and fold it, class by class, into the nodes whose
lists hold it.  The registers must equal the oracle's (Alg. 1, Eq. hll-union)
bit for bit after every pass, for every group size and with one node per warp
(group_nodes = 1), across slice widths from 16 to 1024 bytes (both lane
shapes of the lean gather), both table schemes, 8- and 4-bit registers, split
hubs (which stay per node beside the groups), change-tracked passes (a group
is recomputed when any of its nodes needs it), ragged last groups, graphs with
isolated nodes, and register shards.
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
        elif name == "open1x301":  # one grid row: 301 nodes, a ragged last group for 2, 4 and 8
            obst = workloads.open_grid(301, 1)
        elif name == "sparse":  # scattered obstacles: short runs, many classes per group
            rng = np.random.default_rng(11)
            obst = (rng.random((41, 37)) < 0.3).astype(np.uint8)
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
    ("tiny2", 10, 3, 8, 128, 3, 0, 1),
    ("tiny3", 8, 0, 8, 16, 5, 0, 2),
    ("tiny4", 12, 2, 8, 1024, 5, 0, 1),
    ("tiny5", 9, 0, 4, 32, 3, 0, 0),
    ("tiny1", 10, 0, 4, 256, 5, 0, 1),
    ("tiny2", 8, 0, 8, 64, 3, 7, 1),
    ("comb", 8, 0, 8, 16, 3, 0, 0),
    ("open1x301", 6, 0, 8, 64, 5, 0, 1),
    ("sparse", 10, 0, 8, 512, 3, 0, 1),
    ("rect96", 10, 0, 8, 128, 0, 0, 0),
]


@pytest.mark.parametrize("nodes", [1, 2, 4, 8])
@pytest.mark.parametrize("name,p,d,bits,S,levels,hub,first", CASES)
def test_grouped_union_bit_exact(vga, name, p, d, bits, S, levels, hub, first, nodes):
    off, b = graph(name)
    T = 16
    ref = oracle.hyperball(off, b, p, d, seed=77, trace=T, reg_bits=bits)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, p, d, seed=77, max_trace=T, slice_bytes=S, union_mode=2,
                                      register_bits=0 if bits == 8 else bits, hub_lookups=hub, table_levels=levels,
                                      first_pass=first, group_nodes=nodes)
    assert got["iterations"] <= T
    assert_same_run(got, ref)


@pytest.mark.parametrize("nodes", [2, 4, 8])
@pytest.mark.parametrize("warps", [1, 3, 16])
def test_grouped_union_cta_sizes(vga, nodes, warps):
    # 16 warps of 8 groups of 1024-byte rows need more than 48 KB of shared memory
    off, b = graph("tiny3")
    ref = oracle.hyperball(off, b, 10, 0, seed=5, trace=12)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, 10, 0, seed=5, max_trace=12, slice_bytes=1024, warps_per_cta=warps,
                                      union_mode=2, group_nodes=nodes)
    assert_same_run(got, ref)


@pytest.mark.parametrize("nodes", [2, 4, 8])
@pytest.mark.parametrize("name,S,levels,hub,bits", [("tiny1", 0, 0, 0, 8), ("tiny2", 32, 3, 3, 8),
                                                     ("rect96", 128, 0, 0, 8), ("tiny4", 32, 5, 0, 4)])
def test_grouped_union_tracked_every_pass(vga, nodes, name, S, levels, hub, bits):
    off, b = graph(name)
    ref = oracle.hyperball(off, b, 10, 0, seed=31, trace=16, reg_bits=bits)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, 10, 0, seed=31, max_trace=16, slice_bytes=S, union_mode=2,
                                      register_bits=0 if bits == 8 else bits, table_levels=levels, hub_lookups=hub,
                                      track_changes=2, group_nodes=nodes)
    assert_same_run(got, ref)


@pytest.mark.parametrize("nodes", [2, 4, 8])
def test_grouped_union_split_hubs_skewed(vga, nodes):
    # hubs of 4000-6000 lookups split under the automatic threshold; their
    # chunks run per node beside the groups of the other nodes
    from test_gpu_parity import _skewed_csr
    off, b = _skewed_csr()
    ref = oracle.hyperball(off, b, 8, 3, seed=9, trace=3)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, 8, 3, seed=9, max_trace=3, union_mode=2, group_nodes=nodes)
    assert_same_run(got, ref)


def test_grouped_union_isolated_nodes_and_components(vga):
    # two walled-off rooms and single free cells between obstacles: nodes with
    # empty lists sit inside groups
    obst = workloads.open_grid(23, 17)
    obst[:, 11] = 1
    obst[8, :] = 1
    obst[3, 3] = obst[3, 5] = obst[2, 4] = obst[4, 4] = 1
    _, cells = oracle.main_component(obst)
    off, b, _ = oracle.build_graph(obst)
    ref = oracle.hyperball(off, b, 8, 0, seed=2, trace=12)
    with vga.vga_graph_load(off, b) as g:
        for nodes in (2, 4, 8):
            got = vga.hyperball_run_trace(g, 8, 0, seed=2, max_trace=12, union_mode=2, group_nodes=nodes)
            assert_same_run(got, ref)


def test_grouped_union_rejects_bad_size(vga):
    off, b = graph("tiny1")
    with vga.vga_graph_load(off, b) as g:
        for bad in (3, 5, 9, -1):
            with pytest.raises(vga.VgaError):
                vga.hyperball_run_trace(g, 8, 1, max_trace=1, union_mode=2, group_nodes=bad)


@pytest.mark.parametrize("nodes", [2, 4, 8])
def test_grouped_union_register_shards(vga, nodes):
    torch = pytest.importorskip("torch")
    from paper_2604_08374_gb300.sharded import hyperball_run_sharded_local
    off, b = graph("tiny2")
    ref = oracle.hyperball(off, b, 10, 0, seed=8)
    with vga.vga_graph_load(off, b) as g:
        md = torch.empty(g.n_nodes, dtype=torch.float64, device="cuda")
        ball = torch.empty_like(md)
        it = hyperball_run_sharded_local(g, 10, 0, 8, 4, md, ball, slice_bytes=128, union_mode=2,
                                         group_nodes=nodes)
        torch.cuda.synchronize()
    assert it == ref["iterations"]
    assert np.array_equal(md.cpu().numpy(), ref["mean_depth"], equal_nan=True)
    assert np.array_equal(ball.cpu().numpy(), ref["ball"])


# ----------------------------------------------------------------------------
# groups from the grid geometry (2 x 1, 2 x 2, 4 x 2 blocks of cells)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("order", ["raster", "hilbert"])
@pytest.mark.parametrize("name", ["tiny3", "rect96", "sparse", "open1x301"])
def test_groups_from_cell_blocks(vga, name, order):
    # graphs from the builder carry their cells, so their groups are blocks of
    # cells; the same CSR loaded without geometry groups consecutive ids, and
    # with vga_graph_set_cells blocks again: all must equal the oracle
    if name.startswith("tiny"):
        obst = workloads.tiny(int(name[4:]))
    elif name == "rect96":
        obst = workloads.rectangles_until(96, 96, (2, 12), int(96 * 96 * 0.88), seed=4)
    elif name == "open1x301":
        obst = workloads.open_grid(301, 1)
    else:
        rng = np.random.default_rng(11)
        obst = (rng.random((41, 37)) < 0.3).astype(np.uint8)
    H, W = obst.shape
    off, b, cells = oracle.build_graph(obst, order=order)
    ref = oracle.hyperball(off, b, 10, 0, seed=12, trace=16)
    g_built, gcells = vga.vga_visibility_build(obst, return_cells=True, order=order)
    with g_built as g1, vga.vga_graph_load(off, b) as g2:
        assert np.array_equal(gcells.astype(np.int64), cells)
        for nodes in (2, 4, 8):
            assert_same_run(vga.hyperball_run_trace(g1, 10, 0, seed=12, max_trace=16, union_mode=2,
                                                    group_nodes=nodes), ref)
            assert_same_run(vga.hyperball_run_trace(g2, 10, 0, seed=12, max_trace=16, union_mode=2,
                                                    group_nodes=nodes), ref)
        g2.set_cells(W, H, cells)
        for nodes in (2, 4, 8):
            assert_same_run(vga.hyperball_run_trace(g2, 10, 0, seed=12, max_trace=16, union_mode=2,
                                                    group_nodes=nodes, hub_lookups=3 if nodes == 4 else 0), ref)
        g2.set_cells(W, H, None)
        assert_same_run(vga.hyperball_run_trace(g2, 10, 0, seed=12, max_trace=16, union_mode=2), ref)


def test_set_cells_rejects_bad_maps(vga):
    obst = workloads.tiny(1)
    H, W = obst.shape
    off, b, cells = oracle.build_graph(obst)
    with vga.vga_graph_load(off, b) as g:
        bad = cells.copy()
        bad[5] = bad[4]  # a cell used twice
        with pytest.raises(vga.VgaError):
            g.set_cells(W, H, bad)
        bad = cells.copy()
        bad[0] = W * H  # outside the grid
        with pytest.raises(vga.VgaError):
            g.set_cells(W, H, bad)
        with pytest.raises(vga.VgaError):
            g.set_cells(0, H, cells)
        g.set_cells(W, H, cells)  # a valid map is accepted
