"""GPU parity of the first pass computed as a scatter (vga_tuning.first_pass).

After the initialisation of Algorithm 1 every counter holds one register, so
pass 1 of Eq. hll-union can fold the neighbours' hashes straight into per-warp
register cells instead of gathering register rows.  Both ways must give the
oracle's registers bit for bit after every pass (the later passes start from
the scattered registers), across p = 4 .. 13, both table schemes, 8- and 4-bit
registers, slice widths from 16 to 1024 bytes, split hubs and register-range
shards, in both union variants (the per-neighbour one decodes the CSR for the
scatter); p above 13 falls back to the gather.
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


def tiny_graph(seed):
    if seed not in _cache:
        off, b, cells = oracle.build_graph(workloads.tiny(seed))
        _cache[seed] = (off, b, cells)
    return _cache[seed]


def assert_same_run(got, ref):
    assert got["iterations"] == ref["iterations"]
    for t in range(got["iterations"] + 1):
        assert np.array_equal(got["regs"][t], ref["regs"][t]), f"registers differ after pass {t}"
        assert np.array_equal(got["c"][t], ref["c"][t]), f"estimates differ after pass {t}"
    assert np.array_equal(got["mean_depth"], ref["mean_depth"], equal_nan=True)
    assert np.array_equal(got["ball"], ref["ball"])


CASES = [
    # seed, p, d, register bits, slice bytes, table levels, hub lookups
    (1, 10, 3, 8, 0, 0, 0),
    (2, 10, 0, 8, 128, 3, 0),
    (3, 10, 0, 8, 64, 5, 0),
    (1, 4, 0, 8, 16, 5, 0),
    (2, 5, 0, 4, 16, 3, 0),
    (3, 8, 2, 8, 256, 3, 7),
    (4, 12, 3, 8, 1024, 3, 0),
    (5, 13, 2, 8, 0, 5, 0),
    (1, 13, 1, 4, 512, 3, 0),
    (2, 10, 0, 4, 64, 5, 3),
    (3, 9, 0, 8, 32, 3, 1),
]


@pytest.mark.parametrize("seed,p,d,bits,S,levels,hub", CASES)
def test_first_pass_scatter_bit_exact(vga, seed, p, d, bits, S, levels, hub):
    off, b, _ = tiny_graph(seed)
    T = 12
    ref = oracle.hyperball(off, b, p, d, seed=seed * 131 + 7, trace=T, reg_bits=bits)
    with vga.vga_graph_load(off, b) as g:
        for first in (2, 1):
            got = vga.hyperball_run_trace(g, p, d, seed=seed * 131 + 7, max_trace=T, slice_bytes=S, union_mode=2,
                                          register_bits=0 if bits == 8 else bits, hub_lookups=hub,
                                          table_levels=levels, first_pass=first)
            assert_same_run(got, ref)


@pytest.mark.parametrize("grid", ["open40x30", "open1x300", "comb"])
@pytest.mark.parametrize("levels", [3, 5])
def test_first_pass_long_runs(vga, grid, levels):
    # complete graphs (lists of one or two runs up to N-1 ids: windows of every
    # width, the last window of a run overlapping the one before) and a comb of
    # walls (many short runs)
    if grid == "open40x30":
        obst = workloads.open_grid(40, 30)
    elif grid == "open1x300":
        obst = workloads.open_grid(300, 1)
    else:
        obst = workloads.open_grid(33, 21)
        obst[2:19:2, 3:30] = 1
    off, b, _ = oracle.build_graph(obst)
    ref = oracle.hyperball(off, b, 10, 0, seed=21, trace=6)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, 10, 0, seed=21, max_trace=6, union_mode=2, table_levels=levels,
                                      first_pass=2)
    assert_same_run(got, ref)


def _skewed_csr(n=9000, seed=4):
    """Hubs that see every second or third node (single-id runs) beside nodes
    with a few short runs."""
    rng = np.random.default_rng(seed)
    lists = []
    hubs = {0: 2, 4500: 3, 8999: 2}
    for v in range(n):
        if v in hubs:
            ids = np.arange(1 if v == 0 else 0, n, hubs[v])
        else:
            starts = rng.integers(0, n - 20, size=5)
            ids = np.unique(np.concatenate([np.arange(s, s + rng.integers(1, 20)) for s in starts]))
        ids = ids[ids != v]
        lists.append(ids.astype(np.uint32))
    row_ptr = np.zeros(n + 1, np.uint64)
    row_ptr[1:] = np.cumsum([len(x) for x in lists])
    return oracle.csr_encode(row_ptr, np.concatenate(lists))


@pytest.mark.parametrize("hub", [0, 500, 2048])
def test_first_pass_split_hubs(vga, hub):
    # the hubs' chunks merge into next[v] by word-wise atomic max
    off, b = _skewed_csr()
    ref = oracle.hyperball(off, b, 10, 2, seed=3, trace=2)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, 10, 2, seed=3, max_trace=2, union_mode=2, hub_lookups=hub, first_pass=2)
    assert_same_run(got, ref)


def test_first_pass_isolated_and_tiny_graphs(vga):
    # nodes without neighbours keep their own counter and raise no change flag;
    # a graph whose every node is isolated converges after one pass
    for obst in (workloads.open_grid(1, 1), workloads.open_grid(2, 1), workloads.open_grid(3, 3)):
        off, b, _ = oracle.build_graph(obst)
        ref = oracle.hyperball(off, b, 8, 0, seed=1, trace=4)
        with vga.vga_graph_load(off, b) as g:
            got = vga.hyperball_run_trace(g, 8, 0, seed=1, max_trace=4, union_mode=2, first_pass=2)
        assert_same_run(got, ref)
    row_ptr = np.zeros(6, np.uint64)
    off, b = oracle.csr_encode(row_ptr, np.zeros(0, np.uint32))
    ref = oracle.hyperball(off, b, 8, 0, seed=1, trace=3)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, 8, 0, seed=1, max_trace=3, union_mode=2, first_pass=2)
    assert got["iterations"] == ref["iterations"] == 1
    assert_same_run(got, ref)


@pytest.mark.parametrize("seed,p,d,bits,S", [(1, 4, 0, 8, 16), (2, 8, 0, 8, 64), (3, 10, 3, 8, 0), (4, 12, 2, 8, 256),
                                              (5, 13, 1, 8, 0), (1, 10, 0, 4, 32), (2, 6, 0, 4, 16)])
def test_first_pass_scatter_per_neighbour(vga, seed, p, d, bits, S):
    # the per-neighbour variant decodes the CSR itself for the scatter
    off, b, _ = tiny_graph(seed)
    ref = oracle.hyperball(off, b, p, d, seed=seed * 17 + 3, trace=12, reg_bits=bits)
    with vga.vga_graph_load(off, b) as g:
        for first in (2, 1):
            got = vga.hyperball_run_trace(g, p, d, seed=seed * 17 + 3, max_trace=12, slice_bytes=S, union_mode=1,
                                          register_bits=0 if bits == 8 else bits, first_pass=first)
            assert_same_run(got, ref)


def test_first_pass_fallbacks_and_errors(vga):
    off, b, _ = tiny_graph(2)
    ref = oracle.hyperball(off, b, 14, 2, seed=8, trace=2)
    with vga.vga_graph_load(off, b) as g:
        # p = 14 takes the gather for pass 1 in both variants
        assert_same_run(vga.hyperball_run_trace(g, 14, 2, seed=8, max_trace=2, union_mode=2), ref)
        assert_same_run(vga.hyperball_run_trace(g, 14, 2, seed=8, max_trace=2, union_mode=1), ref)
        for kw in (dict(p=14, union_mode=2, first_pass=2), dict(p=14, union_mode=1, first_pass=2),
                   dict(p=10, union_mode=2, first_pass=3), dict(p=10, union_mode=2, first_pass=-1)):
            p = kw.pop("p")
            with pytest.raises(vga.VgaError) as e:
                vga.hyperball_run_trace(g, p, 1, max_trace=1, **kw)
            assert e.value.status == vga.VGA_EINVAL


def test_first_pass_profile_counters(vga):
    # the scatter is timed apart from the union slices: one launch per run
    torch = pytest.importorskip("torch")
    off, b, _ = tiny_graph(3)
    with vga.vga_graph_load(off, b) as g:
        md = torch.empty(g.n_nodes, dtype=torch.float64, device="cuda")
        ball = torch.empty_like(md)
        vga.vga_profile_reset()
        vga.vga_profile_enable(True)
        try:
            it = vga.hyperball_run_dev(g, 10, 3, 0, md, ball, slice_bytes=128, union_mode=2, first_pass=2)
            prof = vga.vga_profile_read()
        finally:
            vga.vga_profile_enable(False)
        edges = g.n_edges
    assert it >= 2
    assert prof["first_pass_launches"] == 1 and prof["first_pass_ms"] > 0
    assert prof["first_pass_edges"] == edges
    assert prof["union_launches"] == (it - 1) * (1024 // 128)


@pytest.mark.parametrize("shards,S,bits", [(2, 16, 8), (3, 64, 8), (4, 16, 4)])
def test_first_pass_on_register_shards(vga, shards, S, bits):
    # each shard scatters every register and keeps its own slices
    torch = pytest.importorskip("torch")
    from paper_2604_08374_gb300.sharded import hyperball_run_sharded_local
    off, b, _ = tiny_graph(4)
    ref = oracle.hyperball(off, b, 8, 0, seed=6, reg_bits=bits)
    with vga.vga_graph_load(off, b) as g:
        md = torch.empty(g.n_nodes, dtype=torch.float64, device="cuda")
        ball = torch.empty_like(md)
        kw = dict(slice_bytes=S, union_mode=2, register_bits=0 if bits == 8 else bits)
        it = hyperball_run_sharded_local(g, 8, 0, 6, shards, md, ball, first_pass=2, **kw)
        md1 = torch.empty_like(md)
        ball1 = torch.empty_like(md)
        it1 = hyperball_run_sharded_local(g, 8, 0, 6, shards, md1, ball1, first_pass=1, **kw)
    assert it == it1 == ref["iterations"]
    assert np.array_equal(md.cpu().numpy(), ref["mean_depth"], equal_nan=True)
    assert np.array_equal(md1.cpu().numpy(), ref["mean_depth"], equal_nan=True)
    assert np.array_equal(ball.cpu().numpy(), ref["ball"])
