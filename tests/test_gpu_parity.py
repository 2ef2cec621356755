"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Registers are compared bit for bit after every pass, as are the HLL estimates
c_t (both sides form the harmonic sum exactly and round once), the iteration
count, and Visual Mean Depth (bit-exact here; the stated tolerance, 1e-6
relative, is asserted as well).  Sizes span several slices and CTAs with
ragged tails: the tiny 32 x 32 configuration (N ~ 900, ~4e5 edges) and small
grids, at p from 4 to 12, forced slice widths from 16 to 1024 bytes, several
CTA sizes, both convergence rules, d = 1, 3 and unlimited.
"""
import math

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
MD_RTOL = 1e-6


@pytest.fixture(scope="module")
def vga():
    from paper_2604_08374_gb300 import build
    build.build()
    import paper_2604_08374_gb300 as v
    return v


_cache = {}


def tiny_graph(seed):
    if seed not in _cache:
        obst = workloads.tiny(seed)
        off, b, cells = oracle.build_graph(obst)
        _cache[seed] = (obst, off, b, cells)
    return _cache[seed]


def assert_same_run(got, ref, check_regs=True):
    assert got["iterations"] == ref["iterations"]
    T = got["iterations"]
    for t in range(T + 1):
        if check_regs:
            assert np.array_equal(got["regs"][t], ref["regs"][t]), f"registers differ after pass {t}"
        assert np.array_equal(got["c"][t], ref["c"][t]), f"estimates differ after pass {t}"
    np.testing.assert_allclose(got["mean_depth"], ref["mean_depth"], rtol=MD_RTOL, atol=0)
    assert np.array_equal(got["mean_depth"], ref["mean_depth"], equal_nan=True)
    assert np.array_equal(got["ball"], ref["ball"])


# ----------------------------------------------------------------------------
# graph residency and the builder
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [1, 2, 3])
def test_load_round_trip(vga, seed):
    _, off, b, cells = tiny_graph(seed)
    row_ptr, _ = oracle.decode_csr(off, b)
    with vga.vga_graph_load(off, b) as g:
        assert (g.n_nodes, g.n_bytes, g.n_edges) == (len(cells), len(b), int(row_ptr[-1]))
        o2, b2, deg = g.copy_csr()
        assert np.array_equal(o2, off) and np.array_equal(b2, b)
        assert np.array_equal(deg, np.diff(row_ptr.astype(np.int64)))


@pytest.mark.parametrize("grid", ["tiny1", "tiny2", "tiny3", "tiny4", "tiny5", "rect40x23", "open9x7", "thin1x50",
                                  "wall", "maze"])
def test_builder_matches_oracle(vga, grid):
    if grid.startswith("tiny"):
        obst = workloads.tiny(int(grid[4:]))
    elif grid == "rect40x23":
        obst = workloads.random_rectangles(40, 23, 9, (1, 7), seed=11)
    elif grid == "open9x7":
        obst = workloads.open_grid(9, 7)
    elif grid == "thin1x50":
        obst = workloads.open_grid(50, 1)
    elif grid == "wall":
        obst = workloads.open_grid(20, 12)
        obst[:, 9] = 1
        obst[5, 9] = 0
    else:
        rng = np.random.default_rng(3)
        obst = (rng.random((37, 41)) < 0.3).astype(np.uint8)
    off, b, cells = oracle.build_graph(obst)
    g, gcells = vga.vga_visibility_build(obst, return_cells=True)
    with g:
        o2, b2, _ = g.copy_csr()
        assert np.array_equal(gcells.astype(np.int64), cells)
        assert np.array_equal(o2, off)
        assert np.array_equal(b2, b)
        assert g.n_nodes == vga.vga_visibility_count(obst)


def _builder_grid(name):
    if name == "wall":
        obst = workloads.open_grid(20, 12)
        obst[:, 9] = 1
        obst[5, 9] = 0
        return obst
    if name == "maze":
        return (np.random.default_rng(3).random((37, 41)) < 0.3).astype(np.uint8)
    if name == "dense":
        return (np.random.default_rng(8).random((29, 33)) < 0.45).astype(np.uint8)
    return workloads.random_rectangles(40, 23, 9, (1, 7), seed=11)


@pytest.mark.parametrize("limits", [(1, 0), (2, 1), (0, 1)], ids=["global-lists", "both", "global-bitmap"])
@pytest.mark.parametrize("grid", ["wall", "maze", "dense", "rect40x23"])
def test_builder_fallbacks_match_oracle(vga, grid, limits):
    # The sweep's two fallbacks, forced on small grids: interval lists that
    # outgrow shared memory are redone with global lists (capacity 1 or 2
    # sends nearly every source there), and the node bitmap in global memory.
    obst = _builder_grid(grid)
    off, b, cells = oracle.build_graph(obst)
    vga.vga_set_visibility_sweep_limits(*limits)
    try:
        g = vga.vga_visibility_build(obst)
    finally:
        vga.vga_set_visibility_sweep_limits(0, 0)
    with g:
        o2, b2, _ = g.copy_csr()
        assert np.array_equal(o2, off) and np.array_equal(b2, b)


def test_builder_comb_overflows_shared_lists(vga):
    # A column of single-cell pillars two rows apart leaves ~135 open slope
    # intervals behind it for sources near the corner, more than the 48 the
    # shared-memory lists hold: those sources take the global-list retry.
    W = H = 280
    obst = np.zeros((H, W), np.uint8)
    obst[0:H:2, 270] = 1
    g, gcells = vga.vga_visibility_build(obst, return_cells=True)
    with g:
        noc, cells = oracle.main_component(obst)
        assert np.array_equal(gcells.astype(np.int64), cells)
        n = g.n_nodes
        corner = [int(noc[y * W + x]) for y in range(4) for x in range(4)]
        rng = np.random.default_rng(0)
        sample = np.unique(np.concatenate([corner, rng.choice(n, 12, replace=False), [n - 1]])).astype(np.int64)
        row_ptr, col = oracle.visibility_csr(obst, cells, nodes=sample)
        g_off, g_bytes, _ = g.copy_csr()
        for k, v in enumerate(sample):
            got = oracle.decode_list(g_bytes, int(g_off[v]), int(g_off[v + 1]), n)
            assert np.array_equal(got, col[row_ptr[k]:row_ptr[k + 1]]), f"neighbour list of node {v}"


# ----------------------------------------------------------------------------
# HyperBall, bit-exact at every pass
# ----------------------------------------------------------------------------

CASES = [
    # seed, p, d, slice_bytes, warps_per_cta, conv_mode
    (1, 10, 3, 0, 0, 0),
    (1, 10, 0, 0, 0, 0),
    (2, 10, 0, 256, 8, 0),
    (3, 10, 0, 64, 4, 0),
    (4, 8, 3, 16, 16, 0),
    (5, 12, 3, 1024, 8, 0),
    (1, 4, 0, 16, 3, 0),
    (2, 6, 0, 32, 5, 0),
    (3, 12, 2, 512, 1, 0),
    (1, 10, 0, 128, 8, 1),
    (2, 9, 1, 0, 7, 0),
]


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("seed,p,d,S,warps,conv", CASES)
def test_hyperball_bit_exact(vga, seed, p, d, S, warps, conv, mode):
    # mode 1: one gather per neighbour; mode 2: per run of consecutive ids via range maxima
    _, off, b, cells = tiny_graph(seed)
    T = 12
    ref = oracle.hyperball(off, b, p, d, seed=seed * 7, conv_mode=conv, trace=T)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, p, d, seed=seed * 7, conv_mode=conv, max_trace=T, slice_bytes=S,
                                      warps_per_cta=warps, union_mode=mode)
    assert got["iterations"] <= T
    assert_same_run(got, ref)


_regime_graph = {}


def regime_graph():
    # 60 x 60, 40 rectangles with sides 2..8: N = 2655 > 2.5 x 1024, and the
    # balls grow past 2.5 m over passes 2 and 3 (every node crosses at p = 10)
    if not _regime_graph:
        obst = workloads.random_rectangles(60, 60, 40, (2, 8), seed=1)
        _regime_graph["g"] = oracle.build_graph(obst)
    return _regime_graph["g"]


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("p", [9, 10])
def test_estimator_regime_switch_every_node(vga, p, mode):
    # The estimator takes linear counting while E <= 2.5 m and the raw estimate
    # above it (Sec. 2.3, Sec. 3.3).  On this graph every node's counter passes
    # from one regime to the other inside the traced passes, and many sit
    # within 2 % of the threshold; every node and pass is compared.
    off, b, cells = regime_graph()
    m = 1 << p
    ref = oracle.hyperball(off, b, p, 0, seed=5, trace=12)
    alpha_mm = oracle.hll_alpha(p) * m * m
    lc_side = [alpha_mm / np.sum(np.ldexp(1.0, -r.astype(np.int64)), axis=1) <= 2.5 * m
               for r in ref["regs"][: ref["iterations"] + 1]]
    crossed = np.zeros(len(cells), bool)
    for a, b_ in zip(lc_side, lc_side[1:]):
        crossed |= a & ~b_
    assert crossed.all(), "every node should cross from linear counting to the raw estimate"
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, p, 0, seed=5, max_trace=12, union_mode=mode)
    assert_same_run(got, ref)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("grid", ["open40x30", "open1x300", "comb"])
def test_long_runs(vga, grid, mode):
    # complete graphs (every list is one or two runs of up to N-1 ids) and a comb
    # of walls (many short runs): range lookups of every level, windows split
    # into 16-row pieces, runs ending at the last node id
    if grid == "open40x30":
        obst = workloads.open_grid(40, 30)
    elif grid == "open1x300":
        obst = workloads.open_grid(300, 1)
    else:
        obst = workloads.open_grid(33, 21)
        obst[2:19:2, 3:30] = 1
    off, b, cells = oracle.build_graph(obst)
    ref = oracle.hyperball(off, b, 8, 0, seed=3, trace=10)
    with vga.vga_graph_load(off, b) as g:
        for S in (0, 16, 256):
            got = vga.hyperball_run_trace(g, 8, 0, seed=3, max_trace=10, slice_bytes=S, union_mode=mode)
            assert_same_run(got, ref)


def test_hyperball_run_plain(vga):
    _, off, b, cells = tiny_graph(1)
    ref = oracle.hyperball(off, b, 10, 3, seed=0)
    with vga.vga_graph_load(off, b) as g:
        md, ball, it = vga.hyperball_run(g, 10, 3, 0)
    assert it == ref["iterations"] == 3
    assert np.array_equal(md, ref["mean_depth"]) and np.array_equal(ball, ref["ball"])


def test_hyperball_hash_seed_large(vga):
    _, off, b, _ = tiny_graph(2)
    seed = 0xDEADBEEFCAFEF00D
    ref = oracle.hyperball(off, b, 10, 0, seed=seed, trace=10)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, 10, 0, seed=seed, max_trace=10)
    assert_same_run(got, ref)


def test_component_sizes_and_isolated_nodes(vga):
    # two components of the visibility graph kept together, with their exact sizes
    obst = workloads.open_grid(12, 7)
    obst[:, 5] = 1
    _, cells = oracle.main_component(workloads.open_grid(5, 7))
    rp1, col1 = oracle.visibility_csr(workloads.open_grid(5, 7), cells)
    n1 = len(cells)
    rp2, col2 = oracle.visibility_csr(workloads.open_grid(6, 7), oracle.main_component(workloads.open_grid(6, 7))[1])
    n2 = len(rp2) - 1
    row_ptr = np.concatenate([rp1, rp2[1:] + rp1[-1], [rp1[-1] + rp2[-1]]]).astype(np.uint64)
    col = np.concatenate([col1, col2 + n1]).astype(np.uint32)
    n = n1 + n2 + 1  # plus one isolated node
    off, b = oracle.csr_encode(row_ptr, col)
    comp = np.array([n1] * n1 + [n2] * n2 + [1], np.uint32)
    ref = oracle.hyperball(off, b, 8, 0, comp_size=comp, trace=8)
    with vga.vga_graph_load(off, b, comp_size=comp) as g:
        got = vga.hyperball_run_trace(g, 8, 0, max_trace=8)
    assert_same_run(got, ref)
    assert math.isnan(got["mean_depth"][-1])


def test_degenerate_graphs(vga):
    for n in (0, 1):
        off = np.zeros(n + 1, np.uint64)
        ref = oracle.hyperball(off, np.zeros(0, np.uint8), 10, 0, trace=2)
        with vga.vga_graph_load(off, np.zeros(0, np.uint8)) as g:
            got = vga.hyperball_run_trace(g, 10, 0, max_trace=2)
        assert got["iterations"] == ref["iterations"]
        assert np.array_equal(np.isnan(got["mean_depth"]), np.isnan(ref["mean_depth"]))
    off, b, _ = oracle.build_graph(workloads.open_grid(2, 1))
    ref = oracle.hyperball(off, b, 10, 0, trace=3)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, 10, 0, max_trace=3)
    assert_same_run(got, ref)


# ----------------------------------------------------------------------------
# errors
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("stream,n", [
    (bytes([0x80]), 2),                          # unterminated varint
    (bytes([0x81, 0x81, 0x81, 0x81, 0x81, 0x01]), 2),  # six-byte varint
    (bytes([0x01, 0x00]), 3),                    # duplicate neighbour (zero delta)
    (bytes([0x05]), 3),                          # id >= n
    (bytes([0x00]), 2),                          # self loop on node 0
    (bytes([0xFF, 0xFF, 0xFF, 0xFF, 0x7F]), 2),  # value above 32 bits
])
def test_corrupt_streams_rejected(vga, stream, n):
    off = np.zeros(n + 1, np.uint64)
    off[1:] = len(stream)
    with pytest.raises(vga.VgaError) as e:
        vga.vga_graph_load(off, np.frombuffer(stream, np.uint8).copy())
    assert e.value.status == vga.VGA_ECORRUPT


def test_bad_offsets_rejected(vga):
    with pytest.raises(vga.VgaError) as e:
        vga.vga_graph_load(np.array([0, 2, 1], np.uint64), np.array([1, 0], np.uint8))
    assert e.value.status == vga.VGA_ECORRUPT


def test_bad_arguments(vga):
    _, off, b, _ = tiny_graph(1)
    with vga.vga_graph_load(off, b) as g:
        for p in (3, 17):
            with pytest.raises(vga.VgaError) as e:
                vga.hyperball_run(g, p, 3, 0)
            assert e.value.status == vga.VGA_EINVAL
        for S in (8, 48, 2048):
            with pytest.raises(vga.VgaError):
                vga.hyperball_run_trace(g, 10, 1, slice_bytes=S, max_trace=1)
        with pytest.raises(vga.VgaError):
            vga.hyperball_run_trace(g, 6, 1, slice_bytes=128, max_trace=1)  # slice wider than m = 64
        with pytest.raises(vga.VgaError):
            vga.hyperball_run_trace(g, 10, 1, max_trace=1, union_mode=3)


# ----------------------------------------------------------------------------
# device outputs, user workspace, streams, files
# ----------------------------------------------------------------------------

def test_run_dev_with_torch_buffers(vga):
    torch = pytest.importorskip("torch")
    _, off, b, cells = tiny_graph(3)
    n = len(cells)
    ref = oracle.hyperball(off, b, 10, 0, seed=5)
    with vga.vga_graph_load(off, b) as g:
        ws = torch.empty(vga.hyperball_workspace_bytes(g, 10), dtype=torch.uint8, device="cuda")
        md = torch.empty(n, dtype=torch.float64, device="cuda")
        ball = torch.empty(n, dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        it = vga.hyperball_run_dev(g, 10, 0, 5, md, ball, workspace=ws, stream=s)
        s.synchronize()
    assert it == ref["iterations"]
    assert np.array_equal(md.cpu().numpy(), ref["mean_depth"])
    assert np.array_equal(ball.cpu().numpy(), ref["ball"])


def test_file_round_trip(vga, tmp_path):
    _, off, b, _ = tiny_graph(2)
    path = str(tmp_path / "g.vgacsr")
    with vga.vga_graph_load(off, b) as g:
        g.save(path)
    with vga.vga_graph_load_file(path) as g2:
        o2, b2, _ = g2.copy_csr()
    assert np.array_equal(o2, off) and np.array_equal(b2, b)
    with open(path, "r+b") as f:
        f.write(b"XXXX")
    with pytest.raises(vga.VgaError) as e:
        vga.vga_graph_load_file(path)
    assert e.value.status == vga.VGA_ECORRUPT


# ----------------------------------------------------------------------------
# closed-form metrics (Sec. 3.3 "Metric derivation")
# ----------------------------------------------------------------------------

def test_metrics_match_oracle(vga):
    torch = pytest.importorskip("torch")
    _, off, b, cells = tiny_graph(4)
    n = len(cells)
    row_ptr, _ = oracle.decode_csr(off, b)
    deg = np.diff(row_ptr.astype(np.int64)).astype(np.uint32)
    comp = np.full(n, n, np.uint32)
    comp[:3] = [2, 1, 40]  # degenerate and small components too
    ref_md = oracle.hyperball(off, b, 10, 3, comp_size=comp)["mean_depth"]
    md_in = ref_md.copy()
    md_in[5] = 1.0          # exact MD = 1 gives HH = +inf
    ref = oracle.metrics(md_in, deg, comp_size=comp)
    with vga.vga_graph_load(off, b, comp_size=comp) as g:
        md_dev = torch.from_numpy(md_in).cuda()
        got = vga.vga_metrics(g, md_dev).cpu().numpy()
        torch.cuda.synchronize()
        # the same MD straight from the GPU run feeds the same metrics
        md_gpu = torch.empty(n, dtype=torch.float64, device="cuda")
        vga.hyperball_run_dev(g, 10, 3, 0, md_gpu, None)
        got_run = vga.vga_metrics(g, md_gpu).cpu().numpy()
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.array_equal(np.isinf(got), np.isinf(ref))
    fin = np.isfinite(ref)
    np.testing.assert_allclose(got[fin], ref[fin], rtol=1e-12, atol=0)
    ref_run = oracle.metrics(ref_md, deg, comp_size=comp)
    fin = np.isfinite(ref_run)
    np.testing.assert_allclose(got_run[fin], ref_run[fin], rtol=MD_RTOL, atol=0)


# ----------------------------------------------------------------------------
# Hilbert node order (Sec. 3.2, optional Hilbert reordering)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("grid", ["tiny2", "rect40x23", "open9x7"])
def test_hilbert_builder_and_hyperball(vga, grid):
    if grid == "tiny2":
        obst = workloads.tiny(2)
    elif grid == "rect40x23":
        obst = workloads.random_rectangles(40, 23, 9, (1, 7), seed=11)
    else:
        obst = workloads.open_grid(9, 7)
    off, b, cells = oracle.build_graph(obst, order="hilbert")
    g, gcells = vga.vga_visibility_build(obst, return_cells=True, order="hilbert")
    with g:
        o2, b2, _ = g.copy_csr()
        assert np.array_equal(gcells.astype(np.int64), cells)
        assert np.array_equal(o2, off) and np.array_equal(b2, b)
        ref = oracle.hyperball(off, b, 10, 0, seed=2, trace=10)
        for mode in (1, 2):
            got = vga.hyperball_run_trace(g, 10, 0, seed=2, max_trace=10, union_mode=mode)
            assert_same_run(got, ref)


# ----------------------------------------------------------------------------
# 4-bit registers (the paper's packed format, Sec. 3.3)
# ----------------------------------------------------------------------------

def _seed_with_clamp(n, p):
    """A hash seed for which some node's rho exceeds 15 (the 4-bit clamp bites)."""
    # the hash input is v ^ seed: seeds must reach above the node ids, or every
    # seed only permutes the same few inputs
    for k in range(1, 5000):
        seed = k * 0x9E3779B97F4A7C15 % (1 << 63)
        if any(oracle.hll_hash(v, seed, p)[1] > 15 for v in range(n)):
            return seed
    raise AssertionError("no seed found")


@pytest.mark.parametrize("p,S,mode", [(10, 0, 1), (10, 0, 2), (8, 16, 2), (12, 256, 1), (5, 16, 1), (10, 64, 2)])
def test_four_bit_registers_bit_exact(vga, p, S, mode):
    _, off, b, cells = tiny_graph(3)
    seed = _seed_with_clamp(len(cells), p)
    ref = oracle.hyperball(off, b, p, 0, seed=seed, trace=12, reg_bits=4)
    assert ref["regs"][0].max() == 15
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, p, 0, seed=seed, max_trace=12, slice_bytes=S, union_mode=mode,
                                      register_bits=4)
    assert_same_run(got, ref)


def test_four_bit_rejects_small_p(vga):
    _, off, b, _ = tiny_graph(1)
    with vga.vga_graph_load(off, b) as g:
        with pytest.raises(vga.VgaError):
            vga.hyperball_run_trace(g, 4, 1, max_trace=1, register_bits=4)
        with pytest.raises(vga.VgaError):
            vga.hyperball_run_trace(g, 10, 1, max_trace=1, register_bits=6)


# ----------------------------------------------------------------------------
# split hubs in the run-aware union
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("hub,S,bits", [(1, 0, 8), (3, 64, 8), (17, 16, 8), (64, 0, 8), (2, 32, 4), (9, 0, 4)])
def test_hub_split_bit_exact(vga, hub, S, bits):
    # a small threshold splits most nodes into chunks that merge by atomic max
    _, off, b, _ = tiny_graph(2)
    p = 8
    ref = oracle.hyperball(off, b, p, 0, seed=5, trace=12, reg_bits=bits)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, p, 0, seed=5, max_trace=12, slice_bytes=S, union_mode=2,
                                      register_bits=0 if bits == 8 else bits, hub_lookups=hub)
    assert_same_run(got, ref)


def _skewed_csr(n=12000, seed=0):
    """Directed CSR with a few hubs far above the rest: hub h sees every other
    node of a long range (single-id runs, so one lookup per neighbour); the
    other nodes see a few short runs."""
    rng = np.random.default_rng(seed)
    lists = []
    hubs = {0: 2, 5000: 3, 11999: 2}
    for v in range(n):
        if v in hubs:
            ids = np.arange(1 if v == 0 else 0, n, hubs[v])
        else:
            starts = rng.integers(0, n - 8, size=4)
            ids = np.unique(np.concatenate([np.arange(s, s + rng.integers(1, 8)) for s in starts]))
        ids = ids[ids != v]
        lists.append(ids.astype(np.uint32))
    row_ptr = np.zeros(n + 1, np.uint64)
    row_ptr[1:] = np.cumsum([len(x) for x in lists])
    return oracle.csr_encode(row_ptr, np.concatenate(lists))


@pytest.mark.parametrize("hub", [0, 1000, 2500])
def test_hub_split_skewed_graph(vga, hub):
    # hub = 0: the automatic threshold (>= 2048 lookups) splits the 4000- and
    # 6000-lookup hubs; explicit thresholds split them into more chunks
    off, b = _skewed_csr()
    ref = oracle.hyperball(off, b, 8, 3, seed=9, trace=3)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, 8, 3, seed=9, max_trace=3, union_mode=2, hub_lookups=hub)
        got1 = vga.hyperball_run_trace(g, 8, 3, seed=9, max_trace=3, union_mode=1)
    assert_same_run(got, ref)
    assert_same_run(got1, ref)


def test_hub_lookups_rejects_negative(vga):
    _, off, b, _ = tiny_graph(1)
    with vga.vga_graph_load(off, b) as g:
        with pytest.raises(vga.VgaError):
            vga.hyperball_run_trace(g, 8, 1, max_trace=1, union_mode=2, hub_lookups=-3)


# ----------------------------------------------------------------------------
# table schemes of the run-aware union (5 rows: windows 1..16; 3 rows: 1, 4, 16)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("levels,p,S,bits,hub", [(3, 10, 0, 8, 0), (3, 8, 16, 8, 0), (3, 12, 128, 8, 0), (5, 10, 64, 8, 0),
                                                 (3, 10, 64, 4, 0), (3, 8, 32, 8, 5)])
def test_table_levels_bit_exact(vga, levels, p, S, bits, hub):
    _, off, b, _ = tiny_graph(1)
    ref = oracle.hyperball(off, b, p, 0, seed=77, trace=12, reg_bits=bits)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, p, 0, seed=77, max_trace=12, slice_bytes=S, union_mode=2,
                                      register_bits=0 if bits == 8 else bits, hub_lookups=hub, table_levels=levels)
        # the other scheme on the same graph object: its own lookup list
        other = vga.hyperball_run_trace(g, p, 0, seed=77, max_trace=12, slice_bytes=S, union_mode=2,
                                        register_bits=0 if bits == 8 else bits, table_levels=8 - levels)
    assert_same_run(got, ref)
    assert_same_run(other, ref)


@pytest.mark.parametrize("grid", ["open40x30", "open1x300", "comb"])
def test_table_levels_long_runs(vga, grid):
    # runs of every length up to N-1: windows of 1, 4 and 16 rows, 16-row pieces
    if grid == "open40x30":
        obst = workloads.open_grid(40, 30)
    elif grid == "open1x300":
        obst = workloads.open_grid(300, 1)
    else:
        obst = workloads.open_grid(33, 21)
        obst[2:19:2, 3:30] = 1
    off, b, cells = oracle.build_graph(obst)
    ref = oracle.hyperball(off, b, 8, 0, seed=2, trace=6)
    with vga.vga_graph_load(off, b) as g:
        got = vga.hyperball_run_trace(g, 8, 0, seed=2, max_trace=6, union_mode=2, table_levels=3)
    assert_same_run(got, ref)


def test_table_levels_rejects_bad_value(vga):
    _, off, b, _ = tiny_graph(1)
    with vga.vga_graph_load(off, b) as g:
        with pytest.raises(vga.VgaError):
            vga.hyperball_run_trace(g, 8, 1, max_trace=1, union_mode=2, table_levels=4)


@pytest.mark.parametrize("mode", [1, 2])
def test_l2_window_same_result(vga, mode):
    torch = pytest.importorskip("torch")
    _, off, b, _ = tiny_graph(2)
    ref = oracle.hyperball(off, b, 10, 3, seed=4)
    with vga.vga_graph_load(off, b) as g:
        md = torch.empty(g.n_nodes, dtype=torch.float64, device="cuda")
        ball = torch.empty_like(md)
        s = torch.cuda.Stream()
        it = vga.hyperball_run_dev(g, 10, 3, 4, md, ball, stream=s, union_mode=mode, l2_window=1)
        torch.cuda.synchronize()
    assert it == ref["iterations"]
    assert np.array_equal(md.cpu().numpy(), ref["mean_depth"], equal_nan=True)
    assert np.array_equal(ball.cpu().numpy(), ref["ball"])


def test_load_from_device_buffers(vga):
    torch = pytest.importorskip("torch")
    _, off, b, cells = tiny_graph(3)
    off_d = torch.from_numpy(off.view(np.int64).copy()).cuda()
    b_d = torch.from_numpy(b.copy()).cuda()
    with vga.vga_graph_load_device(off_d, b_d, len(b)) as g:
        o2, b2, _ = g.copy_csr()
        assert np.array_equal(o2, off) and np.array_equal(b2, b)
        got = vga.hyperball_run_trace(g, 8, 3, seed=6, max_trace=3)
    ref = oracle.hyperball(off, b, 8, 3, seed=6, trace=3)
    assert_same_run(got, ref)


@pytest.mark.parametrize("S", [16, 64, 128, 1024])
def test_gather_microbenchmark(vga, S):
    for consumer in (0, 1, 2):
        gbs = vga.vga_bench_gather(64 << 20, S, 1 << 22, consumer=consumer)
        assert 100.0 < gbs < 1e6
    with pytest.raises(vga.VgaError):
        vga.vga_bench_gather(64 << 20, 48, 1 << 20)
    with pytest.raises(vga.VgaError):
        vga.vga_bench_gather(64 << 20, S, 1 << 20, consumer=3)
