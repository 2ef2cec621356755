"""GPU test of hyperball_run_noalloc, the entry point for callers that cannot
allocate device memory: code running under a framework's caching allocator
that already holds the GPU's memory, long-running services that must not stall
or fail in cudaMalloc/cudaFree after start-up, and hosts that budget every
device byte up front.  It runs the same analysis as hyperball_run_dev (the
per-neighbour union) but takes its scratch from the library's fixed 64 MiB
array instead of any allocation.

Its results must be those of hyperball_run_dev bit for bit (both build the
same integer registers and round the same estimator once), and those of the
oracle (Alg. 1): iterations, ball sizes and mean depth equal, NaN included.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.  It builds what it needs itself, so
it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
MD_RTOL = 1e-6  # the tolerance the parity tests state for mean depth
LIMIT = 64 * 2**20


@pytest.fixture(scope="module")
def vga():
    from paper_2604_08374_gb300 import build
    build.build()
    import paper_2604_08374_gb300 as v
    return v


def _a(x):
    return (x + 255) // 256 * 256


def documented_scratch_bytes(n, p):
    """The size limit as the header states it for hyperball_run_noalloc."""
    m = 1 << p
    s = max(1, m // 1024)
    b = 2 * _a(n * m) + 3 * _a(8 * n) + _a(8 * (m + 1)) + 256
    if p <= 13:
        b += _a(4 * n)
    if p <= 15:
        b += _a(s * n) + 2 * _a(4 * n)
    return b


def _existing_entry_point(vga, torch, g, p, d, seed):
    n = g.n_nodes
    md = torch.empty(n, dtype=torch.float64, device="cuda")
    ball = torch.empty(n, dtype=torch.float64, device="cuda")
    it = vga.hyperball_run_dev(g, p, d, seed, md, ball)
    torch.cuda.synchronize()
    return md.cpu().numpy(), ball.cpu().numpy(), it


def _noalloc(vga, torch, g, p, d, seed):
    n = g.n_nodes
    md = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    ball = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    it = vga.hyperball_run_noalloc(g, p, d, seed, md, ball)
    torch.cuda.synchronize()
    return md.cpu().numpy(), ball.cpu().numpy(), it


def test_noalloc_matches_existing_entry_point_and_oracle_twice_in_a_row(vga):
    torch = pytest.importorskip("torch")
    obst = workloads.tiny(2)
    offsets, bytes_, cells = oracle.build_graph(obst)
    with vga.vga_graph_load(offsets, bytes_) as g:
        # two calls in a row with different shapes: the second must not see the
        # first one's leftovers in the shared scratch
        for p, d, seed in ((10, 3, 0), (8, 0, 99)):
            assert documented_scratch_bytes(len(cells), p) <= LIMIT
            ref_md, ref_ball, ref_it = _existing_entry_point(vga, torch, g, p, d, seed)
            md, ball, it = _noalloc(vga, torch, g, p, d, seed)
            assert it == ref_it
            np.testing.assert_allclose(md, ref_md, rtol=MD_RTOL, atol=0)
            assert np.array_equal(md, ref_md, equal_nan=True)
            assert np.array_equal(ball, ref_ball)
            orc = oracle.hyperball(offsets, bytes_, p, d, seed=seed)
            assert it == orc["iterations"]
            assert np.array_equal(md, orc["mean_depth"], equal_nan=True)
            assert np.array_equal(ball, orc["ball"])


def test_noalloc_rejects_runs_beyond_the_fixed_scratch(vga):
    obst = workloads.tiny(1)
    offsets, bytes_, cells = oracle.build_graph(obst)
    torch = pytest.importorskip("torch")
    n = len(cells)
    with vga.vga_graph_load(offsets, bytes_) as g:
        assert documented_scratch_bytes(n, 16) > LIMIT   # 903 nodes x 2 x 65,536 registers
        md = torch.empty(n, dtype=torch.float64, device="cuda")
        with pytest.raises(vga.VgaError) as e:
            vga.hyperball_run_noalloc(g, 16, 3, 0, md, None)
        assert e.value.status == vga.VGA_EINVAL
        assert "64 MiB" in str(e.value)


def test_noalloc_limit_is_the_documented_one(vga):
    # A graph of ~20k nodes: at p = 10 the documented (per-neighbour) size fits
    # in 64 MiB while hyperball_workspace_bytes (the automatic run-aware plan)
    # does not, so the run must succeed; at p = 11 the documented size exceeds
    # the limit and the run must be refused.
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    obst = (rng.random((170, 170)) < 0.3).astype(np.uint8)
    with vga.vga_visibility_build(obst) as g:
        n = g.n_nodes
        assert documented_scratch_bytes(n, 10) <= LIMIT < vga.hyperball_workspace_bytes(g, 10)
        ref_md, ref_ball, ref_it = _existing_entry_point(vga, torch, g, 10, 3, 1)
        md, ball, it = _noalloc(vga, torch, g, 10, 3, 1)
        assert it == ref_it
        assert np.array_equal(md, ref_md, equal_nan=True)
        assert np.array_equal(ball, ref_ball)
        for p in (11, 12):
            assert documented_scratch_bytes(n, p) > LIMIT
            with pytest.raises(vga.VgaError) as e:
                _noalloc(vga, torch, g, p, 3, 1)
            assert e.value.status == vga.VGA_EINVAL
            assert str(documented_scratch_bytes(n, p)) in str(e.value)
