"""GPU test of hyperball_run_noalloc, the entry point for callers that cannot
allocate device memory (for example code running under a framework's caching
allocator, or a long-running service that must not call cudaMalloc/cudaFree
after start-up).  It runs the same analysis as hyperball_run_dev but uses the
library's fixed 64 MiB scratch array instead of any allocation.

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


@pytest.fixture(scope="module")
def vga():
    from paper_2604_08374_gb300 import build
    build.build()
    import paper_2604_08374_gb300 as v
    return v


def _existing_entry_point(vga, torch, g, p, d, seed):
    n = g.n_nodes
    md = torch.empty(n, dtype=torch.float64, device="cuda")
    ball = torch.empty(n, dtype=torch.float64, device="cuda")
    it = vga.hyperball_run_dev(g, p, d, seed, md, ball)
    torch.cuda.synchronize()
    return md.cpu().numpy(), ball.cpu().numpy(), it


def test_noalloc_matches_existing_entry_point_twice_in_a_row(vga):
    torch = pytest.importorskip("torch")
    obst = workloads.tiny(2)
    offsets, bytes_, cells = oracle.build_graph(obst)
    n = len(cells)
    with vga.vga_graph_load(offsets, bytes_) as g:
        # two calls in a row with different shapes: the second must not see the
        # first one's leftovers in the shared scratch
        for p, d, seed in ((10, 3, 0), (8, 0, 99)):
            ref_md, ref_ball, ref_it = _existing_entry_point(vga, torch, g, p, d, seed)
            md = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
            ball = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
            it = vga.hyperball_run_noalloc(g, p, d, seed, md, ball)
            torch.cuda.synchronize()
            assert it == ref_it
            np.testing.assert_allclose(md.cpu().numpy(), ref_md, rtol=MD_RTOL, atol=0)
            np.testing.assert_allclose(ball.cpu().numpy(), ref_ball, rtol=MD_RTOL, atol=0)


def test_noalloc_rejects_runs_beyond_the_fixed_scratch(vga):
    obst = workloads.tiny(1)
    offsets, bytes_, cells = oracle.build_graph(obst)
    torch = pytest.importorskip("torch")
    n = len(cells)
    with vga.vga_graph_load(offsets, bytes_) as g:
        assert vga.hyperball_workspace_bytes(g, 16) > 64 * 2**20   # 903 nodes x 2 x 65,536 registers
        md = torch.empty(n, dtype=torch.float64, device="cuda")
        with pytest.raises(vga.VgaError) as e:
            vga.hyperball_run_noalloc(g, 16, 3, 0, md, None)
        assert e.value.status == vga.VGA_EINVAL
        assert "64 MiB" in str(e.value)
