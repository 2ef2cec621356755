"""GPU tests of the batched engine (hyperball_run_batch).

Each job of a mixed batch (graphs of different sizes, p from 4 to 12, depth
limits 0/1/3, both convergence rules, both union variants, empty and one-node
graphs) must give
exactly what a single-graph run of the same job gives (bit for bit), in both
host-driven and CUDA-graph (conditional WHILE node) modes; a few jobs are also
checked against the CPU oracle directly.
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
    grids = [workloads.tiny(s) for s in (1, 2, 3)]
    grids += [workloads.rectangles_until(96, 96, (2, 12), int(96 * 96 * 0.88), seed=4),
              workloads.open_grid(20, 11), workloads.open_grid(2, 1), workloads.open_grid(1, 1),
              workloads.rectangles_until(60, 45, (2, 9), int(60 * 45 * 0.85), seed=9)]
    out = []
    for obst in grids:
        off, b, cells = oracle.build_graph(obst)
        out.append((vga.vga_graph_load(off, b), off, b))
    empty = vga.vga_graph_load(np.zeros(1, np.uint64), np.zeros(0, np.uint8))
    out.append((empty, np.zeros(1, np.uint64), np.zeros(0, np.uint8)))
    yield out
    for g, _, _ in out:
        g.free()


def _jobs(torch, graphs):
    rng = np.random.default_rng(7)
    jobs = []
    for k in range(26):
        g, off, b = graphs[k % len(graphs)]
        p = [4, 8, 10, 12, 10, 6][k % 6]
        d = [0, 3, 1, 3, 0][k % 5]
        conv = 1 if k % 7 == 3 else 0
        n = g.n_nodes
        jobs.append(dict(graph=g, off=off, b=b, p=p, d=d, seed=int(rng.integers(0, 2**62)), conv_mode=conv,
                         union_mode=[0, 1, 2][k % 3],
                         mean_depth=torch.full((max(n, 1),), -7.0, dtype=torch.float64, device="cuda"),
                         ball=torch.full((max(n, 1),), -7.0, dtype=torch.float64, device="cuda")))
    return jobs


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_matches_single_runs(vga, graphs, use_graph):
    torch = pytest.importorskip("torch")
    jobs = _jobs(torch, graphs)
    its = vga.hyperball_run_batch(jobs, use_graph=use_graph)
    torch.cuda.synchronize()
    for k, j in enumerate(jobs):
        g, n = j["graph"], j["graph"].n_nodes
        if n == 0:
            assert its[k] == 0
            continue
        md = torch.empty(n, dtype=torch.float64, device="cuda")
        ball = torch.empty(n, dtype=torch.float64, device="cuda")
        it = vga.hyperball_run_dev(g, j["p"], j["d"], j["seed"], md, ball, conv_mode=j["conv_mode"])
        torch.cuda.synchronize()
        assert its[k] == it, k
        assert np.array_equal(j["mean_depth"][:n].cpu().numpy(), md.cpu().numpy(), equal_nan=True), k
        assert np.array_equal(j["ball"][:n].cpu().numpy(), ball.cpu().numpy()), k


def test_batch_against_oracle(vga, graphs):
    torch = pytest.importorskip("torch")
    jobs = _jobs(torch, graphs)[:6]
    its = vga.hyperball_run_batch(jobs, use_graph=True)
    for k, j in enumerate(jobs):
        n = j["graph"].n_nodes
        if n == 0:
            continue
        ref = oracle.hyperball(j["off"], j["b"], j["p"], j["d"], seed=j["seed"], conv_mode=j["conv_mode"])
        assert its[k] == ref["iterations"]
        np.testing.assert_allclose(j["mean_depth"][:n].cpu().numpy(), ref["mean_depth"], rtol=1e-6)
        assert np.array_equal(j["mean_depth"][:n].cpu().numpy(), ref["mean_depth"], equal_nan=True)


def test_batch_user_workspace_and_repeat(vga, graphs):
    torch = pytest.importorskip("torch")
    jobs = _jobs(torch, graphs)[:9]
    ws = torch.empty(vga.hyperball_batch_workspace_bytes(jobs), dtype=torch.uint8, device="cuda")
    a = vga.hyperball_run_batch(jobs, workspace=ws)
    first = [j["mean_depth"].clone() for j in jobs]
    b = vga.hyperball_run_batch(jobs, workspace=ws)
    assert a == b
    for j, f in zip(jobs, first):
        assert torch.equal(torch.nan_to_num(j["mean_depth"], nan=-1.0), torch.nan_to_num(f, nan=-1.0))


def test_batch_rejects_bad_jobs(vga, graphs):
    torch = pytest.importorskip("torch")
    jobs = _jobs(torch, graphs)[:2]
    jobs[1]["p"] = 17
    with pytest.raises(vga.VgaError) as e:
        vga.hyperball_run_batch(jobs)
    assert e.value.status == vga.VGA_EINVAL


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_scattered_first_pass(vga, graphs, use_graph):
    # run-aware jobs with p <= 13 take pass 1 as the scatter of their keys in
    # engine_start and skip the union launch of pass 1; p = 14 and
    # per-neighbour jobs gather it.  Every job must equal a single run whose
    # pass 1 is the gather, including jobs that stop right after pass 1.
    torch = pytest.importorskip("torch")
    jobs = []
    for k, (p, d, mode, conv) in enumerate([(13, 2, 2, 0), (14, 2, 2, 0), (9, 1, 2, 0), (9, 1, 1, 0), (4, 0, 2, 1),
                                            (12, 0, 0, 0), (13, 1, 2, 1), (10, 3, 2, 0)]):
        g = graphs[k % 4][0]
        n = g.n_nodes
        jobs.append(dict(graph=g, p=p, d=d, seed=1000 + k, conv_mode=conv, union_mode=mode,
                         mean_depth=torch.full((n,), -7.0, dtype=torch.float64, device="cuda"),
                         ball=torch.full((n,), -7.0, dtype=torch.float64, device="cuda")))
    its = vga.hyperball_run_batch(jobs, use_graph=use_graph)
    torch.cuda.synchronize()
    for k, j in enumerate(jobs):
        g, n = j["graph"], j["graph"].n_nodes
        md = torch.empty(n, dtype=torch.float64, device="cuda")
        ball = torch.empty_like(md)
        it = vga.hyperball_run_dev(g, j["p"], j["d"], j["seed"], md, ball, conv_mode=j["conv_mode"],
                                   union_mode=j["union_mode"], first_pass=1)
        torch.cuda.synchronize()
        assert its[k] == it, k
        assert np.array_equal(j["mean_depth"].cpu().numpy(), md.cpu().numpy(), equal_nan=True), k
        assert np.array_equal(j["ball"].cpu().numpy(), ball.cpu().numpy()), k
