"""GPU tests of the 3-row table of range maxima (windows of 1, 4 and 16 rows)
in every path that uses the run-aware union: graphs loaded after
vga_set_table_scheme_nodes(1) get that table, so the single-graph runs, the
batched engine, register shards and the server all run it on small graphs,
and must give the oracle's (and the unsharded, unbatched) results exactly.
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
    v.vga_set_table_scheme_nodes(1)
    yield v
    v.vga_set_table_scheme_nodes(0)


@pytest.fixture(scope="module")
def graphs(vga):
    out = []
    for obst in (workloads.tiny(1), workloads.tiny(4), workloads.open_grid(30, 20),
                 workloads.rectangles_until(60, 45, (2, 9), int(60 * 45 * 0.85), seed=9)):
        off, b, _ = oracle.build_graph(obst)
        out.append((vga.vga_graph_load(off, b), off, b))
    yield out
    for g, _, _ in out:
        g.free()


def test_single_runs(vga, graphs):
    for g, off, b in graphs:
        ref = oracle.hyperball(off, b, 8, 0, seed=21, trace=10)
        got = vga.hyperball_run_trace(g, 8, 0, seed=21, max_trace=10, union_mode=2)
        assert got["iterations"] == ref["iterations"]
        for t in range(ref["iterations"] + 1):
            assert np.array_equal(got["regs"][t], ref["regs"][t])
        assert np.array_equal(got["mean_depth"], ref["mean_depth"], equal_nan=True)


def test_batch(vga, graphs):
    torch = pytest.importorskip("torch")
    jobs = []
    for k, (g, off, b) in enumerate(graphs):
        n = g.n_nodes
        jobs.append(dict(graph=g, p=[8, 10, 12, 10][k], d=[0, 3, 0, 2][k], seed=5 + k, union_mode=2,
                         mean_depth=torch.empty(n, dtype=torch.float64, device="cuda"),
                         ball=torch.empty(n, dtype=torch.float64, device="cuda")))
    its = vga.hyperball_run_batch(jobs, use_graph=True)
    for j, (g, off, b), it in zip(jobs, graphs, its):
        ref = oracle.hyperball(off, b, j["p"], j["d"], seed=j["seed"])
        assert it == ref["iterations"]
        assert np.array_equal(j["mean_depth"].cpu().numpy(), ref["mean_depth"], equal_nan=True)
        assert np.array_equal(j["ball"].cpu().numpy(), ref["ball"])


def test_shards(vga, graphs):
    torch = pytest.importorskip("torch")
    from paper_2604_08374_gb300.sharded import hyperball_run_sharded_local
    g, off, b = graphs[3]
    md = torch.empty(g.n_nodes, dtype=torch.float64, device="cuda")
    ball = torch.empty_like(md)
    it = hyperball_run_sharded_local(g, 8, 0, 3, 4, md, ball, slice_bytes=16)
    ref = oracle.hyperball(off, b, 8, 0, seed=3)
    assert it == ref["iterations"]
    assert np.array_equal(md.cpu().numpy(), ref["mean_depth"], equal_nan=True)


def test_server(vga, graphs):
    with vga.Server(hbm_budget_bytes=4 << 30, solo_nodes=1000) as srv:
        ids = [(srv.submit(g, 10, 3, 9), off, b) for g, off, b in graphs]
        for rid, off, b in ids:
            out = srv.wait(rid, timeout_s=120)
            ref = oracle.hyperball(off, b, 10, 3, seed=9)
            assert out["iterations"] == ref["iterations"]
            assert np.array_equal(out["mean_depth"], ref["mean_depth"], equal_nan=True)
