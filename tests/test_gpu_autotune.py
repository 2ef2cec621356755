"""GPU tests of the autotuner (vga_autotune, vga_tune_table_*).

The tuner may pick any launch shape, so what is checked is that (1) it
returns one valid entry per degree bucket, (2) an installed table really
steers the runs that leave their tuning at 0 (the profile records the variant
and slice width used), and (3) results under the tuned choices are exactly
the oracle's, single-graph and batched.
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
    yield v
    v.vga_tune_table_set([])


@pytest.fixture(scope="module")
def graphs(vga):
    grids = [workloads.tiny(1), workloads.tiny(2),
             workloads.rectangles_until(96, 96, (2, 12), int(96 * 96 * 0.88), seed=4),
             workloads.open_grid(12, 10)]
    out = []
    for obst in grids:
        off, b, _ = oracle.build_graph(obst)
        out.append((vga.vga_graph_load(off, b), off, b))
    yield out
    for g, _, _ in out:
        g.free()


def _bucket(g):
    return int(np.floor(np.log2(g.n_edges // g.n_nodes)))


def test_autotune_entries_and_steering(vga, graphs):
    gs = [g for g, _, _ in graphs]
    entries = vga.vga_autotune(gs, p=8, install=True)
    buckets = {_bucket(g) for g in gs}
    assert {e["degree_log2"] for e in entries} == buckets
    for e in entries:
        assert e["union_mode"] in (1, 2) and e["warps_per_cta"] in (4, 8, 16) and e["p"] == 8
        assert 16 <= e["slice_bytes"] <= 256 and e["geu_per_s"] > 0
        assert e["group_nodes"] in (0, 1, 2, 8)
    assert vga.vga_tune_table_get() == entries
    # every graph runs with its bucket's variant and width, and stays exact
    by_bucket = {e["degree_log2"]: e for e in entries}
    for g, off, b in graphs:
        e = by_bucket[_bucket(g)]
        vga.vga_profile_reset()
        vga.vga_profile_enable(True)
        got = vga.hyperball_run_trace(g, 8, 0, seed=3, max_trace=10)
        vga.vga_profile_enable(False)
        prof = vga.vga_profile_read()
        assert prof["union_mode"] == e["union_mode"]
        assert prof["slice_bytes"] <= e["slice_bytes"]
        ref = oracle.hyperball(off, b, 8, 0, seed=3, trace=10)
        assert got["iterations"] == ref["iterations"]
        for t in range(ref["iterations"] + 1):
            assert np.array_equal(got["regs"][t], ref["regs"][t])
        assert np.array_equal(got["mean_depth"], ref["mean_depth"], equal_nan=True)


def test_tuned_table_in_batch(vga, graphs):
    torch = pytest.importorskip("torch")
    gs = [g for g, _, _ in graphs]
    table = {}
    for g in gs:
        table.setdefault(_bucket(g), {"degree_log2": _bucket(g), "union_mode": 1 + len(table) % 2,
                                      "slice_bytes": 32, "warps_per_cta": 8})
    vga.vga_tune_table_set(list(table.values()))
    jobs = []
    for g, off, b in graphs:
        n = g.n_nodes
        jobs.append(dict(graph=g, p=8, d=0, seed=11, mean_depth=torch.empty(n, dtype=torch.float64, device="cuda"),
                         ball=torch.empty(n, dtype=torch.float64, device="cuda")))
    its = vga.hyperball_run_batch(jobs, use_graph=True)
    for j, (g, off, b), it in zip(jobs, graphs, its):
        ref = oracle.hyperball(off, b, 8, 0, seed=11)
        assert it == ref["iterations"]
        assert np.array_equal(j["mean_depth"].cpu().numpy(), ref["mean_depth"], equal_nan=True)
    vga.vga_tune_table_set([])
    assert vga.vga_tune_table_get() == []


@pytest.mark.parametrize("group_nodes", [1, 2, 8])
def test_tuned_group_size_single_and_batch(vga, graphs, group_nodes):
    # a tuned group size steers single runs (any of 1, 2, 8) and batched jobs
    # (the engine honours 1 and groups 4 nodes otherwise); results stay exact
    torch = pytest.importorskip("torch")
    gs = [g for g, _, _ in graphs]
    table = {}
    for g in gs:
        table.setdefault(_bucket(g), {"degree_log2": _bucket(g), "union_mode": 2, "slice_bytes": 64,
                                      "warps_per_cta": 4, "group_nodes": group_nodes})
    vga.vga_tune_table_set(list(table.values()))
    try:
        jobs = []
        for g, off, b in graphs:
            ref = oracle.hyperball(off, b, 8, 0, seed=21, trace=10)
            got = vga.hyperball_run_trace(g, 8, 0, seed=21, max_trace=10)
            assert got["iterations"] == ref["iterations"]
            for t in range(ref["iterations"] + 1):
                assert np.array_equal(got["regs"][t], ref["regs"][t])
            n = g.n_nodes
            jobs.append(dict(graph=g, p=8, d=0, seed=21,
                             mean_depth=torch.empty(n, dtype=torch.float64, device="cuda"),
                             ball=torch.empty(n, dtype=torch.float64, device="cuda")))
        its = vga.hyperball_run_batch(jobs, use_graph=False)
        for j, (g, off, b), it in zip(jobs, graphs, its):
            ref = oracle.hyperball(off, b, 8, 0, seed=21)
            assert it == ref["iterations"]
            assert np.array_equal(j["mean_depth"].cpu().numpy(), ref["mean_depth"], equal_nan=True)
    finally:
        vga.vga_tune_table_set([])


def test_tune_table_rejects_bad_entries(vga):
    for bad in ({"degree_log2": 3, "union_mode": 3, "slice_bytes": 64},
                {"degree_log2": 3, "union_mode": 2, "slice_bytes": 64, "group_nodes": 3},
                {"degree_log2": 3, "union_mode": 1, "slice_bytes": 48},
                {"degree_log2": 3, "union_mode": 2, "slice_bytes": 64, "warps_per_cta": 17},
                {"degree_log2": 3, "union_mode": 2, "slice_bytes": 64, "hub_lookups": -1}):
        with pytest.raises(vga.VgaError) as e:
            vga.vga_tune_table_set([bad])
        assert e.value.status == vga.VGA_EINVAL
    with pytest.raises(vga.VgaError):
        vga.vga_autotune([], p=8)
