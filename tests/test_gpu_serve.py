"""GPU tests of the request server (vga_server_*).

Requests submitted from several threads, at random moments, over a pool of
graphs of different sizes (some above the solo-lane threshold), with mixed p,
d and convergence rules, must each give exactly the result of the same
analysis run alone (bit for bit; the stated mean-depth tolerance 1e-6 is
asserted too).  A tight HBM budget forces requests to queue for admission;
they must still all complete, and the budget must never be exceeded.
"""
import threading
import time

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
def pool(vga):
    grids = [workloads.tiny(s) for s in (1, 2, 3, 4)]
    grids += [workloads.rectangles_until(96, 96, (2, 12), int(96 * 96 * 0.88), seed=4),
              workloads.rectangles_until(70, 64, (2, 9), int(70 * 64 * 0.86), seed=2),
              workloads.open_grid(3, 1)]
    gs = [vga.vga_visibility_build(o) for o in grids]
    yield gs
    for g in gs:
        g.free()


def _requests(pool, count, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        g = pool[int(rng.integers(len(pool)))]
        out.append(dict(g=g, p=int(rng.choice([6, 8, 10, 12])), d=int(rng.choice([0, 3, 5])),
                        seed=int(rng.integers(0, 2**40)), conv=int(rng.random() < 0.2)))
    return out


def _alone(vga, r):
    md, ball, it = None, None, None
    torch = pytest.importorskip("torch")
    n = r["g"].n_nodes
    md = torch.empty(n, dtype=torch.float64, device="cuda")
    ball = torch.empty(n, dtype=torch.float64, device="cuda")
    it = vga.hyperball_run_dev(r["g"], r["p"], r["d"], r["seed"], md, ball, conv_mode=r["conv"])
    return md.cpu().numpy(), ball.cpu().numpy(), it


def _check(vga, reqs, results):
    for r, out in zip(reqs, results):
        md, ball, it = _alone(vga, r)
        assert out["iterations"] == it
        np.testing.assert_allclose(out["mean_depth"], md, rtol=1e-6)
        assert np.array_equal(out["mean_depth"], md, equal_nan=True)
        assert np.array_equal(out["ball"], ball)
        assert out["latency_s"] >= out["queued_s"] >= 0


@pytest.mark.parametrize("solo_nodes,lane_priority", [(3000, 0), (1 << 30, 0), (3000, 1), (3000, -1)])
def test_mixed_requests_match_solo_runs(vga, pool, solo_nodes, lane_priority):
    reqs = _requests(pool, 40, seed=solo_nodes % 97)
    with vga.Server(hbm_budget_bytes=8 << 30, max_batch=16, solo_nodes=solo_nodes,
                    lane_priority=lane_priority) as srv:
        ids = [None] * len(reqs)

        def client(lo, hi, delay):
            for k in range(lo, hi):
                ids[k] = srv.submit(reqs[k]["g"], reqs[k]["p"], reqs[k]["d"], reqs[k]["seed"], reqs[k]["conv"])
                time.sleep(delay)

        threads = [threading.Thread(target=client, args=(0, 20, 0.002)),
                   threading.Thread(target=client, args=(20, 40, 0.0005))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        results = [srv.wait(i, timeout_s=120) for i in ids]
        st = srv.stats()
    assert st["submitted"] == st["completed"] == len(reqs)
    assert st["batched_peak"] >= 1
    _check(vga, reqs, results)


def test_tight_budget_queues_requests(vga, pool):
    reqs = _requests(pool, 24, seed=5)
    budget = 24 << 20
    # a run-aware job holds two register copies and five table rows per node
    # and slice (N x m bytes each) plus 56 bytes of per-node doubles
    reqs = [r for r in reqs if r["g"].n_nodes * (7 << r["p"]) + 64 * r["g"].n_nodes + 4096 < budget // 2]
    assert len(reqs) >= 6
    with vga.Server(hbm_budget_bytes=budget, max_batch=8, solo_nodes=1 << 30) as srv:
        ids = [srv.submit(r["g"], r["p"], r["d"], r["seed"], r["conv"]) for r in reqs]
        results = [srv.wait(i, timeout_s=120) for i in ids]
        st = srv.stats()
    assert st["budget_peak"] <= budget
    assert st["budget_used"] == 0
    assert max(r["queued_s"] for r in results) > 0
    _check(vga, reqs, results)


def test_server_errors(vga, pool):
    with vga.Server(hbm_budget_bytes=1 << 20, max_batch=4) as srv:
        big = max(pool, key=lambda g: g.n_nodes)
        with pytest.raises(vga.VgaError) as e:
            srv.submit(big, 12, 3)  # needs far more than 1 MiB
        assert e.value.status == vga.VGA_EBUSY
        with pytest.raises(vga.VgaError) as e:
            srv.submit(big, 3, 3)
        assert e.value.status == vga.VGA_EINVAL
        rid = srv.submit(pool[-1], 4, 0)   # 3 nodes: tiny
        out = srv.wait(rid, timeout_s=60)
        off, b, _ = oracle.build_graph(workloads.open_grid(3, 1))
        ref = oracle.hyperball(off, b, 4, 0)
        assert out["iterations"] == ref["iterations"]
        assert np.array_equal(out["mean_depth"], ref["mean_depth"])


def test_server_rejects_bad_lane_settings(vga):
    for kw in (dict(lane_priority=2), dict(lane_priority=-2), dict(batched_share=101)):
        with pytest.raises(vga.VgaError) as e:
            vga.Server(hbm_budget_bytes=1 << 20, **kw)
        assert e.value.status == vga.VGA_EINVAL
