"""CPU tests of the register-shard driver (paper_2604_08374_gb300.sharded)
over gloo ranks (world sizes 2 and 3), with a numpy stand-in for the
library's shard object.

The stand-in keeps only its rank's register columns, unions them, and writes
the same partial block as the library (u64 partial harmonic sums, then u32
zero counts, at 256-byte aligned offsets).  The driver's all-gather, flag
reduction and stop rule must then reproduce the oracle's whole-counter run:
iterations, mean depth and ball sizes.  The kernels behind the real shard
object are checked against unsharded runs on the GPU.
"""
import math
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _align256(x):
    return (x + 255) // 256 * 256


class FakeShard:
    def __init__(self, off, b, p, seed, rank, world, S):
        import oracle
        n = len(off) - 1
        m = 1 << p
        slices = m // S
        s0, s1 = rank * slices // world, (rank + 1) * slices // world
        self.n, self.p, self.m, self.K = n, p, m, 65 - p
        self.cur = oracle.hll_init(n, p, seed)[:, s0 * S:s1 * S].copy()
        rp, col = oracle.decode_csr(off, b)
        self.nbrs = [col[rp[v]:rp[v + 1]].astype(np.int64) for v in range(n)]
        self.zeros_off = _align256(8 * n)
        self.partial_bytes = self.zeros_off + _align256(4 * n)
        self.alpha_mm = oracle.hll_alpha(p) * m * m
        self.c_prev = np.zeros(n)
        self.sum_d = np.zeros(n)
        self.t = -1

    def _write(self, buf):
        M = self.cur.astype(np.uint64)
        terms = np.where(M > 0, np.left_shift(np.uint64(1), (np.uint64(self.K) - M) % np.uint64(64)), 0)
        a = buf.numpy()
        a[: 8 * self.n].view(np.uint64)[:] = terms.sum(axis=1, dtype=np.uint64)
        a[self.zeros_off: self.zeros_off + 4 * self.n].view(np.uint32)[:] = (self.cur == 0).sum(axis=1)

    def start(self, own, stream):
        self._write(own)
        self.t = 0

    def union(self, own, stream):
        nxt = self.cur.copy()
        for v, nb in enumerate(self.nbrs):
            if len(nb):
                nxt[v] = np.maximum(nxt[v], self.cur[nb].max(axis=0))
        changed = int(not np.array_equal(nxt, self.cur))
        self.cur = nxt
        self._write(own)
        self.t += 1
        return changed

    def estimate(self, allp, stream):
        a = allp.numpy()
        blocks = len(a) // self.partial_bytes
        c = np.empty(self.n)
        for v in range(self.n):
            total, zeros = 0, 0
            for k in range(blocks):
                blk = a[k * self.partial_bytes:(k + 1) * self.partial_bytes]
                total += int(blk[: 8 * self.n].view(np.uint64)[v])
                zeros += int(blk[self.zeros_off: self.zeros_off + 4 * self.n].view(np.uint32)[v])
            Z = float(zeros * (1 << self.K) + total) * 2.0 ** -self.K
            E = self.alpha_mm / Z
            c[v] = self.m * math.log(self.m / zeros) if (E <= 2.5 * self.m and zeros > 0) else E
        inc = 0
        if self.t > 0:
            diff = c - self.c_prev
            self.sum_d = self.sum_d + self.t * diff
            inc = int((diff > 0.5).any())
        self.c_prev = c
        return inc

    def finalize(self, md, ball, stream):
        md.numpy()[:] = self.sum_d / (self.n - 1)
        ball.numpy()[:] = self.c_prev


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist

    import oracle
    import workloads
    from paper_2604_08374_gb300.sharded import hyperball_run_sharded
    dist.init_process_group("gloo", rank=rank, world_size=world)
    off, b, cells = oracle.build_graph(workloads.tiny(case["grid"]))
    n = len(cells)
    md = torch.empty(n, dtype=torch.float64)
    ball = torch.empty(n, dtype=torch.float64)
    it = hyperball_run_sharded(None, case["p"], case["d"], case["seed"], md, ball, conv_mode=case["conv"],
                               shard_factory=lambda r, w: FakeShard(off, b, case["p"], case["seed"], r, w,
                                                                    case["S"]))
    out[rank] = (it, md.numpy().copy(), ball.numpy().copy())
    dist.destroy_process_group()


@pytest.mark.parametrize("world,case", [
    (2, dict(grid=1, p=8, d=0, seed=3, conv=0, S=32)),
    (3, dict(grid=2, p=6, d=3, seed=7, conv=0, S=16)),
    (2, dict(grid=3, p=8, d=0, seed=1, conv=1, S=64)),
])
def test_sharded_driver_matches_oracle(world, case):
    import oracle
    import workloads
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    off, b, _ = oracle.build_graph(workloads.tiny(case["grid"]))
    ref = oracle.hyperball(off, b, case["p"], case["d"], seed=case["seed"], conv_mode=case["conv"])
    for r in range(world):
        it, md, ball = out[r]
        assert it == ref["iterations"]
        assert np.array_equal(md, ref["mean_depth"], equal_nan=True)
        assert np.array_equal(ball, ref["ball"])
