"""One analysis over several ranks, split by register index (vga_shard_*).

Eq. hll-union maxes each register independently, so rank k keeps slices
[s0, s1) of every node's counter and unions them alone.  Per pass the ranks
exchange one partial block each (per node: the exact partial harmonic sum and
zero count of the rank's registers) with an all-gather, from which every rank
evaluates the same c_t and Eq. sumD; the changed flags are OR-reduced for the
stop rule of Alg. 1.  Compute runs in the library's kernels; this module only
orders the calls and the collectives.

hyperball_run_sharded        one rank per process (torch.distributed group).
hyperball_run_sharded_local  all shards in one process on one device, in
                             lockstep (the same calls, the gather done by
                             placing the blocks side by side): every rank's
                             arithmetic without a second GPU.
"""
from __future__ import annotations

from typing import Callable, Optional


def _stop(conv_mode: int, any_changed: int, increase: int, t: int, d: int) -> bool:
    """Alg. 1's end of the pass loop, as in hyperball_run_dev."""
    stop = (increase == 0) if conv_mode == 1 else (any_changed == 0)
    return stop or (d > 0 and t >= d)


def hyperball_run_sharded(g, p: int, d: int, seed: int, mean_depth_dev, ball_size_dev, conv_mode: int = 0,
                          group=None, shard_factory: Optional[Callable] = None, **tuning) -> int:
    """Run the analysis (g, p, d, seed) with this rank's register shard of the
    process group; every rank ends with the same mean depth and ball sizes in
    its output tensors.  Returns the passes run.

    shard_factory(rank, world) may supply another object with the Shard
    interface (start / union / estimate / finalize / partial_bytes)."""
    import torch
    import torch.distributed as dist

    if g is not None and g.n_nodes == 0:
        return 0  # no node, no pass (as hyperball_run_dev)
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    if shard_factory is None:
        from . import vga_shard_create
        sh = vga_shard_create(g, p, seed, rank, world, **tuning)
    else:
        sh = shard_factory(rank, world)
    dev = mean_depth_dev.device if hasattr(mean_depth_dev, "device") else torch.device("cuda")
    stream = torch.cuda.current_stream(dev) if dev.type == "cuda" else None
    pb = sh.partial_bytes
    own = torch.empty(pb, dtype=torch.uint8, device=dev)
    parts = [torch.empty_like(own) for _ in range(world)]
    allp = torch.empty(world * pb, dtype=torch.uint8, device=dev)

    def exchange():
        dist.all_gather(parts, own, group=group)
        torch.cat(parts, out=allp)

    def any_changed(changed: int) -> int:
        flag = torch.tensor([changed], dtype=torch.int32, device=dev)
        dist.all_reduce(flag, op=dist.ReduceOp.MAX, group=group)
        return int(flag.item())

    try:
        sh.start(own, stream)
        exchange()
        sh.estimate(allp, stream)
        t = 0
        while True:
            t += 1
            changed = sh.union(own, stream)
            exchange()
            increase = sh.estimate(allp, stream)
            if _stop(conv_mode, any_changed(changed), increase, t, d):
                break
        sh.finalize(mean_depth_dev, ball_size_dev, stream)
    finally:
        if shard_factory is None:
            sh.free()
    return t


def hyperball_run_sharded_local(g, p: int, d: int, seed: int, n_shards: int, mean_depth_dev=None,
                                ball_size_dev=None, conv_mode: int = 0, stream=None, **tuning) -> int:
    """All n_shards register shards of one analysis in this process, on the
    current device, step by step as the ranks of hyperball_run_sharded would
    run them.  Shard 0 writes the outputs; every shard's estimate is checked
    to agree on the paper's increase flag.  Returns the passes run."""
    import torch

    from . import vga_shard_create
    if g.n_nodes == 0:
        return 0
    shards = [vga_shard_create(g, p, seed, k, n_shards, **tuning) for k in range(n_shards)]
    try:
        pb = shards[0].partial_bytes
        allp = torch.empty(n_shards * pb, dtype=torch.uint8, device="cuda")
        own = [allp[k * pb:(k + 1) * pb] for k in range(n_shards)]
        for sh, blk in zip(shards, own):
            sh.start(blk, stream)
        for sh in shards:
            sh.estimate(allp, stream)
        t = 0
        while True:
            t += 1
            changed = max(sh.union(blk, stream) for sh, blk in zip(shards, own))
            increases = {sh.estimate(allp, stream) for sh in shards}
            if len(increases) != 1:
                raise RuntimeError("shards disagree on the estimate")
            if _stop(conv_mode, changed, increases.pop(), t, d):
                break
        shards[0].finalize(mean_depth_dev, ball_size_dev, stream)
    finally:
        for sh in shards:
            sh.free()
    return t
