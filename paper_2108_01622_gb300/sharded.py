"""Loop hafnians split over ranks (one process per GPU).

The sieve terms of Eq. fdsieve are independent (App. B.6 distributes them over MPI ranks), so a
single loop hafnian shards by contiguous term ranges: each rank sums its range with
``Context.lhaf_range`` (an unscaled double-double partial of 4 doubles), one all-gather moves the
partials, and ``combine`` adds them in double-double and applies the exact 2^-h. A batch shards
by items, assigned longest-processing-time first on the per-item flop model; one all-reduce of a
zero-filled result vector assembles it (x + 0 is exact, so the sum is the owner's value).

The collectives run through ``torch.distributed`` (``gloo`` on the host, ``nccl`` with CUDA
tensors); no kernel waits on another rank.
"""
from __future__ import annotations

import heapq
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import BATCH_B_PER_ITEM, combine, flops_per_term, plan


def term_shard(T: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous range [begin, end) of the T sieve terms owned by `rank` (sizes differ by <= 1)."""
    if world <= 0 or not 0 <= rank < world or T < 0:
        raise ValueError("invalid shard")
    q, r = divmod(T, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def item_shard(costs: Sequence[float], world: int) -> List[List[int]]:
    """Items per rank, longest processing time first: each item, in order of decreasing cost, goes
    to the rank with the least assigned cost (ties: lowest rank)."""
    if world <= 0:
        raise ValueError("invalid world size")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(world)]
    owned: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        owned[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(o) for o in owned]


def item_costs(reps, flags: int = 0) -> np.ndarray:
    """Model flops of each item's sieve (terms x flops per term of the bordered problem)."""
    r = np.asarray(reps, dtype=np.int32)
    out = np.zeros(r.shape[0])
    for i, row in enumerate(r):
        if int(row.sum()) == 0:
            continue
        T, nd, h, _ = plan(row, flags, True)
        out[i] = T * flops_per_term(nd, h, True)
    return out


def _dist(group):
    import torch.distributed as dist

    if not dist.is_initialized():
        raise RuntimeError("torch.distributed is not initialised")
    return dist, dist.get_rank(group), dist.get_world_size(group)


def _device_for(dist, group):
    import torch

    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")


def gather_partials(part, group=None) -> np.ndarray:
    """All-gather of n 4-double partials per rank (the same n on every rank) -> (world * n) x 4
    array in rank order (so in term order when each rank's partials are in term order)."""
    import torch

    dist, _, world = _dist(group)
    t = torch.as_tensor(np.ascontiguousarray(np.asarray(part, dtype=np.float64).reshape(-1, 4)))
    t = t.to(_device_for(dist, group))
    outs = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(outs, t, group=group)
    return np.concatenate([o.cpu().numpy() for o in outs], axis=0)


def lhaf_sharded(ctx, B, gamma=None, reps=None, flags: int = 0, group=None) -> complex:
    """lhaf(B_n) with the sieve terms split over the ranks of `group`; every rank returns the value.
    `ctx` is this rank's Context (host inputs)."""
    _, rank, world = _dist(group)
    M = np.asarray(B).shape[0]
    r = np.ones(M, np.int32) if reps is None else np.asarray(reps, dtype=np.int32)
    if int(r.sum()) == 0:
        return 1.0 + 0j
    T, _, h, _ = plan(r, flags, True)
    b, e = term_shard(T, rank, world)
    part = ctx.lhaf_range(B, gamma, r, b, e, flags)
    return combine(gather_partials(part, group), h)


def lhaf_batched_sharded(ctx, B, gammas, reps, flags: int = 0, group=None,
                         costs: Optional[Sequence[float]] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Batch of loop hafnians with the items split over the ranks of `group` (longest processing
    time first on `costs`, default the flop model); every rank returns (values, item_status)."""
    import torch

    dist, rank, world = _dist(group)
    r = np.asarray(reps, dtype=np.int32)
    batch = r.shape[0]
    owned = item_shard(item_costs(r, flags) if costs is None else costs, world)[rank]
    vals = np.zeros(batch, np.complex128)
    status = np.zeros(batch, np.int64)
    if owned:
        idx = np.asarray(owned)
        Bi = np.asarray(B)[idx] if flags & BATCH_B_PER_ITEM else B
        gi = None if gammas is None else np.asarray(gammas)[idx]
        v, s = ctx.lhaf_batched(Bi, gi, r[idx], flags)
        vals[idx] = v
        status[idx] = s
    dev = _device_for(dist, group)
    tv = torch.as_tensor(vals.view(np.float64).copy()).to(dev)
    ts = torch.as_tensor(status).to(dev)
    dist.all_reduce(tv, group=group)
    dist.all_reduce(ts, group=group)
    return tv.cpu().numpy().view(np.complex128).copy(), ts.cpu().numpy().astype(np.int32)
