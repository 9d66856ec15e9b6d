"""Multi-rank host logic on CPU: term-range sharding of one loop hafnian and item sharding of a
batch over gloo ranks (world sizes 2 and 3). The per-rank sieve partials come from the oracle
standing in for each rank's GPU, so this checks the split, the collectives and the double-double
combine (App. B.6: independent terms, one reduction), not the kernels."""
import math
import os
import socket

import numpy as np
import pytest

from oracle import lhaf_oracle as lo
from tests.libutil import ensure_built


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _dd(xs):
    hi = math.fsum(xs)
    return hi, math.fsum(list(xs) + [-hi])


class OracleRank:
    """A rank's Context on a host without a GPU: ranges of the library's T (halved) terms map onto
    proportional ranges of the oracle's full digit-vector list, whose sum is the same total."""

    def lhaf_range(self, B, gamma, reps, b, e, flags=0):
        import paper_2108_01622_gb300 as lg

        T, _, _, _ = lg.plan(reps, flags, True)
        pairs, leftover = lo.matched_reps(list(reps))
        full = math.prod(eta + 1 for _, _, eta in pairs) * (2 if leftover is not None else 1)
        gamma = np.diag(B) if gamma is None else gamma
        terms = lo.repeated_sieve_terms(B, gamma, list(reps), b * full // T, e * full // T)
        rh, rl = _dd([t.real for t in terms])
        ih, il = _dd([t.imag for t in terms])
        return np.array([rh, rl, ih, il])

    def lhaf_batched(self, B, gammas, reps, flags=0):
        vals = np.array([lo.lhaf_repeated(B, np.diag(B) if gammas is None else gammas[i], list(row))
                         for i, row in enumerate(reps)], dtype=np.complex128)
        return vals, np.zeros(len(reps), np.int32)


def _problem(seed, M):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))
    return (X + X.T) / 4, (rng.normal(size=M) + 1j * rng.normal(size=M)) / 2


def _worker(rank, world, port):
    import torch.distributed as dist

    import paper_2108_01622_gb300 as lg
    from paper_2108_01622_gb300 import sharded

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ctx = OracleRank()
        B, g = _problem(7, 5)
        cases = [
            ([2, 1, 0, 3, 1], g),    # repeated pairs, odd N (pad pair)
            ([1, 1, 1, 1, 1], g),    # no repeats
            ([2, 0, 0, 0, 0], g),    # a single term: ranks without work
            ([0, 0, 0, 0, 0], g),    # empty pattern
            ([2, 2, 1, 1, 0], None), # loops from diag(B)
        ]
        for reps, gam in cases:
            want = lo.lhaf_repeated(B, np.diag(B) if gam is None else gam, reps)
            got = sharded.lhaf_sharded(ctx, B, gam, reps)
            assert abs(got - want) <= 1e-12 * max(1.0, abs(want)), (reps, got, want)
        # batch split by items
        rng = np.random.default_rng(11)
        reps = rng.integers(0, 3, size=(7, 5))
        gam = (rng.normal(size=(7, 5)) + 1j * rng.normal(size=(7, 5))) / 2
        vals, status = sharded.lhaf_batched_sharded(ctx, B, gam, reps)
        for i in range(7):
            want = lo.lhaf_repeated(B, gam[i], list(reps[i]))
            assert abs(vals[i] - want) <= 1e-12 * max(1.0, abs(want)), (i, vals[i], want)
        assert (status == 0).all()
        # every rank holds the same assembled result
        allv = [None] * world
        dist.all_gather_object(allv, vals.tolist())
        assert all(v == allv[0] for v in allv)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_lhaf_and_batch_over_gloo(world):
    import torch.multiprocessing as mp

    ensure_built()
    mp.spawn(_worker, args=(world, _free_port()), nprocs=world, join=True)


@pytest.mark.parametrize("T", [0, 1, 2, 5, 17, 1 << 20, (1 << 29) + 3])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_term_shard_partitions(T, world):
    from paper_2108_01622_gb300.sharded import term_shard

    ranges = [term_shard(T, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == T
    for (b0, e0), (b1, _) in zip(ranges, ranges[1:]):
        assert e0 == b1
    sizes = [e - b for b, e in ranges]
    assert min(sizes) >= 0 and max(sizes) - min(sizes) <= 1


def test_term_shard_rejects_bad_rank():
    from paper_2108_01622_gb300.sharded import term_shard

    with pytest.raises(ValueError):
        term_shard(10, 2, 2)
    with pytest.raises(ValueError):
        term_shard(10, 0, 0)


def test_item_shard_lpt():
    from paper_2108_01622_gb300.sharded import item_shard

    rng = np.random.default_rng(3)
    costs = rng.pareto(1.5, size=200) + 0.1
    for world in (1, 2, 4, 8):
        owned = item_shard(costs, world)
        flat = sorted(i for o in owned for i in o)
        assert flat == list(range(200))
        loads = [costs[o].sum() for o in owned]
        # LPT: the last item placed on the heaviest rank went to the least-loaded rank
        assert max(loads) - min(loads) <= costs.max() + 1e-9
        assert max(loads) <= (4 / 3) * max(costs.sum() / world, costs.max()) + 1e-9


def test_item_costs_follow_the_plan():
    lg = ensure_built()
    from paper_2108_01622_gb300.sharded import item_costs

    reps = np.array([[1, 1, 1, 1], [2, 2, 0, 0], [0, 0, 0, 0]])
    c = item_costs(reps)
    T, nd, h, _ = lg.plan(reps[0], 0, True)
    assert c[0] == pytest.approx(T * lg.flops_per_term(nd, h, True))
    assert c[2] == 0.0 and c[1] > 0.0
