"""GPU parity: the CUDA sieve (through the C ABI) against the CPU oracle on the same seeded inputs.

Tolerance: 1e-10 relative for the FP64 path (the paper's complex128 path, App. B.4; the oracle sums
its fp64 terms exactly with math.fsum). Where the value is near zero by cancellation (odd N with
gamma = 0) the bar is relative to the sum of |terms|, which the oracle supplies."""
import math
import os

import numpy as np
import pytest

from oracle import lhaf_oracle as lo
from paper_2108_01622_gb300 import workloads as wl
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


@pytest.fixture(scope="module")
def ctx(lg):
    c = lg.Context(0)
    yield c
    c.close()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


SMALL = [(2, 1, 0, 3), (4, 0, 0, 2), (3, 2, 2, 1), (1, 1, 1), (5, 0, 0, 0), (2, 2, 2, 2), (1,), (2,),
         (3, 1), (6, 1, 1), (0, 3, 0, 4), (1, 1, 1, 1, 1, 1, 1, 1), (2, 2, 1, 1, 0, 3), (7, 5),
         (1, 1, 1, 1, 1, 1, 1, 1, 1), (3, 3, 3, 3, 1)]


@pytest.mark.parametrize("reps", SMALL)
@pytest.mark.parametrize("loops", [True, False])
def test_small_patterns_vs_oracle(ctx, reps, loops):
    p = wl.small_problem(seed=sum(reps) + 31 * len(reps), M=len(reps), reps=reps, loops=loops)
    ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
    got = ctx.lhaf(p.B, p.gamma, p.reps)
    if abs(ref) < 1e-12:
        assert abs(got) < 1e-11
    else:
        assert rel(got, ref) < TOL, (got, ref)


def test_empty_pattern_is_one(ctx):
    p = wl.small_problem(1, 3, (0, 0, 0))
    assert ctx.lhaf(p.B, p.gamma, p.reps) == 1.0


@pytest.mark.parametrize("team", ["8", "16", "32", "64", "128"])
def test_every_team_size_agrees(ctx, team, monkeypatch):
    p = wl.single_lhaf_24(seed=11, n_photons=14)
    ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
    monkeypatch.setenv("LHAF_TEAM", team)
    got, st = ctx.lhaf(p.B, p.gamma, p.reps, stats=True)
    assert st["team"] == int(team)
    assert rel(got, ref) < TOL
    p2 = wl.collision_lhaf_40(seed=12, n_modes=8, n_photons=14)
    ref2 = lo.lhaf_repeated(p2.B, p2.gamma, p2.reps)
    assert rel(ctx.lhaf(p2.B, p2.gamma, p2.reps), ref2) < TOL


def test_collision_free_24_photons(ctx):
    # 24-mode Haar kernel, one photon per mode: 2^11 evaluated terms, working dimension 25
    p = wl.single_lhaf_24(seed=1)
    ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
    got, st = ctx.lhaf(p.B, p.gamma, p.reps, stats=True)
    assert st["terms"] == 2 ** 11 and st["n_dim"] == 25 and st["h"] == 12
    assert rel(got, ref) < TOL


def test_collision_pattern_40_photons(ctx):
    # 100-mode Haar kernel, 40 photons over 22 modes, counts 1..4, gamma = 0
    p = wl.collision_lhaf_40(seed=2)
    ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
    got, st = ctx.lhaf(p.B, p.gamma, p.reps, stats=True)
    assert rel(got, ref) < TOL
    # the explicit duplicated-row sieve (every photon paired singly) gives the same value
    dup = ctx.lhaf(p.B, p.gamma, p.reps, flags=0x8)
    assert rel(dup, ref) < TOL


def test_odd_pattern_without_loops_is_zero(ctx):
    p = wl.small_problem(5, 5, (3, 1, 2, 0, 1), loops=False)
    got = ctx.lhaf(p.B, p.gamma, p.reps)
    assert abs(got) < 1e-12


def test_range_partials_add_up(ctx, lg):
    p = wl.single_lhaf_24(seed=3, n_photons=18)
    T, nd, h, P = lg.plan(p.reps)
    full = ctx.lhaf(p.B, p.gamma, p.reps)
    cuts = [0, 7, 100, 101, T // 2, T]
    parts = [ctx.lhaf_range(p.B, p.gamma, p.reps, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    assert rel(lg.combine(np.array(parts), h), full) < 1e-13
    empty = ctx.lhaf_range(p.B, p.gamma, p.reps, 5, 5)
    assert np.all(empty == 0)


def test_device_pointer_path_matches_host(ctx):
    import torch

    p = wl.collision_lhaf_40(seed=7, n_modes=10, n_photons=20)
    p.gamma = wl.complex_normal(np.random.default_rng(0), len(p.gamma))
    host = ctx.lhaf(p.B, p.gamma, p.reps)
    Bd = torch.from_numpy(p.B).cuda()
    gd = torch.from_numpy(p.gamma).cuda()
    out = ctx.lhaf(Bd, gd, p.reps)
    torch.cuda.synchronize()
    assert rel(complex(out.cpu()[0]), host) < 1e-14
    ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
    assert rel(host, ref) < TOL


def test_gamma_none_uses_diagonal(ctx):
    p = wl.small_problem(9, 4, (2, 1, 1, 2))
    ref = lo.lhaf_repeated(p.B, np.diag(p.B).copy(), p.reps)
    assert rel(ctx.lhaf(p.B, None, p.reps), ref) < TOL


def test_invalid_inputs_are_rejected(ctx, lg):
    p = wl.small_problem(9, 3, (1, 1, 1))
    bad = p.B.copy()
    bad[0, 1] = np.nan
    with pytest.raises(lg.LhafError) as e:
        ctx.lhaf(bad, p.gamma, p.reps)
    assert e.value.status == 1
    with pytest.raises(lg.LhafError) as e:
        ctx.lhaf(p.B, p.gamma, (1, -2, 1))
    assert e.value.status == 1


def test_fp32_terms_stated_error(ctx):
    # FP32 per-term arithmetic, double-double accumulation: error stated against the FP64 oracle
    p = wl.single_lhaf_24(seed=1, n_photons=16)
    ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
    got = ctx.lhaf(p.B, p.gamma, p.reps, flags=0x2)
    assert rel(got, ref) < 1e-3


def test_plain_accumulation_close(ctx):
    p = wl.single_lhaf_24(seed=1)
    a = ctx.lhaf(p.B, p.gamma, p.reps)
    b = ctx.lhaf(p.B, p.gamma, p.reps, flags=0x4)
    assert rel(b, a) < 1e-11


@pytest.mark.parametrize("seed,loops", [(21, False), (22, True), (23, True)])
def test_zero_digit_groups_match_full_matrix_and_oracle(ctx, lg, seed, loops):
    # collision patterns (counts 1..4): pairs with even eta run as zero-digit groups by default
    p = wl.collision_lhaf_40(seed=seed, n_modes=9, n_photons=19 if loops else 18)
    if loops:
        p.gamma = wl.complex_normal(np.random.default_rng(seed), len(p.gamma))
    ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
    split, st = ctx.lhaf(p.B, p.gamma, p.reps, stats=True)
    full, st0 = ctx.lhaf(p.B, p.gamma, p.reps, flags=lg.NO_ZERO_SPLIT, stats=True)
    assert st["terms"] == lg.plan(p.reps)[0] and st0["terms"] == lg.plan(p.reps, flags=lg.NO_ZERO_SPLIT)[0]
    assert rel(split, ref) < TOL and rel(full, ref) < TOL
    assert st["flops_model"] < st0["flops_model"]


@pytest.mark.parametrize("force", ["0", "1"])
def test_working_dimension_classes_same_value(ctx, lg, monkeypatch, force):
    # the sieves of one loop hafnian launched in classes of equal working dimension (the default
    # for large sieves) or all in one launch: the same value (the oracle's) either way, for the
    # zero-digit groups and for the eigenvalue-trace sieves
    monkeypatch.setenv("LHAF_ND_CLASSES", force)
    p = wl.collision_lhaf_40(seed=22, n_modes=9, n_photons=19)
    p.gamma = wl.complex_normal(np.random.default_rng(22), len(p.gamma))
    ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
    assert rel(ctx.lhaf(p.B, p.gamma, p.reps), ref) < TOL
    q = wl.small_problem(seed=5, M=7, reps=(2, 1, 1, 3, 1, 2, 1), loops=True)
    assert rel(ctx.lhaf(q.B, q.gamma, q.reps, flags=lg.ET), lo.lhaf_repeated(q.B, q.gamma, q.reps)) < TOL
    # degree 25, 16 zero-digit groups (a well-conditioned instance: sum |terms| / |sum| = 3.9e3),
    # with the series staged (default up to degree 32) and inline in the terms kernel
    u = wl.small_problem(seed=2, M=8, reps=(8, 8, 8, 8, 6, 6, 4, 2), loops=True, scale=1.0)
    ref_u = lo.lhaf_repeated(u.B, u.gamma, u.reps)
    assert rel(ctx.lhaf(u.B, u.gamma, u.reps), ref_u) < TOL
    monkeypatch.setenv("LHAF_STAGE", "0")
    assert rel(ctx.lhaf(u.B, u.gamma, u.reps), ref_u) < TOL


def test_zero_digit_range_partials_cross_groups(ctx, lg):
    p = wl.collision_lhaf_40(seed=12, n_modes=8, n_photons=16)
    p.gamma = wl.complex_normal(np.random.default_rng(3), len(p.gamma))
    T, nd, h, P = lg.plan(p.reps)
    full = ctx.lhaf(p.B, p.gamma, p.reps)
    cuts = sorted({0, 1, 3, T // 5, T // 3, T // 2 + 1, T - 1, T})
    parts = [ctx.lhaf_range(p.B, p.gamma, p.reps, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    assert rel(lg.combine(np.array(parts), h), full) < 1e-13
    assert rel(full, lo.lhaf_repeated(p.B, p.gamma, p.reps)) < TOL
    with pytest.raises(lg.LhafError):
        ctx.lhaf_range(p.B, p.gamma, p.reps, 0, T + 1)


@pytest.mark.parametrize("series", ["staged", "inline"])
@pytest.mark.parametrize("loops", [False, True])
def test_zero_digit_groups_inline_series(ctx, lg, loops, series, monkeypatch):
    # h = 25 > the staged-series limit: the groups finish their series inside the team. Repeat
    # counts 6-7 make the signed sum cancel by ~1e8 (sum |terms| / |lhaf|), beyond what an FP64
    # sum can resolve to 1e-10, so the reference is the oracle in extended precision and the bar
    # is the forward error of the sum: 1e-13 * sum |terms| * 2^-h (each term carries a relative
    # error of order 1e-15; measured about 1e-15).
    if series == "inline":
        monkeypatch.setenv("LHAF_STAGE", "0")
    reps = (7, 7, 6, 6, 6, 6, 6, 6)
    p = wl.small_problem(seed=77, M=len(reps), reps=reps, loops=loops)
    ref = complex(lo.lhaf_repeated(p.B, p.gamma, p.reps, dtype=np.clongdouble))
    scale = sum(abs(t) for t in lo.repeated_sieve_terms(p.B, p.gamma, p.reps)) / 2.0 ** 25
    got, st = ctx.lhaf(p.B, p.gamma, p.reps, stats=True)
    full = ctx.lhaf(p.B, p.gamma, p.reps, flags=lg.NO_ZERO_SPLIT)
    assert st["h"] == 25 and lg.plan_groups(reps) == 8
    assert abs(got - ref) <= 1e-13 * scale and abs(full - ref) <= 1e-13 * scale


@pytest.mark.parametrize("reps", [(25, 25), (33, 33)])
def test_inline_series_well_conditioned(ctx, lg, reps):
    # h = 25 (staged) and h = 33 (above the staging limit: inline) with single repeats over two
    # modes, no zero-digit split
    p = wl.small_problem(seed=5, M=2, reps=reps, loops=True)
    ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
    got, st = ctx.lhaf(p.B, p.gamma, p.reps, stats=True)
    assert st["h"] == reps[0] and lg.plan_groups(reps) == 0
    assert rel(got, ref) < TOL


def test_zero_digit_groups_device_pointers_and_fp32(ctx, lg):
    import torch

    p = wl.collision_lhaf_40(seed=31, n_modes=10, n_photons=22)
    ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
    Bd = torch.from_numpy(p.B).cuda()
    gd = torch.from_numpy(p.gamma).cuda()
    out = ctx.lhaf(Bd, gd, p.reps, flags=lg.NO_LOOPS)
    torch.cuda.synchronize()
    assert rel(complex(out.cpu()[0]), ref) < TOL
    out = ctx.lhaf(Bd, gd, p.reps)  # loop border kept (gamma = 0 on the device is not inspected)
    torch.cuda.synchronize()
    assert rel(complex(out.cpu()[0]), ref) < TOL
    assert rel(ctx.lhaf(p.B, p.gamma, p.reps, flags=lg.FP32_TERMS), ref) < 1e-3


@pytest.mark.parametrize("flags", [0, 0x40])
def test_staging_reuse_with_more_coefficient_rows(ctx, flags):
    _staging_reuse(ctx, flags)


def _staging_reuse(ctx, flags):
    # A staged call with many terms and few coefficient rows, then a new problem shape with more
    # rows and few terms (autotuned on its first call): both must match the oracle.
    p1 = wl.collision_lhaf_40(seed=2)  # no loops: h = 20 rows, 34,560 terms
    assert rel(ctx.lhaf(p1.B, p1.gamma, p1.reps, flags=flags), lo.lhaf_repeated(p1.B, p1.gamma, p1.reps)) < TOL
    b = wl.chain_rule_batch(seed=3, count=64)
    for i in range(len(b.reps)):
        r = b.reps[i]
        if 30 <= r.sum() <= 34:  # loops: 2h + 1 rows
            got = ctx.lhaf(b.B, b.gammas[i], r, flags=flags)
            assert rel(got, lo.lhaf_repeated(b.B, b.gammas[i], r)) < TOL
            break
