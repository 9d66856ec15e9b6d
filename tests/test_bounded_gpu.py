"""Bounded launches and checkpoint/resume on the 60-photon collision-free loop hafnian (working
dimension 61, degree 30), with the series staged (the default up to degree 32) and finished inside
the team. Every launch of the sieve-term kernel covers at most the flop budget, its terms are
summed in term order (the same bits for the same range whichever CTA took which term), and a sum interrupted between chunks and
resumed from its checkpoint equals the uninterrupted one bit for bit (App. B.6: the terms are
independent, so range partials add)."""
import math

import numpy as np
import pytest

from paper_2108_01622_gb300 import workloads as wl
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def p60():
    return wl.large_lhaf_60(seed=5)


def _val(part):
    return complex(part[0] + part[1], part[2] + part[3])


@pytest.mark.parametrize("series", ["staged", "inline"])
def test_launch_budget_splits_and_agrees(ctx, lg, p60, monkeypatch, series):
    if series == "inline":  # the series finished inside the team, per-term partials in term order
        monkeypatch.setenv("LHAF_STAGE", "0")
    S = 1 << 13
    T, nd, h, _ = lg.plan(p60.reps)
    assert (T, nd, h) == (1 << 29, 61, 30)
    whole, st1 = ctx.lhaf_range(p60.B, p60.gamma, p60.reps, 0, S, stats=True)
    assert st1["term_launches"] == 1
    fpt = lg.flops_per_term(nd, h, True)
    monkeypatch.setenv("LHAF_LAUNCH_MFLOPS", "1000")  # 1e9 model flops: ~600 terms per launch
    split, st2 = ctx.lhaf_range(p60.B, p60.gamma, p60.reps, 0, S, stats=True)
    tpc = max(1, 32 // st2["team"])  # terms per chunk: teams per one-warp CTA
    per_launch = math.floor(1e9 / fpt / tpc) * tpc
    assert abs(st2["term_launches"] - math.ceil(S / max(per_launch, 1))) <= 1
    assert st2["term_launches"] >= 10
    assert abs(_val(split) - _val(whole)) <= 1e-14 * abs(_val(whole))
    again = ctx.lhaf_range(p60.B, p60.gamma, p60.reps, 0, S)
    assert np.array_equal(again, split)  # the same range and launches: the same bits


def test_default_launches_stay_short(ctx, lg, p60):
    S = 1 << 18
    _, st = ctx.lhaf_range(p60.B, p60.gamma, p60.reps, 1 << 20, (1 << 20) + S, stats=True)
    assert st["term_launches"] >= 2
    assert st["kernel_ms"] / st["term_launches"] < 1000.0


def test_resumed_slice_is_bit_identical(ctx, lg, p60, tmp_path):
    from paper_2108_01622_gb300 import resumable

    b0, b1, chunk = 4096, 4096 + (1 << 14), 1 << 12
    ref = resumable.range_checkpointed(ctx, p60.B, p60.gamma, p60.reps, b0, b1, str(tmp_path / "ref.json"), chunk)

    class Stop(Exception):
        pass

    def stop(i, b, e):
        if i == 1:
            raise Stop

    path = str(tmp_path / "ck.json")
    with pytest.raises(Stop):
        resumable.range_checkpointed(ctx, p60.B, p60.gamma, p60.reps, b0, b1, path, chunk, on_chunk=stop)
    res = resumable.range_checkpointed(ctx, p60.B, p60.gamma, p60.reps, b0, b1, path, chunk)
    assert res.shape == (4, 4) and np.array_equal(res, ref)
    direct = ctx.lhaf_range(p60.B, p60.gamma, p60.reps, b0, b1)
    assert abs(lg.combine(res, 0) - _val(direct)) <= 1e-14 * abs(_val(direct))
