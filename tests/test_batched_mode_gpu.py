"""GPU parity of the batched mode of one chain-rule step (App. A.2, App. B.5): every outcome
n = 0..n_cut of the batched mode against the oracle's own loop hafnian of that pattern (its own
greedy pairing), and against one lhaf call per outcome."""
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


def _check(ctx, B, gamma, reps, mode, n_cut):
    out = ctx.lhaf_batched_mode(B, gamma, reps, mode, n_cut)
    assert out.shape == (n_cut + 1,)
    g = np.diag(B).copy() if gamma is None else gamma
    for n in range(n_cut + 1):
        r = np.array(reps, dtype=np.int64).copy()
        r[mode] = n
        ref = lo.lhaf_repeated(B, g, r)
        if abs(ref) < 1e-12:
            assert abs(out[n]) < 1e-11, (reps, mode, n, out[n], ref)
        else:
            assert rel(out[n], ref) < TOL, (reps, mode, n, out[n], ref)
    return out


@pytest.mark.parametrize("reps,mode,n_cut", [
    ((1, 1, 0, 2), 2, 6),       # N_fixed even, a repeated fixed pair
    ((1, 2, 0, 2), 2, 7),       # N_fixed odd: the odd outcomes pair the leftover with the mode
    ((0, 0, 0, 0), 1, 6),       # nothing fixed: the single-mode loop hafnians
    ((2, 0, 2, 0), 1, 5),       # only even fixed pairs
    ((3, 1, 1, 0, 1), 3, 8),
])
@pytest.mark.parametrize("loops", [True, False])
def test_batched_mode_small_vs_oracle(ctx, reps, mode, n_cut, loops):
    p = wl.small_problem(seed=sum(reps) + 7 * mode + n_cut, M=len(reps), reps=reps, loops=loops)
    _check(ctx, p.B, p.gamma, list(reps), mode, n_cut)


def test_batched_mode_gamma_none_and_n_cut_zero(ctx):
    p = wl.small_problem(seed=3, M=5, reps=(1, 1, 1, 0, 1), loops=True)
    _check(ctx, p.B, None, [1, 1, 1, 0, 1], 3, 4)
    out = ctx.lhaf_batched_mode(p.B, p.gamma, [1, 1, 1, 0, 1], 3, 0)
    assert rel(out[0], lo.lhaf_repeated(p.B, p.gamma, [1, 1, 1, 0, 1])) < TOL


def test_batched_mode_chain_rule_step_matches_single_calls(ctx, lg):
    # a chain-rule step on the lossy 50-mode state: 15 photons fixed, the next mode batched to 8.
    # This item is well conditioned (sum |terms| / |sum| <= 160 over the outcomes), so the two
    # exact sieves (the batched mode pairs the mode with itself, the single call pairs greedily)
    # and the oracle agree to TOL. (On the 31-photon item of the same batch the ratio reaches
    # 5.3e6 and the two sieves differ by up to ~5e-10, within their rounding.)
    b = wl.chain_rule_batch(seed=5, count=8)
    reps = np.array(b.reps[1], dtype=np.int32)
    gamma = np.array(b.gammas[1])
    mode = int(np.nonzero(reps == 0)[0][0])
    n_cut = 8
    out, st = ctx.lhaf_batched_mode(b.B, gamma, reps, mode, n_cut, stats=True)
    for n in range(n_cut + 1):
        r = reps.copy()
        r[mode] = n
        single = ctx.lhaf(b.B, gamma, r)
        ref = lo.lhaf_repeated(b.B, gamma, r)
        assert rel(out[n], ref) < TOL, (n, out[n], ref)
        assert rel(single, ref) < TOL, (n, single, ref)
    assert st["terms"] > 0 and st["launches"] >= 4


def test_batched_mode_rejects_bad_arguments(ctx, lg):
    p = wl.small_problem(seed=4, M=3, reps=(1, 1, 1), loops=True)
    with pytest.raises(lg.LhafError) as e:
        ctx.lhaf_batched_mode(p.B, p.gamma, [1, 1, 1], 1, 3)  # the batched mode must be empty
    assert e.value.status == 1
    with pytest.raises(lg.LhafError) as e:
        ctx.lhaf_batched_mode(p.B, p.gamma, [20, 20, 0], 2, 12)  # degree 26 > 24
    assert e.value.status == 2


@pytest.mark.parametrize("reps,mode", [((2, 0, 2, 0, 1), 1), ((4, 2, 0, 2, 1, 1), 2), ((2, 2, 2, 0), 3)])
def test_batched_mode_zero_digit_groups(ctx, lg, monkeypatch, reps, mode):
    # fixed pairs with even repeats: their middle digits run as zero-digit groups (forced here; by
    # default only for large sieves); the same outcomes with LHAF_NO_ZERO_SPLIT and from the oracle
    monkeypatch.setenv("LHAF_MODE_SPLIT", "1")
    p = wl.small_problem(seed=40 + sum(reps), M=len(reps), reps=reps, loops=True)
    a = ctx.lhaf_batched_mode(p.B, p.gamma, list(reps), mode, 6)
    b = ctx.lhaf_batched_mode(p.B, p.gamma, list(reps), mode, 6, flags=lg.NO_ZERO_SPLIT)
    for n in range(7):
        r = np.array(reps, dtype=np.int64)
        r[mode] = n
        ref = lo.lhaf_repeated(p.B, p.gamma, r)
        assert rel(a[n], ref) < TOL and rel(b[n], ref) < TOL, (n, a[n], b[n], ref)
