"""GBS pattern probabilities of mixed (lossy) Gaussian states through the C ABI (App. A, Eq.
mixed_prob with the 2M x 2M matrix A): against the oracle's dense finite difference sieve of A_n,
textbook closed forms for thermal and displaced thermal light, the pure-state path, and
normalisation."""
import itertools
import math

import numpy as np
import pytest

from oracle import gbs_oracle as go
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


@pytest.mark.parametrize("nbar", [0.2, 1.7])
def test_thermal_mode_is_geometric(ctx, nbar):
    # a thermal mode has sigma = (nbar + 1/2) I and P(k) = nbar^k / (1 + nbar)^(k + 1)
    sigma = (nbar + 0.5) * np.eye(2, dtype=complex)
    for k in range(9):
        p, _ = ctx.gbs_pattern_prob_mixed(sigma, None, [k])
        assert p == pytest.approx(nbar ** k / (1 + nbar) ** (k + 1), rel=1e-12)


def test_displaced_thermal_mode_is_laguerre(ctx):
    # P(k) = nbar^k / (1 + nbar)^(k+1) exp(-|a|^2 / (1 + nbar)) L_k(-|a|^2 / (nbar (1 + nbar)))
    special = pytest.importorskip("scipy.special")
    nbar, a = 0.6, 0.8 - 0.3j
    sigma = (nbar + 0.5) * np.eye(2, dtype=complex)
    x = abs(a) ** 2
    for k in range(9):
        p, _ = ctx.gbs_pattern_prob_mixed(sigma, [a], [k])
        ref = nbar ** k / (1 + nbar) ** (k + 1) * math.exp(-x / (1 + nbar)) * special.eval_laguerre(
            k, -x / (nbar * (1 + nbar)))
        assert p == pytest.approx(ref, rel=1e-11)


@pytest.mark.parametrize("M", [2, 3, 5])
def test_lossy_states_against_oracle(ctx, M):
    st = wl.lossy_state(seed=10 + M, M=M)
    rng = np.random.default_rng(M)
    for _ in range(4):
        n = rng.integers(0, 3, size=M)
        if n.sum() > 6:
            n[np.argmax(n)] -= n.sum() - 6
        p, _ = ctx.gbs_pattern_prob_mixed(st.sigma, st.alpha, n)
        assert p == pytest.approx(go.pattern_prob_mixed(st.sigma, st.alpha, n), rel=1e-10, abs=1e-300)


def test_pure_state_matches_pure_path(ctx):
    # with no loss A = diag(B, B^*) and lhaf(A_n) = |lhaf(B_n)|^2 (Eq. Adef)
    st = wl.lossy_state(seed=3, M=4, eta=1.0)
    for n in ([1, 1, 0, 2], [2, 0, 1, 1], [0, 0, 0, 0], [3, 1, 0, 0]):
        p, lhA = ctx.gbs_pattern_prob_mixed(st.sigma, st.alpha, n)
        pp, lhB = ctx.gbs_pattern_prob(st.U, st.r, st.alpha, n)
        assert p == pytest.approx(pp, rel=1e-10, abs=1e-300)
        assert abs(lhA - abs(lhB) ** 2) <= 1e-10 * abs(lhB) ** 2


def test_normalisation_two_lossy_modes(ctx):
    st = wl.lossy_state(seed=6, M=2, r_lo=0.2, r_hi=0.4, eta=0.5)
    total = sum(ctx.gbs_pattern_prob_mixed(st.sigma, st.alpha, n)[0]
                for n in itertools.product(range(10), repeat=2))
    assert total == pytest.approx(1.0, abs=1e-5)


def test_collision_pattern_on_larger_lossy_state(ctx):
    # 12 modes, 10 photons with collisions: 2M = 24, working dimension 20; against the oracle's
    # repeated-pair sieve of the same A_n (the dense sieve is too slow here)
    from oracle import lhaf_oracle as lo
    st = wl.lossy_state(seed=21, M=12, r_lo=0.6, r_hi=1.0, eta=0.7)
    n = np.array([2, 0, 1, 0, 3, 0, 1, 1, 0, 2, 0, 0])
    A, gamma, P0 = go.gbs_kernel(st.sigma, st.alpha)
    ref_lh = lo.lhaf_repeated(A, gamma, np.concatenate([n, n]))
    p, lh = ctx.gbs_pattern_prob_mixed(st.sigma, st.alpha, n)
    assert abs(lh - ref_lh) <= 1e-10 * abs(ref_lh)
    ref = (P0 * ref_lh).real / math.prod(math.factorial(int(k)) for k in n)
    assert p == pytest.approx(ref, rel=1e-10)


def test_mixed_rejects_bad_arguments(ctx, lg):
    st = wl.lossy_state(seed=1, M=2)
    with pytest.raises(lg.LhafError) as e:
        ctx.gbs_pattern_prob_mixed(st.sigma, st.alpha, [1, -1])
    assert e.value.status == 1
    bad = st.sigma.copy()
    bad[0, 0] = np.nan
    with pytest.raises(lg.LhafError) as e:
        ctx.gbs_pattern_prob_mixed(bad, st.alpha, [1, 1])
    assert e.value.status == 1


def test_mixed_empty_pattern_is_vacuum_probability(ctx):
    # no photon anywhere: P = P0 = exp(-alpha^dag sigma_Q^-1 alpha / 2) / sqrt(det sigma_Q)
    st = wl.lossy_state(seed=4, M=3)
    p, lh = ctx.gbs_pattern_prob_mixed(st.sigma, st.alpha, [0, 0, 0])
    assert lh == 1.0
    assert p == pytest.approx(go.gbs_kernel(st.sigma, st.alpha)[2].real, rel=1e-12)


def test_mixed_by_inclusion_exclusion_lhafmix(ctx, lg):
    # the paper's lhafmix form (inclusion/exclusion over included copies, LHAF_ET) gives the same
    # probability as the default sieve and the oracle
    st = wl.lossy_state(seed=13, M=4)
    for n in ([1, 2, 0, 1], [2, 0, 2, 1]):
        p_et, _ = ctx.gbs_pattern_prob_mixed(st.sigma, st.alpha, n, flags=lg.ET)
        p_fds, _ = ctx.gbs_pattern_prob_mixed(st.sigma, st.alpha, n)
        ref = go.pattern_prob_mixed(st.sigma, st.alpha, n)
        assert p_et == pytest.approx(ref, rel=1e-10) and p_fds == pytest.approx(ref, rel=1e-10)
