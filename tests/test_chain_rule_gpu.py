"""One chain-rule sampler step through the C ABI (App. A.2): the conditional distribution of one
mode's photon number given the photon numbers and coherent amplitudes of the others, against the
oracle's pattern probabilities of the state displaced by -beta (projecting a mode on |beta> counts
no photons after D(-beta)), the drawn outcome against the inverse cumulative distribution, and the
path past the batched mode's degree limit against one loop hafnian per outcome."""
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


def oracle_conditional(U, r, alpha, beta, n, mode, n_cut):
    shift = np.zeros(len(r), complex) if beta is None else np.array(beta, complex).copy()
    shift[mode] = 0.0
    a = (np.zeros(len(r), complex) if alpha is None else np.asarray(alpha, complex)) - shift
    p = []
    for k in range(n_cut + 1):
        pat = np.array(n).copy()
        pat[mode] = k
        p.append(go.pattern_prob_pure(U, r, a, pat)[0])
    p = np.array(p)
    return p / p.sum()


def state(seed, M):
    rng = np.random.default_rng(seed)
    U = wl.haar_unitary(rng, M)
    r = rng.uniform(0.3, 0.9, size=M)
    alpha = wl.complex_normal(rng, M, 0.2)
    return U, r, alpha


def test_last_mode_without_coherent_modes(ctx):
    U, r, alpha = state(1, 4)
    n = [1, 0, 2, 0]
    cond, drawn = ctx.gbs_chain_rule_step(U, r, alpha, None, n, 3, 6)
    assert drawn == -1
    np.testing.assert_allclose(cond, oracle_conditional(U, r, alpha, None, n, 3, 6), rtol=1e-10, atol=1e-15)
    assert cond.sum() == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("mode", [0, 2])
def test_step_with_coherent_modes(ctx, mode):
    U, r, alpha = state(2 + mode, 5)
    rng = np.random.default_rng(40 + mode)
    beta = wl.complex_normal(rng, 5, 0.6)
    n = [0] * 5
    sampled = [1, 3] if mode == 2 else [1]
    for i, v in zip(sampled, (2, 1)):
        n[i] = v
        beta[i] = 0.0
    cond, _ = ctx.gbs_chain_rule_step(U, r, alpha, beta, n, mode, 7)
    np.testing.assert_allclose(cond, oracle_conditional(U, r, alpha, beta, n, mode, 7), rtol=1e-10, atol=1e-15)


def test_uncoupled_modes_ignore_the_other_amplitude(ctx):
    # with no interferometer the modes are independent: the photon number of mode 0 given any
    # coherent amplitude of mode 1 follows the single-mode law of the squeezed, displaced mode 0
    r = [0.6, 0.9]
    alpha = [0.3 - 0.2j, 0.5j]
    for beta1 in (0.0, 1.2 + 0.4j, -0.7j):
        cond, _ = ctx.gbs_chain_rule_step(np.eye(2), r, alpha, [0.0, beta1], [0, 0], 0, 7)
        ref = np.array([go.pattern_prob_pure(np.eye(1), r[:1], alpha[:1], [k])[0] for k in range(8)])
        np.testing.assert_allclose(cond, ref / ref.sum(), rtol=1e-10, atol=1e-15)


def test_draw_is_inverse_cdf(ctx):
    U, r, alpha = state(5, 3)
    n = [1, 0, 0]
    for u in (0.0, 0.05, 0.3, 0.5, 0.77, 0.999999):
        cond, drawn = ctx.gbs_chain_rule_step(U, r, alpha, [0, 0.3 - 0.2j, 0], n, 1, 8, u=u)
        assert drawn == int(np.searchsorted(np.cumsum(cond), u, side="right"))


def test_past_batched_mode_limit_matches_single_calls(ctx):
    # 40 fixed photons and n_cut = 10: degree 25 is above the batched mode's staged limit, so the
    # step runs one batched call over the 11 patterns; compare with one loop hafnian per outcome
    rng = np.random.default_rng(9)
    M = 50
    U = wl.haar_unitary(rng, M)
    r = rng.uniform(0.8, 1.2, size=M)
    alpha = wl.complex_normal(rng, M, 0.1)
    n = wl.pattern_multinomial(rng, M, 40, 3)
    mode = int(np.nonzero(n == 0)[0][0])
    cond, _ = ctx.gbs_chain_rule_step(U, r, alpha, None, n, mode, 10)
    B, gB, _ = go.pure_kernel_B(U, r, alpha)
    lw = []
    for k in range(11):
        pat = n.copy()
        pat[mode] = k
        lh = ctx.lhaf(B, gB, pat)
        lw.append(2 * math.log(abs(lh)) - math.lgamma(k + 1))
    lw = np.array(lw)
    ref = np.exp(lw - lw.max())
    ref /= ref.sum()
    np.testing.assert_allclose(cond, ref, rtol=1e-8, atol=1e-14)


def test_rejects_bad_arguments(ctx, lg):
    U, r, alpha = state(6, 3)
    for n, mode in (([1, 1, 0], 1), ([1, 0, 0], 3), ([-1, 0, 0], 1)):
        with pytest.raises(lg.LhafError) as e:
            ctx.gbs_chain_rule_step(U, r, alpha, None, n, mode, 4)
        assert e.value.status == 1


def test_cutoff_zero_and_vacuum_mode(ctx):
    U, r, alpha = state(7, 3)
    cond, drawn = ctx.gbs_chain_rule_step(U, r, alpha, None, [1, 0, 0], 2, 0, u=0.4)
    assert cond.tolist() == [1.0] and drawn == 0
    # a mode in vacuum (no squeezing, no displacement, no coupling) never holds a photon
    cond, drawn = ctx.gbs_chain_rule_step(np.eye(2), [0.7, 0.0], [0.2, 0.0], None, [2, 0], 1, 5, u=0.99)
    assert cond[0] == pytest.approx(1.0, abs=1e-15) and drawn == 0
