"""GBS pattern probabilities through the C ABI (App. A, Eq. mixed_prob) against the oracle's
independent numpy implementation and textbook closed forms."""
import itertools
import math

import numpy as np
import pytest

from oracle import gbs_oracle as go
from paper_2108_01622_gb300 import workloads as wl
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lg = ensure_built()
    c = lg.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("r", [0.3, 1.1])
def test_single_mode_squeezed_vacuum(ctx, r):
    for k in range(0, 9):
        p, _ = ctx.gbs_pattern_prob(np.eye(1), [r], None, [k])
        if k % 2:
            assert abs(p) < 1e-15
        else:
            m = k // 2
            ref = math.factorial(2 * m) / (2**m * math.factorial(m)) ** 2 * math.tanh(r) ** k / math.cosh(r)
            assert p == pytest.approx(ref, rel=1e-12)


def test_coherent_state_is_poisson(ctx):
    a = 0.7 + 0.5j
    for k in range(0, 7):
        p, _ = ctx.gbs_pattern_prob(np.eye(1), [0.0], [a], [k])
        assert p == pytest.approx(math.exp(-abs(a) ** 2) * abs(a) ** (2 * k) / math.factorial(k), rel=1e-12)


def test_random_states_against_oracle(ctx):
    rng = np.random.default_rng(8)
    for M in (2, 4, 6):
        U = wl.haar_unitary(rng, M)
        r = rng.uniform(0.2, 0.9, size=M)
        alpha = wl.complex_normal(rng, M, 0.3)
        for _ in range(4):
            n = rng.integers(0, 3, size=M)
            p, lh = ctx.gbs_pattern_prob(U, r, alpha, n)
            pr, lhr = go.pattern_prob_pure(U, r, alpha, n)
            assert p == pytest.approx(pr, rel=1e-10, abs=1e-300)
            assert abs(lh - lhr) <= 1e-10 * abs(lhr)


def test_normalisation_two_modes(ctx):
    rng = np.random.default_rng(9)
    U = wl.haar_unitary(rng, 2)
    r = [0.35, 0.2]
    alpha = [0.2 - 0.1j, 0.15j]
    total = sum(ctx.gbs_pattern_prob(U, r, alpha, n)[0] for n in itertools.product(range(10), repeat=2))
    assert total == pytest.approx(1.0, abs=1e-4)
