"""Several loop-weight vectors on one sieve (App. A.2 threshold sub-detectors, App. B.5: only the
diagonal changes) through the C ABI: every vector's value against the oracle's sieve for that
vector and against one lhaf call, with odd patterns (pad index), even repeats (delta' = 0 columns),
zero loops, many vectors, the degree limit and bad arguments."""
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


@pytest.mark.parametrize("reps", [
    (1, 1, 1, 1, 1, 1),
    (1, 1, 1, 1, 1),        # odd: the pad slot's loop weight 1
    (2, 1, 0, 3),
    (2, 2, 2, 2),           # even repeats: middle digits with delta' = 0
    (4, 0, 1, 3, 2, 1),
    (3, 3, 1, 2, 2, 1, 1),
])
def test_multi_gamma_matches_oracle(ctx, reps):
    rng = np.random.default_rng(sum(reps) + len(reps))
    M = len(reps)
    p = wl.small_problem(seed=len(reps) + 3, M=M, reps=reps, loops=True)
    G = wl.complex_normal(rng, (5, M))
    G[2] = 0.0  # no loops for one vector
    out = ctx.lhaf_multi_gamma(p.B, G, list(reps))
    for g in range(5):
        ref = lo.lhaf_repeated(p.B, G[g], np.array(reps))
        if abs(ref) < 1e-13:
            assert abs(out[g]) < 1e-12, (reps, g, out[g], ref)
        else:
            assert rel(out[g], ref) < TOL, (reps, g, out[g], ref)


def test_multi_gamma_many_vectors_collision_pattern(ctx, lg):
    # a 40-photon collision pattern (degree 20) with 32 loop vectors, against one call per vector
    p = wl.collision_lhaf_40(seed=2)
    rng = np.random.default_rng(3)
    G = wl.complex_normal(rng, (32, len(p.reps)))
    out, st = ctx.lhaf_multi_gamma(p.B, G, p.reps, stats=True)
    for g in (0, 7, 31):
        assert rel(out[g], ctx.lhaf(p.B, G[g], p.reps)) < TOL
    assert st["terms"] > 0 and st["launches"] >= 4


def test_multi_gamma_single_vector_and_no_repeat(ctx, lg):
    p = wl.small_problem(seed=9, M=5, reps=(2, 1, 1, 2, 1), loops=True)
    reps = [2, 1, 1, 2, 1]
    out = ctx.lhaf_multi_gamma(p.B, p.gamma[None, :], reps)
    assert rel(out[0], lo.lhaf_repeated(p.B, p.gamma, np.array(reps))) < TOL
    out2 = ctx.lhaf_multi_gamma(p.B, p.gamma[None, :], reps, flags=lg.NO_REPEAT_SPEEDUP)
    assert rel(out2[0], out[0]) < TOL


def test_multi_gamma_limits(ctx, lg):
    p = wl.small_problem(seed=1, M=3, reps=(1, 1, 1), loops=True)
    with pytest.raises(lg.LhafError) as e:
        ctx.lhaf_multi_gamma(p.B, np.zeros((0, 3), complex), [1, 1, 1])
    assert e.value.status == 1
    with pytest.raises(lg.LhafError) as e:
        ctx.lhaf_multi_gamma(p.B, p.gamma[None, :], [20, 20, 10])  # degree 25 > 24
    assert e.value.status == 2
    out = ctx.lhaf_multi_gamma(p.B, np.ones((3, 3), complex), [0, 0, 0])
    assert np.all(out == 1.0)


def test_multi_gamma_vector_count_limit(ctx, lg):
    p = wl.small_problem(seed=6, M=4, reps=(1, 1, 0, 1), loops=True)
    G = wl.complex_normal(np.random.default_rng(6), (256, 4))
    out = ctx.lhaf_multi_gamma(p.B, G, [1, 1, 0, 1])
    for g in (0, 255):
        assert rel(out[g], lo.lhaf_repeated(p.B, G[g], np.array([1, 1, 0, 1]))) < TOL
    with pytest.raises(lg.LhafError) as e:
        ctx.lhaf_multi_gamma(p.B, np.ones((257, 4), complex), [1, 1, 0, 1])
    assert e.value.status == 1


@pytest.mark.parametrize("n_gamma", [4, 16, 24])
def test_multi_gamma_both_paths_on_even_repeats(ctx, lg, n_gamma):
    # a pattern with zero-digit groups: fewer than 16 vectors run as a batch of single loop
    # hafnians, 16 and more share each term's reduction; both against the oracle
    reps = (2, 2, 2, 2, 1, 1)
    p = wl.small_problem(seed=13, M=len(reps), reps=reps, loops=True)
    G = wl.complex_normal(np.random.default_rng(n_gamma), (n_gamma, len(reps)))
    out = ctx.lhaf_multi_gamma(p.B, G, list(reps))
    for g in (0, n_gamma // 2, n_gamma - 1):
        assert rel(out[g], lo.lhaf_repeated(p.B, G[g], np.array(reps))) < TOL
