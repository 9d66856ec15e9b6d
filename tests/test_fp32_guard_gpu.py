"""The FP32-term variant is offered only where its stated error holds: up to degree 18 (N <= 36
photons) with a bound of 1e-2 relative error against FP64 references from the oracles, and refused
(LHAF_ETOOBIG) above that, in every entry point that takes the flag."""
import numpy as np
import pytest

from oracle import csieve
from oracle import lhaf_oracle as lo
from paper_2108_01622_gb300 import workloads as wl
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu

FP32_BOUND = 1e-2


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


def test_fp32_refused_above_degree_18(ctx, lg):
    p = wl.large_lhaf_60(seed=100, n_photons=38)  # h = 19
    with pytest.raises(lg.LhafError) as e:
        ctx.lhaf(p.B, p.gamma, p.reps, flags=lg.FP32_TERMS)
    assert e.value.status == 2
    with pytest.raises(lg.LhafError) as e:
        ctx.lhaf_range(p.B, p.gamma, p.reps, 0, 64, flags=lg.FP32_TERMS)
    assert e.value.status == 2
    ok = wl.large_lhaf_60(seed=100, n_photons=12)
    reps = np.stack([p.reps, ok.reps])
    gam = np.stack([p.gamma, p.gamma])
    vals, status = ctx.lhaf_batched(p.B, gam, reps, flags=lg.FP32_TERMS)
    assert list(status) == [2, 0]
    ref = lo.lhaf_repeated(p.B, p.gamma, ok.reps)
    assert abs(vals[1] - ref) <= FP32_BOUND * abs(ref)
    # FP64 is not limited
    assert np.isfinite(ctx.lhaf_range(p.B, p.gamma, p.reps, 0, 64)).all()


def test_fp32_error_bound_at_36_photons_gbs_instance(ctx, lg):
    # the 60-photon workload's family at N = 36 (2^17 evaluated terms), reference: the C oracle
    p = wl.large_lhaf_60(seed=101, n_photons=36)
    ref = csieve.lhaf(p.B, p.gamma, p.reps)
    got = ctx.lhaf(p.B, p.gamma, p.reps, flags=lg.FP32_TERMS)
    assert abs(ctx.lhaf(p.B, p.gamma, p.reps) - ref) <= 1e-10 * abs(ref)
    assert abs(got - ref) <= FP32_BOUND * abs(ref)


@pytest.mark.parametrize("seed", [3601, 3602])
def test_fp32_error_bound_at_36_photons_block_diagonal(ctx, lg, seed):
    # App. B.4's construction: lhaf(A1 (+) A2) = lhaf(A1) lhaf(A2), halves by the oracle
    bp = wl.block_diagonal_pair(seed=seed, n=18)
    ones = [1] * 18
    ref = lo.lhaf_repeated(bp.A1, np.diag(bp.A1), ones) * lo.lhaf_repeated(bp.A2, np.diag(bp.A2), ones)
    got = ctx.lhaf(bp.C, None, [1] * 36, flags=lg.FP32_TERMS)
    assert abs(got - ref) <= FP32_BOUND * abs(ref)
