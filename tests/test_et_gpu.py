"""The eigenvalue-trace variant (App. B.1 Eq. ET_loop, repeated pairs as in App. B.2) through the C
ABI: values against the oracle's finite difference sieve and its own inclusion/exclusion sum,
term ranges, FP32 terms, rejected entry points, and the accuracy comparison of App. B.4
(Fig. glynn_accuracy) on block-diagonal matrices."""
import math

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
    (1, 1, 1, 1, 1),            # odd N: the pad pair is one of the pairs
    (2, 1, 0, 3),               # the paper's worked pattern
    (3, 3, 2, 2, 1),
    (2, 2, 2, 2),
    (4, 0, 1, 3, 2, 1),
    (1, 2, 3, 1, 2, 1, 1, 2),
])
@pytest.mark.parametrize("loops", [True, False])
def test_et_matches_oracle(ctx, lg, reps, loops):
    p = wl.small_problem(seed=len(reps) * 31 + sum(reps), M=len(reps), reps=reps, loops=loops)
    got = ctx.lhaf(p.B, p.gamma, list(reps), flags=lg.ET)
    ref = lo.lhaf_repeated(p.B, p.gamma, np.array(reps))
    if ref == 0:
        # odd N without loops: the exact value is 0 and the inclusion/exclusion sum (terms of
        # order one here, entries ~0.5) cancels to rounding level, ~1e-12 at N = 11 with repeats
        assert abs(got) < 1e-10, (reps, loops, got)
    else:
        assert rel(got, ref) < TOL, (reps, loops, got, ref)


def test_et_duplicated_matches_oracle_et(ctx, lg):
    # one photon per index of the explicit duplicated matrix: the paper's plain Eq. ET_loop, against
    # the oracle's literal subset sum on the same matrix
    p = wl.small_problem(seed=12, M=4, reps=(2, 1, 3, 2), loops=True)
    A = lo.expand_pattern(p.B, p.gamma, [2, 1, 3, 2])
    got = ctx.lhaf(A, None, [1] * A.shape[0], flags=lg.ET)
    assert rel(got, lo.lhaf_et(A)) < TOL
    got2 = ctx.lhaf(p.B, p.gamma, [2, 1, 3, 2], flags=lg.ET | lg.NO_REPEAT_SPEEDUP)
    assert rel(got2, lo.lhaf_et(A)) < TOL


def test_et_ranges_add_up(ctx, lg):
    p = wl.small_problem(seed=5, M=7, reps=(2, 1, 1, 3, 1, 2, 1), loops=True)
    reps = [2, 1, 1, 3, 1, 2, 1]
    T, _, h, _ = lg.plan(reps, flags=lg.ET)
    cuts = [0, 1, 7, T // 3, T // 2 + 1, T - 2, T]
    parts = [ctx.lhaf_range(p.B, p.gamma, reps, a, b, flags=lg.ET) for a, b in zip(cuts[:-1], cuts[1:])]
    got = lg.combine(np.array(parts), h)
    assert rel(got, ctx.lhaf(p.B, p.gamma, reps, flags=lg.ET)) < 1e-13
    assert rel(got, lo.lhaf_repeated(p.B, p.gamma, np.array(reps))) < TOL


def test_et_fp32_terms(ctx, lg):
    p = wl.small_problem(seed=8, M=8, reps=(1,) * 8, loops=True)
    got = ctx.lhaf(p.B, p.gamma, [1] * 8, flags=lg.ET | lg.FP32_TERMS)
    assert rel(got, lo.lhaf_repeated(p.B, p.gamma, np.ones(8, dtype=int))) < 1e-3


def test_et_rejected_where_unsupported(ctx, lg):
    p = wl.small_problem(seed=2, M=4, reps=(1, 1, 1, 1), loops=True)
    for call in (lambda: ctx.lhaf_batched(p.B, np.array([p.gamma]), np.array([[1, 1, 1, 1]]), flags=lg.ET),
                 lambda: ctx.lhaf_grad(p.B, p.gamma, [1, 1, 1, 1], flags=lg.ET)):
        with pytest.raises(lg.LhafError) as e:
            call()
        assert e.value.status == 1


def test_block_diagonal_accuracy_fds_vs_et(ctx, lg):
    # App. B.4, Fig. glynn_accuracy: error of lhaf(A1 (+) A2) against lhaf(A1) lhaf(A2), every pair
    # crossing the blocks; the halves come from the oracle. Both variants must be accurate at
    # these sizes; the finite difference sieve's median error must not exceed the
    # eigenvalue-trace one's.
    err_fds, err_et = [], []
    for seed in range(6):
        bp = wl.block_diagonal_pair(seed=100 + seed, n=12)
        ref = lo.lhaf_repeated(bp.A1, np.diag(bp.A1), np.ones(12, dtype=int)) * \
            lo.lhaf_repeated(bp.A2, np.diag(bp.A2), np.ones(12, dtype=int))
        ones = [1] * 24
        err_fds.append(rel(ctx.lhaf(bp.C, None, ones), ref))
        err_et.append(rel(ctx.lhaf(bp.C, None, ones, flags=lg.ET), ref))
    assert max(err_fds) < 1e-11, err_fds
    assert max(err_et) < 1e-6, err_et
    assert np.median(err_fds) <= np.median(err_et), (err_fds, err_et)


def test_et_degenerate_patterns(ctx, lg):
    # empty pattern: 1; one photon: its loop weight (the pad pair); two photons of one mode: B_mm +
    # gamma_m^2 (a pair or two loops)
    p = wl.small_problem(seed=31, M=3, reps=(1, 0, 2), loops=True)
    assert ctx.lhaf(p.B, p.gamma, [0, 0, 0], flags=lg.ET) == 1.0
    assert rel(ctx.lhaf(p.B, p.gamma, [1, 0, 0], flags=lg.ET), p.gamma[0]) < TOL
    assert rel(ctx.lhaf(p.B, p.gamma, [0, 0, 2], flags=lg.ET), p.B[2, 2] + p.gamma[2] ** 2) < TOL
