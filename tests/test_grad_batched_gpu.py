"""Batched gradients (lhaf_grad_batched, through the C ABI): every item against the single-outcome
adjoint and the minor identity from the oracle (App. B definition: the derivative of a matching
sum is the matching sum of the minor), per-item statuses, the 32-photon outcome shape of the
differentiated workload, and the batched torch.autograd log-probability against the per-outcome
one."""
import numpy as np
import pytest

from oracle import lhaf_oracle as lo
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


def _batch(seed, M, count, n_photons, cap):
    rng = np.random.default_rng(seed)
    reps = np.stack([wl.pattern_multinomial(rng, M, n_photons, cap) for _ in range(count)]).astype(np.int32)
    return reps


def test_batched_matches_single_and_oracle_minors(ctx):
    p = wl.small_problem(seed=5, M=6, reps=(1,) * 6)
    reps = np.array([[2, 1, 0, 3, 0, 1], [1, 1, 1, 1, 1, 1], [0, 0, 0, 0, 0, 0], [3, 0, 2, 0, 1, 1],
                     [1, 2, 1, 0, 0, 1]], np.int32)
    rng = np.random.default_rng(3)
    gam = wl.complex_normal(rng, (len(reps), 6))
    vals, dB, dg, st = ctx.lhaf_grad_batched(p.B, gam, reps)
    assert list(st) == [0] * len(reps)
    for i, r in enumerate(reps):
        v1, dB1, dg1 = ctx.lhaf_grad(p.B, gam[i], r)
        assert abs(vals[i] - v1) <= 1e-13 * max(abs(v1), 1.0)
        assert np.abs(dB[i] - dB1).max() <= 1e-13 * max(np.abs(dB1).max(), 1.0)
        assert np.abs(dg[i] - dg1).max() <= 1e-13 * max(np.abs(dg1).max(), 1.0)
        dBr, dgr = lo.lhaf_grad_minor(p.B, gam[i], r)
        scale = max(np.abs(dBr).max(), np.abs(dgr).max(), 1e-300)
        assert np.abs(dB[i] - dBr).max() <= 1e-9 * scale and np.abs(dg[i] - dgr).max() <= 1e-9 * scale
    assert vals[2] == 1.0 and not dB[2].any()


def test_batched_item_status_and_loops_from_diagonal(ctx):
    p = wl.small_problem(seed=8, M=4, reps=(1,) * 4)
    reps = np.array([[1, 1, 2, 0], [1, -1, 0, 0], [2, 2, 0, 1]], np.int32)
    vals, dB, dg, st = ctx.lhaf_grad_batched(p.B, None, reps)
    assert list(st) == [0, 1, 0] and dg is None
    assert vals[1] == 0 and not dB[1].any()
    for i in (0, 2):
        v1, dB1, _ = ctx.lhaf_grad(p.B, None, reps[i])
        assert abs(vals[i] - v1) <= 1e-13 * abs(v1)
        assert np.abs(dB[i] - dB1).max() <= 1e-13 * np.abs(dB1).max()


def test_batched_32_photon_outcomes(ctx):
    # the differentiated workload's shape: 32-photon outcomes of a 40-mode state
    b = wl.gradient_batch(seed=4, count=4)
    reps = np.stack(b.reps).astype(np.int32)
    gam = np.stack(b.gammas)
    vals, dB, dg, st = ctx.lhaf_grad_batched(b.B, gam, reps)
    assert list(st) == [0] * 4
    for i in range(4):
        ref = ctx.lhaf(b.B, gam[i], reps[i])
        assert abs(vals[i] - ref) <= 1e-10 * abs(ref)
    # central differences on one loop weight and one coupling of item 1 (h = 1e-6)
    h = 1e-6
    occ = np.nonzero(reps[1])[0]
    m, mp = occ[0], occ[2]
    e = np.zeros(40, complex)
    e[m] = h
    fd = (ctx.lhaf(b.B, gam[1] + e, reps[1]) - ctx.lhaf(b.B, gam[1] - e, reps[1])) / (2 * h)
    assert abs(fd - dg[1][m]) <= 1e-6 * max(abs(dg[1][m]), abs(vals[1]))
    E = np.zeros((40, 40), complex)
    E[m, mp] = E[mp, m] = h
    fd = (ctx.lhaf(b.B + E, gam[1], reps[1]) - ctx.lhaf(b.B - E, gam[1], reps[1])) / (2 * h)
    assert abs(fd - dB[1][m, mp]) <= 1e-6 * max(abs(dB[1][m, mp]), abs(vals[1]))


def test_batched_log_prob_autograd_matches_per_outcome(ctx):
    import torch

    from paper_2108_01622_gb300.autograd import gbs_log_prob_batch_torch, gbs_log_prob_torch

    rng = np.random.default_rng(21)
    M = 6
    U = torch.from_numpy(wl.haar_unitary(rng, M))
    ns = _batch(22, M, 5, 6, 3)
    r = torch.tensor(rng.uniform(0.3, 0.8, M), dtype=torch.float64, requires_grad=True)
    a = torch.tensor(wl.complex_normal(rng, M, 0.2), dtype=torch.complex128, requires_grad=True)
    L = gbs_log_prob_batch_torch(U, r, a, ns, ctx).sum()
    L.backward()
    gr, ga = r.grad.clone(), a.grad.clone()
    r.grad = None
    a.grad = None
    L1 = sum(gbs_log_prob_torch(U, r, a, n, ctx) for n in ns)
    L1.backward()
    assert abs(L.item() - L1.item()) <= 1e-12 * abs(L1.item())
    assert torch.allclose(gr, r.grad, rtol=1e-10, atol=1e-12)
    assert torch.allclose(ga, a.grad, rtol=1e-10, atol=1e-12)
