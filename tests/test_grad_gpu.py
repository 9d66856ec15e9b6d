"""Gradients from the adjoint kernel (lhaf_grad, through the C ABI) against the minor identity of
the definition (minors from the oracle), central finite differences (h = 1e-6), and the chain rule
through the GBS log-probability (torch.autograd)."""
import numpy as np
import pytest

from oracle import csieve
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


@pytest.mark.parametrize("reps", [(1, 1, 1, 1), (2, 1, 0, 3), (3, 2, 2, 1), (1, 2, 1), (4, 1, 1, 0, 2), (2, 2, 2)])
@pytest.mark.parametrize("loops", [True, False])
def test_grad_matches_minor_identity(ctx, reps, loops):
    p = wl.small_problem(seed=sum(reps) * 3 + len(reps), M=len(reps), reps=reps, loops=loops)
    val, dB, dg = ctx.lhaf_grad(p.B, p.gamma, p.reps)
    ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
    dB_ref, dg_ref = lo.lhaf_grad_minor(p.B, p.gamma, p.reps)
    scale = max(np.abs(dB_ref).max(), np.abs(dg_ref).max(), 1e-300)
    assert abs(val - ref) <= 1e-10 * abs(ref) + 1e-14
    assert np.abs(dB - dB_ref).max() <= 1e-9 * scale
    assert np.abs(dg - dg_ref).max() <= 1e-9 * scale


def test_grad_gamma_none_folds_loops_into_diagonal(ctx):
    p = wl.small_problem(seed=4, M=3, reps=(2, 1, 2))
    d = np.diag(p.B).copy()
    val, dB, dg = ctx.lhaf_grad(p.B, None, p.reps)
    dB_ref, dg_ref = lo.lhaf_grad_minor(p.B, d, p.reps)
    dB_ref[np.diag_indices(3)] += dg_ref
    assert dg is None
    assert np.abs(dB - dB_ref).max() <= 1e-9 * np.abs(dB_ref).max()


def test_grad_central_differences(ctx):
    p = wl.single_lhaf_24(seed=6, n_photons=14)
    val, dB, dg = ctx.lhaf_grad(p.B, p.gamma, p.reps)
    h = 1e-6
    rng = np.random.default_rng(0)
    occ = np.nonzero(p.reps)[0]
    for _ in range(4):
        i, j = sorted(rng.choice(occ, size=2, replace=False))
        E = np.zeros_like(p.B)
        E[i, j] = E[j, i] = 1.0
        fd = (ctx.lhaf(p.B + h * E, p.gamma, p.reps) - ctx.lhaf(p.B - h * E, p.gamma, p.reps)) / (2 * h)
        assert abs(fd - dB[i, j]) <= 1e-6 * max(abs(dB[i, j]), abs(val))
        m = rng.choice(occ)
        e = np.zeros_like(p.gamma)
        e[m] = 1.0
        fd = (ctx.lhaf(p.B, p.gamma + h * e, p.reps) - ctx.lhaf(p.B, p.gamma - h * e, p.reps)) / (2 * h)
        assert abs(fd - dg[m]) <= 1e-6 * max(abs(dg[m]), abs(val))


def test_grad_32_photon_outcome_against_oracle_minors(ctx):
    # 32 photons over a 40-mode state (collisions allowed): d lhaf / d B_mm' = n_m n_m' lhaf(n - e_m - e_m'),
    # d lhaf / d B_mm = C(n_m, 2) lhaf(n - 2 e_m), d lhaf / d gamma_m = n_m lhaf(n - e_m), every
    # minor and the value from the oracle's repeated-pair sieve
    b = wl.gradient_batch(seed=4, count=2)
    B, g, reps = b.B, b.gammas[0], b.reps[0]
    val, dB, dg = ctx.lhaf_grad(B, g, reps)
    ref_val = lo.lhaf_repeated(B, g, reps)
    assert abs(val - ref_val) <= 1e-10 * abs(ref_val)
    occ = np.nonzero(reps)[0]
    twice = [m for m in occ if reps[m] >= 2]
    for m, mp in [(occ[0], occ[1]), (occ[2], occ[5]), (twice[0], twice[0])]:
        r = reps.copy()
        if m == mp:
            r[m] -= 2
            ref = reps[m] * (reps[m] - 1) / 2 * lo.lhaf_repeated(B, g, r)
        else:
            r[m] -= 1
            r[mp] -= 1
            ref = reps[m] * reps[mp] * lo.lhaf_repeated(B, g, r)
        assert abs(dB[m, mp] - ref) <= 1e-9 * abs(ref), (m, mp)
    for m in (occ[1], twice[1]):
        r = reps.copy()
        r[m] -= 1
        ref = reps[m] * lo.lhaf_repeated(B, g, r)
        assert abs(dg[m] - ref) <= 1e-9 * abs(ref)


@pytest.mark.parametrize("team", [8, 16, 32, 64])
def test_grad_every_team_size(ctx, team, monkeypatch):
    # the adjoint's team forced to 8, 16, 32 and 64 lanes: the same minors as the default choice
    monkeypatch.setenv("LHAF_GRAD_TEAM", str(team))
    for reps, loops in (((3, 2, 2, 1), True), ((2, 1, 2, 2, 1), False)):
        p = wl.small_problem(seed=5 + len(reps), M=len(reps), reps=reps, loops=loops)
        val, dB, dg = ctx.lhaf_grad(p.B, p.gamma, p.reps)
        dB_ref, dg_ref = lo.lhaf_grad_minor(p.B, p.gamma, p.reps)
        scale = max(np.abs(dB_ref).max(), np.abs(dg_ref).max(), abs(val))
        assert np.abs(dB - dB_ref).max() <= 1e-10 * scale
        assert np.abs(dg - dg_ref).max() <= 1e-10 * scale


def test_grad_37_wide_against_c_oracle_minors(ctx):
    # 36 photons on distinct modes of a 40-mode state: working dimension 37 (more rows than the
    # 32 lanes of a team); sampled entries against minors from the C oracle's sieve
    b = wl.gradient_batch(seed=11, count=1, n_photons=2)
    rng = np.random.default_rng(11)
    reps = np.zeros(40, np.int32)
    reps[rng.choice(40, 36, replace=False)] = 1
    B, g = b.B, b.gammas[0]
    val, dB, dg = ctx.lhaf_grad(B, g, reps)
    ref_val = csieve.lhaf(B, g, reps)
    assert abs(val - ref_val) <= 1e-10 * abs(ref_val)
    occ = np.nonzero(reps)[0]
    for m, mp in [(occ[0], occ[1]), (occ[7], occ[30]), (occ[35], occ[2])]:
        r = reps.copy()
        r[m] -= 1
        r[mp] -= 1
        ref = csieve.lhaf(B, g, r)
        assert abs(dB[m, mp] - ref) <= 1e-9 * abs(ref), (m, mp)
    for m in (occ[3], occ[34]):
        r = reps.copy()
        r[m] -= 1
        ref = csieve.lhaf(B, g, r)
        assert abs(dg[m] - ref) <= 1e-9 * abs(ref)


@pytest.mark.parametrize("team", [0, 8, 16, 64])
def test_grad_zero_digit_groups_match_full_matrix(ctx, team, monkeypatch):
    # patterns with even pairs: the adjoint over the zero-digit groups (each on its smaller matrix,
    # gradient sums in the full problem's slots) equals the full-matrix sieve (LHAF_NO_ZERO_SPLIT)
    # and the oracle's minors
    import paper_2108_01622_gb300 as lg

    if team:
        monkeypatch.setenv("LHAF_GRAD_TEAM", str(team))
    for reps, loops in (((2, 2, 1, 3), True), ((4, 2, 2), True), ((2, 2, 2, 2), False), ((2, 1, 2, 1, 2), True)):
        p = wl.small_problem(seed=31 + sum(reps), M=len(reps), reps=reps, loops=loops)
        assert lg.plan_groups(p.reps) >= 2
        v1, dB1, dg1 = ctx.lhaf_grad(p.B, p.gamma, p.reps)
        v2, dB2, dg2 = ctx.lhaf_grad(p.B, p.gamma, p.reps, flags=lg.NO_ZERO_SPLIT)
        dB_ref, dg_ref = lo.lhaf_grad_minor(p.B, p.gamma, p.reps)
        scale = max(np.abs(dB_ref).max(), np.abs(dg_ref).max(), abs(v2))
        assert abs(v1 - v2) <= 1e-12 * scale
        assert np.abs(dB1 - dB2).max() <= 1e-12 * scale and np.abs(dg1 - dg2).max() <= 1e-12 * scale
        assert np.abs(dB1 - dB_ref).max() <= 1e-10 * scale and np.abs(dg1 - dg_ref).max() <= 1e-10 * scale


def test_grad_too_many_groups_runs_the_full_matrix(ctx):
    # 26 modes with two photons each: 13 pairs of count 2, 2^13 - 1 zero-digit groups, above the
    # grouped adjoint's 4096, so the full-matrix adjoint runs (the same bits as LHAF_NO_ZERO_SPLIT);
    # the value against the C oracle
    import paper_2108_01622_gb300 as lg

    b = wl.gradient_batch(seed=12, count=1, n_photons=2)
    reps = np.zeros(40, np.int32)
    reps[np.random.default_rng(12).choice(40, 26, replace=False)] = 2
    assert lg.plan_groups(reps) > 4096
    v1, dB1, dg1 = ctx.lhaf_grad(b.B, b.gammas[0], reps)
    v2, dB2, dg2 = ctx.lhaf_grad(b.B, b.gammas[0], reps, flags=lg.NO_ZERO_SPLIT)
    assert v1 == v2 and np.array_equal(dB1, dB2) and np.array_equal(dg1, dg2)
    ref, cond = csieve.lhaf_with_condition(b.B, b.gammas[0], reps, extended=False)
    assert abs(v1 - ref) <= max(1e-10, 32 * cond * 2.0 ** -52) * abs(ref)


def test_grad_batched_groups_match_single_calls(ctx):
    # a batch mixing grouped and ungrouped outcomes of the 32-photon workload: per item the same
    # bits as the single call (a fixed chunk assignment); against the full-matrix sieve, two FP64
    # evaluations of one cancelling sum, within its condition number (C oracle) x 2^-52 x 32
    import paper_2108_01622_gb300 as lg

    b = wl.gradient_batch(seed=4, count=6)
    R = np.stack(b.reps).astype(np.int32)
    G = np.stack(b.gammas)
    vals, dB, dg, st = ctx.lhaf_grad_batched(b.B, G, R)
    assert np.all(st == 0)
    for i in range(len(R)):
        v, d1, g1 = ctx.lhaf_grad(b.B, G[i], R[i])
        v2, d2, g2 = ctx.lhaf_grad(b.B, G[i], R[i], flags=lg.NO_ZERO_SPLIT)
        s = max(np.abs(d2).max(), np.abs(g2).max())
        assert vals[i] == v and np.array_equal(dB[i], d1) and np.array_equal(dg[i], g1)
        _, cond = csieve.lhaf_with_condition(b.B, G[i], R[i], extended=False)
        tol = max(1e-11, 32 * cond * 2.0 ** -52)
        assert abs(v - v2) <= tol * abs(v2) and np.abs(d1 - d2).max() <= tol * s


def test_log_prob_chain_rule_squeezing_displacement_phases(ctx):
    import torch

    from paper_2108_01622_gb300.autograd import gbs_log_prob_torch

    rng = np.random.default_rng(12)
    M = 5
    U0 = wl.haar_unitary(rng, M)
    n = np.array([2, 1, 0, 1, 2], np.int32)
    r = torch.tensor(rng.uniform(0.3, 0.8, M), dtype=torch.float64, requires_grad=True)
    a = torch.tensor(wl.complex_normal(rng, M, 0.2), dtype=torch.complex128, requires_grad=True)
    phi = torch.tensor(rng.uniform(0, 1, M), dtype=torch.float64, requires_grad=True)

    def logp(r_, a_, phi_):
        U = torch.from_numpy(U0) @ torch.diag(torch.exp(1j * phi_.to(torch.complex128)))
        return gbs_log_prob_torch(U, r_, a_, n, ctx)

    L = logp(r, a, phi)
    L.backward()
    h = 1e-6
    with torch.no_grad():
        for k in range(M):
            e = torch.zeros(M, dtype=torch.float64)
            e[k] = h
            fd = (logp(r + e, a, phi) - logp(r - e, a, phi)) / (2 * h)
            assert abs(fd.item() - r.grad[k].item()) <= 1e-5 * max(1.0, abs(fd.item()))
            fd = (logp(r, a, phi + e) - logp(r, a, phi - e)) / (2 * h)
            assert abs(fd.item() - phi.grad[k].item()) <= 1e-5 * max(1.0, abs(fd.item()))
            # real loss of a complex input: torch's gradient is dL/dRe + i dL/dIm
            fr = (logp(r, a + e.to(torch.complex128), phi) - logp(r, a - e.to(torch.complex128), phi)) / (2 * h)
            fi = (logp(r, a + 1j * e.to(torch.complex128), phi) - logp(r, a - 1j * e.to(torch.complex128), phi)) / (2 * h)
            assert abs(complex(fr.item(), fi.item()) - complex(a.grad[k].item())) <= 1e-5 * max(1.0, abs(fr.item()))
