"""Pins for the CPU oracle: closed forms, brute force, the paper's worked example and identities
of the loop-hafnian definition (arXiv:2108.01622 App. A-B). No GPU."""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import lhaf_oracle as lo
from oracle import gbs_oracle as go

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rsym(rng, n, real=False):
    X = rng.normal(size=(n, n)) + (0 if real else 1j * rng.normal(size=(n, n)))
    return (X + X.T) / 2


def involutions(n):
    # textbook recurrence: the last element is a fixed point, or swapped with one of n-1 others
    a = [1, 1]
    for k in range(2, n + 1):
        a.append(a[-1] + (k - 1) * a[-2])
    return a[n]


def double_factorial_odd(m):  # (2m-1)!!
    return math.prod(range(1, 2 * m, 2)) if m > 0 else 1


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


# --- closed forms of the definition (App. B) ------------------------------------------------


@pytest.mark.parametrize("n", range(0, 11))
def test_all_ones_gives_involutions(n):
    assert lo.lhaf_bruteforce(np.ones((n, n))).real == pytest.approx(involutions(n), rel=1e-14)


@pytest.mark.parametrize("n", range(0, 11))
def test_sieve_and_et_all_ones_give_involutions(n):
    J = np.ones((n, n))
    assert lo.lhaf_fds_dense(J).real == pytest.approx(involutions(n), rel=1e-12)
    if n <= 10:
        assert lo.lhaf_et(J).real == pytest.approx(involutions(n), rel=1e-12)


@pytest.mark.parametrize("n", range(1, 11))
def test_eigenvalue_traces_all_ones_and_bruteforce(n):
    # the eigenvalue route for the power traces (App. B.1): involutions on the all-ones matrix (its
    # X-paired products are rank one, often nilpotent) and the brute-force sum on random matrices
    ones = np.ones(n, dtype=np.int64)
    J = np.ones((n, n))
    assert lo.lhaf_repeated(J, np.ones(n), ones, traces="eigenvalues").real == pytest.approx(involutions(n), rel=1e-9)
    rng = np.random.default_rng(77 + n)
    A = rsym(rng, n)
    got = lo.lhaf_repeated(A, np.diag(A).copy(), ones, traces="eigenvalues")
    assert rel(got, lo.lhaf_bruteforce(A)) < 1e-10
    reps = [int(x) for x in rng.integers(0, 3, size=4)]
    B = rsym(rng, 4)
    g = rsym(rng, 4).diagonal().copy()
    assert rel(lo.lhaf_repeated(B, g, reps, traces="eigenvalues"), lo.lhaf_repeated(B, g, reps)) < 1e-10


@pytest.mark.parametrize("m", range(1, 6))
def test_hafnian_of_J_minus_I_is_double_factorial(m):
    A = np.ones((2 * m, 2 * m)) - np.eye(2 * m)  # no loops: perfect matchings only
    assert lo.lhaf_bruteforce(A).real == pytest.approx(double_factorial_odd(m))
    assert lo.lhaf_fds_dense(A).real == pytest.approx(double_factorial_odd(m), rel=1e-12)


@pytest.mark.parametrize("n", range(1, 6))
def test_bipartite_block_gives_permanent(n):
    rng = np.random.default_rng(100 + n)
    Bm = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    A = np.zeros((2 * n, 2 * n), dtype=complex)
    A[:n, n:] = Bm
    A[n:, :n] = Bm.T
    perm = lo.permanent_bruteforce(Bm)
    assert rel(lo.lhaf_bruteforce(A), perm) < 1e-12
    assert rel(lo.lhaf_fds_dense(A), perm) < 1e-11
    # perm(J_n) = n!
    assert lo.permanent_bruteforce(np.ones((n, n))).real == pytest.approx(math.factorial(n))


@pytest.mark.parametrize("n", [1, 3, 5, 7])
def test_odd_without_loops_is_zero(n):
    rng = np.random.default_rng(n)
    A = rsym(rng, n)
    np.fill_diagonal(A, 0)
    assert abs(lo.lhaf_bruteforce(A)) < 1e-12
    assert abs(lo.lhaf_fds_dense(A)) < 1e-12
    assert abs(lo.lhaf_et(A)) < 1e-12


# --- the formulas against the definition (brute force) ---------------------------------------


@pytest.mark.parametrize("N", range(0, 11))
@pytest.mark.parametrize("kind", ["complex", "real", "nonneg"])
def test_fds_and_et_match_bruteforce(N, kind):
    rng = np.random.default_rng(1000 * N + len(kind))
    if kind == "nonneg":  # IPS-like proposal matrices (App. C): |B|^2 off-diagonal, |alpha|^2 loops
        A = np.abs(rsym(rng, N)) ** 2
    else:
        A = rsym(rng, N, real=(kind == "real"))
    ref = lo.lhaf_bruteforce(A)
    assert rel(lo.lhaf_fds_dense(A), ref) < 1e-11
    assert rel(lo.lhaf_et(A), ref) < 1e-10


def test_mpmath_bruteforce_agrees():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.default_rng(7)
    A = rsym(rng, 10)
    Amp = [[mpmath.mpc(complex(A[i, j])) for j in range(10)] for i in range(10)]
    ref = complex(lo.lhaf_bruteforce(Amp))
    assert rel(lo.lhaf_fds_dense(A), ref) < 1e-12


def test_block_diagonal_product():
    # App. B.4 accuracy construction: lhaf(diag(A1, A2)) = lhaf(A1) lhaf(A2)
    rng = np.random.default_rng(3)
    A1, A2 = rsym(rng, 6), rsym(rng, 4)
    A = np.zeros((10, 10), dtype=complex)
    A[:6, :6] = A1
    A[6:, 6:] = A2
    ref = lo.lhaf_bruteforce(A1) * lo.lhaf_bruteforce(A2)
    assert rel(lo.lhaf_fds_dense(A), ref) < 1e-11
    assert rel(lo.lhaf_bruteforce(A), ref) < 1e-12


# --- repeated pairs (App. B.2-B.4) -------------------------------------------------------------


def test_worked_example_term_count():
    g = json.load(open(os.path.join(GOLDEN, "paper_worked_example.json")))
    pairs, leftover = lo.matched_reps(g["reps"])
    assert leftover is None
    assert len(pairs) == g["pairings"]
    assert sum(1 for p in pairs if p[2] > 1) == g["repeated_pairings"]
    assert lo.repeated_term_count(g["reps"]) == g["terms_repeated_pairs"]
    N = sum(g["reps"])
    assert 2 ** (N // 2) == g["terms_eigenvalue_trace"]
    assert math.prod(r + 1 for r in g["reps"]) == g["terms_repeated_moment"]


def test_greedy_bounds_and_improvement_rule():
    g = json.load(open(os.path.join(GOLDEN, "paper_bounds.json")))
    M, top = g["pattern_space"]["modes"], g["pattern_space"]["max_count"]
    for reps in itertools.product(range(top + 1), repeat=M):
        N = sum(reps)
        pairs, leftover = lo.matched_reps(reps)
        # every photon is used exactly once
        used = [0] * M
        for a, b, eta in pairs:
            used[a] += eta
            used[b] += eta
        if leftover is not None:
            used[leftover] += 1
        assert used == list(reps)
        etas = [p[2] for p in pairs]
        T = math.prod(e + 1 for e in etas)
        lower = math.prod(math.sqrt(n + 1) for n in reps)
        if N % 2 == 0:
            assert lower <= T * (1 + 1e-12)
            assert T <= 2 ** (N // 2)
        if sum(1 for n in reps if n > 1) >= 2 or max(reps) >= 4:
            assert any(e > 1 for e in etas), reps


@pytest.mark.parametrize(
    "reps",
    [(2, 1, 0, 3), (4, 0, 0, 2), (3, 2, 2, 1), (1, 1, 1), (5, 0, 0, 0), (2, 2, 2, 2), (0, 0, 0, 0),
     (1,), (2,), (3, 1), (6, 1, 1), (0, 3, 0, 4)],
)
@pytest.mark.parametrize("loops", [True, False])
def test_repeated_equals_duplicated(reps, loops):
    rng = np.random.default_rng(sum(reps) * 7 + len(reps))
    M = len(reps)
    B = rsym(rng, M)
    gamma = (rng.normal(size=M) + 1j * rng.normal(size=M)) if loops else np.zeros(M, complex)
    An = lo.expand_pattern(B, gamma, reps)
    ref = lo.lhaf_bruteforce(An)
    got = lo.lhaf_repeated(B, gamma, reps)
    if abs(ref) < 1e-12:
        assert abs(got) < 1e-11
    else:
        assert rel(got, ref) < 1e-11
        assert rel(lo.lhaf_fds_dense(An), ref) < 1e-11


def test_diagonal_only_B_closed_form():
    # B_ij = 0 (i != j): lhaf(B_n) factorises over modes; in mode m the n_m photons form k pairs
    # (weight B_mm each) and n_m - 2k loops (weight gamma_m each): C(n,2k) (2k-1)!! ways.
    rng = np.random.default_rng(11)
    reps = (3, 2, 4)
    d = rng.normal(size=3) + 1j * rng.normal(size=3)
    gam = rng.normal(size=3) + 1j * rng.normal(size=3)
    ref = 1.0
    for n, b, c in zip(reps, d, gam):
        ref *= sum(math.comb(n, 2 * k) * double_factorial_odd(k) * b**k * c ** (n - 2 * k)
                   for k in range(n // 2 + 1))
    assert rel(lo.lhaf_repeated(np.diag(d), gam, reps), ref) < 1e-12


# --- gradients: central differences of the oracle itself ----------------------------------


def test_minor_identity_against_central_differences():
    rng = np.random.default_rng(21)
    M = 3
    reps = (2, 1, 2)
    B = rsym(rng, M)
    gamma = rng.normal(size=M) + 1j * rng.normal(size=M)
    dB, dg = lo.lhaf_grad_minor(B, gamma, reps)
    hstep = 1e-6
    for (i, j) in [(0, 0), (0, 1), (1, 2), (2, 2), (1, 1)]:
        E = np.zeros((M, M), complex)
        E[i, j] = E[j, i] = 1.0
        fd = (lo.lhaf_repeated(B + hstep * E, gamma, reps)
              - lo.lhaf_repeated(B - hstep * E, gamma, reps)) / (2 * hstep)
        assert abs(fd - dB[i, j]) < 1e-6 * max(1, abs(dB[i, j])), (i, j)
    for m in range(M):
        e = np.zeros(M, complex)
        e[m] = 1.0
        fd = (lo.lhaf_repeated(B, gamma + hstep * e, reps)
              - lo.lhaf_repeated(B, gamma - hstep * e, reps)) / (2 * hstep)
        assert abs(fd - dg[m]) < 1e-6 * max(1, abs(dg[m]))


# --- GBS probabilities (App. A) ---------------------------------------------------------------


@pytest.mark.parametrize("r", [0.3, 0.9])
def test_single_mode_squeezed_vacuum(r):
    U = np.eye(1)
    for k in range(0, 7):
        p, _ = go.pattern_prob_pure(U, [r], [0.0], [k])
        if k % 2:
            assert abs(p) < 1e-15
        else:
            m = k // 2
            ref = math.factorial(2 * m) / (2**m * math.factorial(m)) ** 2 * math.tanh(r) ** k / math.cosh(r)
            assert p == pytest.approx(ref, rel=1e-12)


def test_coherent_state_is_poisson():
    a = 0.8 - 0.4j
    for k in range(0, 6):
        p, _ = go.pattern_prob_pure(np.eye(1), [0.0], [a], [k])
        ref = math.exp(-abs(a) ** 2) * abs(a) ** (2 * k) / math.factorial(k)
        assert p == pytest.approx(ref, rel=1e-12)


def _haar(rng, M):
    Z = (rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))) / np.sqrt(2)
    Q, R = np.linalg.qr(Z)
    return Q * (np.diag(R) / np.abs(np.diag(R)))


def test_pure_equals_mixed_and_normalisation():
    rng = np.random.default_rng(5)
    M = 2
    U = _haar(rng, M)
    r = [0.4, 0.25]
    alpha = [0.3 + 0.1j, -0.2j]
    sigma = go.pure_state_sigma(U, r)
    total = 0.0
    for n in itertools.product(range(9), repeat=M):
        p, _ = go.pattern_prob_pure(U, r, alpha, n)
        total += p
        if sum(n) <= 3:  # Eq. Adef: lhaf(A_n) = |lhaf(B_n)|^2 through the 2N x 2N mixed form
            assert p == pytest.approx(go.pattern_prob_mixed(sigma, alpha, n), rel=1e-9, abs=1e-15)
    assert total == pytest.approx(1.0, abs=2e-4)
    p0, _ = go.pattern_prob_pure(U, r, alpha, (0, 0))
    assert p0 == pytest.approx(go.gbs_kernel(sigma, alpha)[2].real, rel=1e-12)


@pytest.mark.parametrize("nbar", [0.3, 2.0])
def test_mixed_thermal_mode_is_geometric(nbar):
    # a thermal mode (sigma = (nbar + 1/2) I, App. A's complex covariance) counts k photons with
    # probability nbar^k / (1 + nbar)^(k + 1): Eq. mixed_prob through the 2N x 2N matrix A_n
    sigma = (nbar + 0.5) * np.eye(2, dtype=complex)
    for k in range(6):
        assert go.pattern_prob_mixed(sigma, [0.0], [k]) == pytest.approx(nbar ** k / (1 + nbar) ** (k + 1), rel=1e-12)


def test_mixed_displaced_thermal_is_laguerre():
    # displaced thermal light: P(k) = nbar^k / (1 + nbar)^(k+1) exp(-|a|^2 / (1 + nbar))
    # L_k(-|a|^2 / (nbar (1 + nbar)))  (the photon statistics of a coherent signal in thermal noise)
    special = pytest.importorskip("scipy.special")
    nbar, a = 0.7, 0.5 + 0.6j
    sigma = (nbar + 0.5) * np.eye(2, dtype=complex)
    x = abs(a) ** 2
    for k in range(6):
        ref = nbar ** k / (1 + nbar) ** (k + 1) * math.exp(-x / (1 + nbar)) * special.eval_laguerre(
            k, -x / (nbar * (1 + nbar)))
        assert go.pattern_prob_mixed(sigma, [a], [k]) == pytest.approx(ref, rel=1e-11)


def test_mixed_two_thermal_modes_factorise_and_lossy_state_normalises():
    # independent thermal modes: the joint probability is the product of the geometric laws
    sigma = np.diag([0.9, 1.6, 0.9, 1.6]).astype(complex)
    for n in itertools.product(range(3), repeat=2):
        ref = math.prod(nb ** k / (1 + nb) ** (k + 1) for nb, k in zip((0.4, 1.1), n))
        assert go.pattern_prob_mixed(sigma, [0, 0], n) == pytest.approx(ref, rel=1e-12)
    # a lossy squeezed, displaced two-mode state (uniform loss eta: sigma -> eta sigma + (1-eta)/2)
    rng = np.random.default_rng(11)
    U = _haar(rng, 2)
    eta = 0.5
    sig = eta * go.pure_state_sigma(U, [0.3, 0.2]) + 0.5 * (1 - eta) * np.eye(4)
    alpha = np.sqrt(eta) * np.array([0.2 + 0.1j, -0.15j])
    total = sum(go.pattern_prob_mixed(sig, alpha, n) for n in itertools.product(range(8), repeat=2))
    assert total == pytest.approx(1.0, abs=1e-5)


# --- planted mistakes: each must be caught by a pin above ---------------------------------


def _pins_pass():
    try:
        test_fds_and_et_match_bruteforce(6, "complex")
        test_repeated_equals_duplicated((2, 1, 0, 3), True)
        test_repeated_equals_duplicated((4, 0, 0, 2), False)
        test_sieve_and_et_all_ones_give_involutions(5)
        return True
    except AssertionError:
        return False


def test_pins_pass_unmutated():
    assert _pins_pass()


def _mutated_g(trace_div=2, loop_shift=0, loop_uses_X=True, loop_half=True):
    """Eq. ET_poly coefficients with one plausible slip planted (for the mutation tests)."""
    def g(C, v, Xs, h):
        T, n, _ = Xs.shape
        out = np.zeros((T, h), dtype=complex)
        CX = np.matmul(C[None], Xs)
        P = np.broadcast_to(np.eye(n, dtype=complex), (T, n, n)).copy()
        left = np.matmul(v[None, None, :], Xs)[:, 0, :] if loop_uses_X else np.broadcast_to(v, (T, n))
        for k in range(1, h + 1):
            Pl = P if loop_shift == 0 else np.matmul(P, CX)
            loop = np.einsum("ti,tij,j->t", left, Pl, v)
            P = np.matmul(P, CX)
            out[:, k - 1] = np.einsum("tii->t", P) / (trace_div * k) + loop * (0.5 if loop_half else 1.0)
        return out
    return g


@pytest.mark.parametrize("mutation", ["drop_loop", "trace_over_k", "loop_no_half", "loop_power_plus_one",
                                      "loop_without_X", "zero_slot_diag", "no_binomial",
                                      "degree_pairs", "et_printed_sign"])
def test_planted_mistakes_are_caught(mutation, monkeypatch):
    orig_g = lo._g_coefficients
    orig_red = lo.reduced_slot_problem
    if mutation == "drop_loop":
        monkeypatch.setattr(lo, "_g_coefficients", lambda C, v, Xs, h: orig_g(C, 0 * v, Xs, h))
    elif mutation == "trace_over_k":
        monkeypatch.setattr(lo, "_g_coefficients", _mutated_g(trace_div=1))
    elif mutation == "loop_no_half":
        monkeypatch.setattr(lo, "_g_coefficients", _mutated_g(loop_half=False))
    elif mutation == "loop_power_plus_one":
        monkeypatch.setattr(lo, "_g_coefficients", _mutated_g(loop_shift=1))
    elif mutation == "loop_without_X":
        monkeypatch.setattr(lo, "_g_coefficients", _mutated_g(loop_uses_X=False))
    elif mutation == "zero_slot_diag":
        def red2(B, gamma, reps):
            C, v, etas, h = orig_red(B, gamma, reps)
            C = C.copy()
            np.fill_diagonal(C, 0)
            return C, v, etas, h
        monkeypatch.setattr(lo, "reduced_slot_problem", red2)
    elif mutation == "no_binomial":
        monkeypatch.setattr(lo.math, "comb", lambda n, k: 1)
    elif mutation == "degree_pairs":
        def red2(B, gamma, reps):
            C, v, etas, h = orig_red(B, gamma, reps)
            return C, v, etas, len(etas)
        monkeypatch.setattr(lo, "reduced_slot_problem", red2)
    elif mutation == "et_printed_sign":
        orig_et = lo.lhaf_et

        def et2(A):
            A = np.asarray(A, dtype=complex)
            N = A.shape[0] + (A.shape[0] % 2)
            return orig_et(A) * (-1) ** (N // 2)
        monkeypatch.setattr(lo, "lhaf_et", et2)
    assert not _pins_pass(), mutation


def _mixed_pins_pass():
    try:
        test_mixed_thermal_mode_is_geometric(0.3)
        test_mixed_displaced_thermal_is_laguerre()
        test_mixed_two_thermal_modes_factorise_and_lossy_state_normalises()
        return True
    except AssertionError:
        return False


def test_mixed_pins_pass_unmutated():
    assert _mixed_pins_pass()


@pytest.mark.parametrize("mutation", ["no_half", "no_X", "gamma_no_conj", "P0_no_sqrt"])
def test_mixed_planted_mistakes_are_caught(mutation, monkeypatch):
    def kernel(sigma, alpha):
        sigma = np.asarray(sigma, dtype=complex)
        n2 = sigma.shape[0]
        M = n2 // 2
        alpha = np.asarray(alpha, dtype=complex)
        af = np.concatenate([alpha, alpha.conj()])
        sQ = sigma + (0.0 if mutation == "no_half" else 0.5) * np.eye(n2)
        sQinv = np.linalg.inv(sQ)
        O = np.eye(n2) - sQinv
        X = np.block([[np.zeros((M, M)), np.eye(M)], [np.eye(M), np.zeros((M, M))]])
        A = O if mutation == "no_X" else X @ O
        gamma = (af if mutation == "gamma_no_conj" else af.conj()) @ sQinv
        det = np.linalg.det(sQ)
        P0 = np.exp(-0.5 * (af.conj() @ sQinv @ af)) / (det if mutation == "P0_no_sqrt" else np.sqrt(det))
        return A, gamma, P0

    monkeypatch.setattr(go, "gbs_kernel", kernel)
    assert not _mixed_pins_pass()


# ---------------------------------------------------------------------------------------------
# The oracle's extended-precision mode (dtype=np.clongdouble), the reference of the most
# ill-conditioned GPU parity cases: exact closed forms, and the definition in 50-digit mpmath.
# ---------------------------------------------------------------------------------------------


def _ld_to_mp(mpmath, x):
    """An extended-precision real as an mpmath number, exactly (two doubles hold its mantissa)."""
    hi = float(x)
    return mpmath.mpf(hi) + mpmath.mpf(float(x - np.longdouble(hi)))


@pytest.mark.parametrize("kind,n", [("involutions", 9), ("involutions", 12), ("double_factorial", 10),
                                    ("double_factorial", 14), ("permanent", 6), ("permanent", 8)])
def test_extended_precision_closed_forms(kind, n):
    # one mode repeated n times with B = gamma = 1 is J_n (involution numbers); with gamma = 0 it
    # is the hafnian of J_n - I ((n - 1)!!); two modes coupled only to each other, n photons
    # each, give the bipartite block [[0, J_n], [J_n, 0]] (perm J_n = n!)
    if kind == "involutions":
        B, g, reps, want = np.ones((1, 1), complex), np.ones(1, complex), (n,), involutions(n)
    elif kind == "double_factorial":
        B, g, reps, want = np.ones((1, 1), complex), np.zeros(1, complex), (n,), math.prod(range(n - 1, 0, -2))
    else:
        B = np.array([[0, 1], [1, 0]], complex)
        g, reps, want = np.zeros(2, complex), (n, n), math.factorial(n)
    got = lo.lhaf_repeated(B, g, reps, dtype=np.clongdouble)
    assert isinstance(got, np.clongdouble)
    assert abs(np.real(got) - np.longdouble(want)) <= 64 * np.finfo(np.longdouble).eps * want
    assert abs(np.imag(got)) <= 64 * np.finfo(np.longdouble).eps * want


def test_extended_precision_beats_complex128_against_mpmath_definition():
    # Repeated patterns with N <= 12 and counts 4..6: the sieve's signed sum cancels (sum |terms|
    # / |lhaf| up to ~70). The definition (brute-force matching sum of the expanded matrix in
    # 50-digit mpmath) is the truth for the same inputs. The extended-precision sieve must land
    # at least 100x closer to it than the complex128 sieve (summed over the instances), and
    # below 1e-17 relative on average; a silent downcast to complex128 anywhere in the dtype
    # plumbing makes the two errors equal and fails both.
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    from paper_2108_01622_gb300 import workloads as wl

    err128, err_ld = [], []
    for reps in [(4, 4, 4), (5, 5, 2), (6, 4, 2), (4, 4, 2, 2), (6, 6)]:
        for seed in range(3):
            p = wl.small_problem(seed=seed, M=len(reps), reps=reps, loops=True)
            A = lo.expand_pattern(p.B, p.gamma, p.reps)
            N = len(A)
            ref = lo.lhaf_bruteforce([[mpmath.mpc(complex(A[i, j])) for j in range(N)] for i in range(N)])
            d = lo.lhaf_repeated(p.B, p.gamma, p.reps)
            e = lo.lhaf_repeated(p.B, p.gamma, p.reps, dtype=np.clongdouble)
            err128.append(float(abs(mpmath.mpc(complex(d)) - ref) / abs(ref)))
            e_mp = mpmath.mpc(_ld_to_mp(mpmath, np.real(e)), _ld_to_mp(mpmath, np.imag(e)))
            err_ld.append(float(abs(e_mp - ref) / abs(ref)))
    assert max(err128) < 1e-13  # the complex128 sieve itself is right
    assert sum(err_ld) / len(err_ld) < 1e-17
    assert sum(err128) >= 100 * sum(err_ld)


@pytest.mark.parametrize("where", ["terms", "coefficients", "series"])
def test_extended_precision_downcast_is_caught(where, monkeypatch):
    # plant a silent complex128 round trip at one step of the extended-precision plumbing
    def down(a):
        return np.asarray(a).astype(np.complex128).astype(np.asarray(a).dtype)

    if where == "terms":
        orig_t = lo.repeated_sieve_terms
        monkeypatch.setattr(lo, "repeated_sieve_terms",
                            lambda *a, **k: [down(np.asarray([t]))[0] for t in orig_t(*a, **k)])
    elif where == "coefficients":
        orig_g = lo._g_coefficients
        monkeypatch.setattr(lo, "_g_coefficients", lambda C, v, Xs, h: down(orig_g(C, v, Xs, h)))
    else:
        orig_e = lo.et_poly_coefficient
        monkeypatch.setattr(lo, "et_poly_coefficient", lambda g, h: down(orig_e(down(g), h)))
    with pytest.raises(AssertionError):
        test_extended_precision_beats_complex128_against_mpmath_definition()
