"""Pins of the plain C oracle (the timed CPU baseline; App. B.2/B.4 sieve with the power traces
from a Householder Hessenberg form and La Budde's recurrence, or from repeated products): the
definition by brute force, closed forms, and the numpy oracle term range by term range."""
import math

import numpy as np
import pytest

from oracle import csieve
from oracle import lhaf_oracle as lo
from paper_2108_01622_gb300 import workloads as wl


def _involutions(n):
    a = [1, 1]
    for k in range(2, n + 1):
        a.append(a[-1] + (k - 1) * a[-2])
    return a[n]


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


@pytest.mark.parametrize("hess", [True, False])
@pytest.mark.parametrize("reps", [(1, 1, 1, 1, 1, 1), (2, 1, 0, 3), (3, 2, 2, 1), (1, 2, 1, 1, 2), (4, 3), (5,)])
def test_c_oracle_matches_bruteforce(reps, hess):
    p = wl.small_problem(seed=sum(reps) + 7 * len(reps), M=len(reps), reps=reps)
    ref = lo.lhaf_bruteforce(lo.expand_pattern(p.B, p.gamma, p.reps))
    assert rel(csieve.lhaf(p.B, p.gamma, p.reps, hess=hess), ref) < 1e-11


@pytest.mark.parametrize("n", [6, 9, 12])
def test_c_oracle_closed_forms(n):
    one = np.ones((1, 1), complex)
    assert rel(csieve.lhaf(one, np.ones(1, complex), (n,)), _involutions(n)) < 1e-12
    m = n if n % 2 == 0 else n + 1
    assert rel(csieve.lhaf(one, np.zeros(1, complex), (m,)), math.prod(range(m - 1, 0, -2))) < 1e-12
    J = np.array([[0, 1], [1, 0]], complex)
    k = n // 2
    assert rel(csieve.lhaf(J, np.zeros(2, complex), (k, k)), math.factorial(k)) < 1e-12
    assert abs(csieve.lhaf(one, np.zeros(1, complex), (m - 1,))) < 1e-12 * math.prod(range(m - 1, 0, -2))


def test_c_oracle_ranges_match_numpy_oracle_terms():
    p = wl.collision_lhaf_40(seed=9, n_modes=9, n_photons=18)
    total = lo.repeated_term_count(p.reps)
    for a, b in ((0, 17), (17, total // 2), (total // 2, total)):
        ref = math.fsum(t.real for t in lo.repeated_sieve_terms(p.B, p.gamma, p.reps, a, b)) + 1j * math.fsum(
            t.imag for t in lo.repeated_sieve_terms(p.B, p.gamma, p.reps, a, b))
        got, _ = csieve.sieve_sum(p.B, p.gamma, p.reps, a, b)
        scale = sum(abs(t) for t in lo.repeated_sieve_terms(p.B, p.gamma, p.reps, a, b))
        assert abs(got - ref) <= 1e-13 * scale


def test_c_oracle_thread_count_does_not_change_the_value():
    p = wl.single_lhaf_24(seed=4, n_photons=16)
    one, u1 = csieve.sieve_sum(p.B, p.gamma, p.reps, threads=1)
    many, un = csieve.sieve_sum(p.B, p.gamma, p.reps, threads=4)
    assert u1 == 1 and un >= 1
    assert abs(one - many) <= 1e-14 * abs(one)
    assert rel(one / 2.0 ** 8, lo.lhaf_repeated(p.B, p.gamma, p.reps)) < 1e-11


# ---------------------------------------------------------------------------------------------
# The extended-precision build (LHAF_ORACLE_EXTENDED: the same steps in long double complex), the
# reference of the ill-conditioned chain-rule items, and the condition number it reports.
# ---------------------------------------------------------------------------------------------


def _ld_to_mp(mpmath, x):
    hi = float(x)
    return mpmath.mpf(hi) + mpmath.mpf(float(x - np.longdouble(hi)))


@pytest.mark.parametrize("hess", [True, False])
def test_extended_build_closed_forms(hess):
    # involution numbers, (2m-1)!! and perm(J_k) = k! exactly up to a few long double ulps
    eps = float(np.finfo(np.longdouble).eps)
    one = np.ones((1, 1), complex)
    for n in (9, 12):
        got = csieve.lhaf(one, np.ones(1, complex), (n,), hess=hess, extended=True)
        assert isinstance(got, np.clongdouble)
        assert abs(got - np.longdouble(_involutions(n))) <= 256 * eps * _involutions(n)
    got = csieve.lhaf(one, np.zeros(1, complex), (14,), hess=hess, extended=True)
    assert abs(got - np.longdouble(math.prod(range(13, 0, -2)))) <= 256 * eps * math.prod(range(13, 0, -2))
    J = np.array([[0, 1], [1, 0]], complex)
    got = csieve.lhaf(J, np.zeros(2, complex), (7, 7), hess=hess, extended=True)
    assert abs(got - np.longdouble(math.factorial(7))) <= 256 * eps * math.factorial(7)


def _extended_vs_fp64_errors(extended_lib_is_fp64=False):
    # Repeated patterns whose sieve cancels (counts 4..6): errors of the FP64 and the extended builds
    # against the definition (brute-force matching sum of the expanded matrix, 50-digit mpmath)
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    e64, eld = [], []
    for reps in [(4, 4, 4), (5, 5, 2), (6, 4, 2)]:
        for seed in range(2):
            p = wl.small_problem(seed=seed, M=len(reps), reps=reps, loops=True)
            A = lo.expand_pattern(p.B, p.gamma, p.reps)
            N = len(A)
            ref = lo.lhaf_bruteforce([[mpmath.mpc(complex(A[i, j])) for j in range(N)] for i in range(N)])
            d = csieve.lhaf(p.B, p.gamma, p.reps, hess=False)
            e = csieve.lhaf(p.B, p.gamma, p.reps, hess=False, extended=True)
            e64.append(float(abs(mpmath.mpc(complex(d)) - ref) / abs(ref)))
            e_mp = mpmath.mpc(_ld_to_mp(mpmath, np.real(e)), _ld_to_mp(mpmath, np.imag(e)))
            eld.append(float(abs(e_mp - ref) / abs(ref)))
    return e64, eld


def test_extended_build_beats_fp64_against_mpmath_definition():
    # the long double build must land >= 100x closer to the definition than the FP64 build, and
    # below 1e-17 relative on average; a build that silently stays in double fails both
    if np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps:
        pytest.skip("long double is double on this platform")
    e64, eld = _extended_vs_fp64_errors()
    assert max(e64) < 1e-12
    assert sum(eld) / len(eld) < 1e-17
    assert sum(e64) >= 100 * sum(eld)


def test_extended_build_in_double_is_caught(monkeypatch):
    # plant the mistake: the extended entry point silently runs the FP64 library
    if np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps:
        pytest.skip("long double is double on this platform")
    real = csieve._lib
    monkeypatch.setattr(csieve, "_lib", lambda extended=False: real(False))
    with pytest.raises(AssertionError):
        test_extended_build_beats_fp64_against_mpmath_definition()


def test_condition_number_of_the_sieve_sum():
    # cond = sum |weight f| / |sum|: against the numpy oracle's weighted terms (the same digit
    # vectors), >= 1, and the same from the FP64 and extended builds
    for reps, seed in (((4, 4, 2, 2), 2), ((3, 2, 2, 1, 1), 5), ((8,), 1)):
        p = wl.small_problem(seed=seed, M=len(reps), reps=reps, loops=True)
        terms = lo.repeated_sieve_terms(p.B, p.gamma, p.reps)
        want = math.fsum(abs(t) for t in terms) / abs(sum(terms))
        v64, c64 = csieve.lhaf_with_condition(p.B, p.gamma, p.reps, extended=False)
        vld, cld = csieve.lhaf_with_condition(p.B, p.gamma, p.reps, extended=True)
        assert c64 >= 1.0
        assert abs(c64 - want) <= 1e-10 * want and abs(cld - want) <= 1e-10 * want
        ref = lo.lhaf_repeated(p.B, p.gamma, p.reps)
        assert abs(v64 - ref) <= 1e-12 * abs(ref) and abs(complex(vld) - ref) <= 1e-12 * abs(ref)
