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
