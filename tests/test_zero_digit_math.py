"""The identities behind the zero-digit groups of the repeated-pair sieve, checked in numpy with
the oracle's per-term function (Eq. ET_poly with X replaced by X_delta', App. B.4):

* a pair at its middle digit (delta' = 0) contributes the same term as the slot matrix with its
  two slots deleted;
* summing the groups (middle digits fixed, constant weight factor, other even pairs without their
  middle digit) reproduces the full sieve sum;
* every group is closed under delta' -> -delta' with weight * f unchanged, so it halves exactly.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import lhaf_oracle as lo


def _f(C, v, deltas, h):
    X = lo._pairing_matrices(np.asarray([deltas], dtype=float))
    return lo.et_poly_coefficient(lo._g_coefficients(C, v, X, h), h)[0]


def _weight(etas, ks):
    return math.prod(math.comb(e, k) * (-1) ** k for e, k in zip(etas, ks))


def _problem(seed, etas):
    rng = np.random.default_rng(seed)
    n = 2 * len(etas)
    A = (rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))) / np.sqrt(2 * n)
    C = A + A.T
    v = (rng.normal(size=n) + 1j * rng.normal(size=n)) / 2
    h = (sum(2 * e for e in etas) + 1) // 2
    return C, v, h


def _keep(C, v, H, kept):
    idx = [q for q in kept] + [H + q for q in kept]
    return C[np.ix_(idx, idx)], v[idx]


@pytest.mark.parametrize("seed", range(4))
def test_middle_digit_equals_deleted_slots(seed):
    etas = [2, 1, 4, 2]
    C, v, h = _problem(seed, etas)
    H = len(etas)
    for ks in [(1, 0, 2, 0), (1, 1, 2, 1), (0, 1, 2, 1), (1, 0, 1, 1)]:
        deltas = [e - 2 * k for e, k in zip(etas, ks)]
        kept = [q for q in range(H) if deltas[q] != 0]
        Ck, vk = _keep(C, v, H, kept)
        full = _f(C, v, deltas, h)
        red = _f(Ck, vk, [deltas[q] for q in kept], h)
        assert abs(full - red) <= 1e-12 * max(1.0, abs(full)), (ks, full, red)


def test_group_sum_reproduces_the_sieve_and_each_group_halves():
    etas = [2, 3, 2, 1]
    C, v, h = _problem(11, etas)
    H = len(etas)
    terms = []
    for ks in itertools.product(*[range(e + 1) for e in etas]):
        terms.append(_weight(etas, ks) * _f(C, v, [e - 2 * k for e, k in zip(etas, ks)], h))
    full = complex(math.fsum(t.real for t in terms), math.fsum(t.imag for t in terms))
    even = [q for q in range(H) if etas[q] % 2 == 0]
    group_terms = []
    for z in itertools.product([0, 1], repeat=len(even)):
        Z = {q for q, zi in zip(even, z) if zi}
        kept = [q for q in range(H) if q not in Z]
        wz = math.prod(math.comb(etas[q], etas[q] // 2) * (-1) ** (etas[q] // 2) for q in Z)
        Ck, vk = _keep(C, v, H, kept)
        digit_sets = [[k for k in range(etas[q] + 1) if not (etas[q] % 2 == 0 and 2 * k == etas[q])] for q in kept]
        gsum = []
        for ks in itertools.product(*digit_sets):
            d = [etas[q] - 2 * k for q, k in zip(kept, ks)]
            t = wz * _weight([etas[q] for q in kept], ks) * _f(Ck, vk, d, h)
            gsum.append(t)
            # the mirror term (k -> eta - k on every kept pair) is in the same group, same value
            ks_m = [etas[q] - k for q, k in zip(kept, ks)]
            d_m = [etas[q] - 2 * k for q, k in zip(kept, ks_m)]
            t_m = wz * _weight([etas[q] for q in kept], ks_m) * _f(Ck, vk, d_m, h)
            assert abs(t - t_m) <= 1e-12 * max(1.0, abs(t))
        group_terms.extend(gsum)
    grouped = complex(math.fsum(t.real for t in group_terms), math.fsum(t.imag for t in group_terms))
    assert abs(grouped - full) <= 1e-12 * max(1.0, abs(full))
