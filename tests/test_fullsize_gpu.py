"""Full-size parity on sampled outputs: the 60-photon collision-free loop hafnian (working dimension
61, degree 30, 2^29 sieve terms) is far beyond the oracle, but any range of its sieve terms is
not. Partial sums of the GPU over term ranges (lhaf_range, the same launch path as a full call)
are compared with the oracle's per-term function (Eq. ET_poly with X replaced by X_delta', App.
B.4) summed over the same digit vectors, which this test decodes from the term numbers itself."""
import math

import numpy as np
import pytest

from oracle import lhaf_oracle as lo
from paper_2108_01622_gb300 import workloads as wl
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu


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


def test_60_photon_sieve_ranges_match_oracle_terms(ctx, lg):
    p = wl.large_lhaf_60(seed=5)
    T, nd, h, P = lg.plan(p.reps)
    assert (T, nd, h, P) == (2 ** 29, 61, 30, 30)
    # one photon per mode: the greedy pairs are consecutive occupied modes in ascending order, all
    # eta = 1; the halved digit is pair 0's (fixed at k = 0, weight x2), so term t has
    # k_q = bit q-1 of t for q = 1..29
    occ = [int(m) for m in np.nonzero(p.reps)[0]]
    pairs, leftover = lo.matched_reps(list(p.reps))
    assert leftover is None and [(a, b) for a, b, _ in pairs] == list(zip(occ[0::2], occ[1::2]))
    C, v, etas, hh = lo.reduced_slot_problem(p.B, p.gamma, p.reps)
    assert hh == h and etas == [1] * 30
    for t0 in (0, 123456789, T - 64):
        ts = np.arange(t0, t0 + 64, dtype=np.int64)
        ks = np.zeros((64, 30), dtype=np.int64)
        for q in range(1, 30):
            ks[:, q] = (ts >> (q - 1)) & 1
        deltas = (1 - 2 * ks).astype(float)
        weights = 2.0 * (-1.0) ** ks.sum(axis=1)
        f = lo.et_poly_coefficient(lo._g_coefficients(C, v, lo._pairing_matrices(deltas), h), h)
        terms = weights * f
        ref = complex(math.fsum(terms.real), math.fsum(terms.imag))
        scale = float(np.sum(np.abs(terms)))
        part = ctx.lhaf_range(p.B, p.gamma, p.reps, int(t0), int(t0) + 64)
        got = complex(part[0] + part[1], part[2] + part[3])
        assert abs(got - ref) <= 1e-12 * scale, (t0, got, ref, scale)
