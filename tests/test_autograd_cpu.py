"""The torch.autograd chain of the GBS log-probability (App. A, Eq. mixed_prob with Eq. Adef) on the
CPU: the library's value and adjoint are replaced by the oracle's (the definition and its minor
identity), so this checks the host side alone: the pure-state kernel in torch, the holomorphic
gradient convention of the autograd Function, and the chain to squeezing and displacement, against
central finite differences and the oracle's probability."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import gbs_oracle as go
from oracle import lhaf_oracle as lo
from paper_2108_01622_gb300 import workloads as wl
from paper_2108_01622_gb300.autograd import gbs_log_prob_torch


class OracleLib:
    """Stands in for the library context: lhaf and lhaf_grad from the oracle."""

    def lhaf(self, B, gamma, reps):
        g = np.diag(B).copy() if gamma is None else gamma
        return lo.lhaf_repeated(B, g, np.asarray(reps))

    def lhaf_grad(self, B, gamma, reps):
        g = np.diag(B).copy() if gamma is None else gamma
        val = lo.lhaf_repeated(B, g, np.asarray(reps))
        dB, dg = lo.lhaf_grad_minor(B, g, reps)
        return val, dB, dg


def test_log_prob_value_and_gradients_match_finite_differences():
    rng = np.random.default_rng(12)
    M = 3
    U = torch.from_numpy(wl.haar_unitary(rng, M))
    r0 = rng.uniform(0.3, 0.8, size=M)
    a0 = wl.complex_normal(rng, M, 0.2)
    n = [1, 2, 1]
    lib = OracleLib()
    r = torch.tensor(r0, dtype=torch.float64, requires_grad=True)
    a = torch.tensor(a0, dtype=torch.complex128, requires_grad=True)
    lp = gbs_log_prob_torch(U, r, a, n, lib)
    ref = go.pattern_prob_pure(U.numpy(), r0, a0, n)[0]
    assert float(lp.detach()) == pytest.approx(math.log(ref), abs=1e-10)
    lp.backward()

    def f(rv, av):
        with torch.no_grad():
            return float(gbs_log_prob_torch(U, torch.tensor(rv), torch.tensor(av), n, lib))

    h = 1e-6
    for i in range(M):
        e = np.zeros(M)
        e[i] = h
        assert float(r.grad[i]) == pytest.approx((f(r0 + e, a0) - f(r0 - e, a0)) / (2 * h), rel=1e-5, abs=1e-7)
        d_re = (f(r0, a0 + e) - f(r0, a0 - e)) / (2 * h)
        d_im = (f(r0, a0 + 1j * e) - f(r0, a0 - 1j * e)) / (2 * h)
        assert float(a.grad[i].real) == pytest.approx(d_re, rel=1e-5, abs=1e-7)
        assert float(a.grad[i].imag) == pytest.approx(d_im, rel=1e-5, abs=1e-7)
