"""Gaussian state -> GBS kernel -> pattern probability (arXiv:2108.01622, App. A).
TEST INFRASTRUCTURE ONLY.

Complex covariance in the basis a = (a_1..a_M, a_1^dag..a_M^dag):
  sigma_ij = 1/2 <a_i a_j^dag + a_j^dag a_i> - alpha_i alpha_j^*          (App. A)
  sigma_Q = sigma + I/2,  O = I - sigma_Q^-1,  A = X O,  gamma = alpha^dag sigma_Q^-1
  P(n) = exp(-1/2 alpha^dag sigma_Q^-1 alpha) / (sqrt(det sigma_Q) prod n_i!) lhaf(A_n)
                                                                    (Eq. mixed_prob)
For a pure state A = diag(B, B^*) and lhaf(A_n) = |lhaf(B_n)|^2 (Eq. Adef).
"""
from __future__ import annotations

import math

import numpy as np

from .lhaf_oracle import expand_pattern, lhaf_fds_dense, lhaf_repeated


def pure_state_sigma(U, r):
    """sigma = 1/2 S S^dag for squeezed vacuum (a -> a cosh r - a^dag sinh r per mode) followed
    by the interferometer a -> U a. S = [[U, 0], [0, U^*]] [[ch, -sh], [-sh, ch]]."""
    U = np.asarray(U, dtype=complex)
    r = np.asarray(r, dtype=float)
    M = len(r)
    ch = np.diag(np.cosh(r))
    sh = np.diag(np.sinh(r))
    Ssq = np.block([[ch, -sh], [-sh, ch]]).astype(complex)
    Su = np.block([[U, np.zeros((M, M))], [np.zeros((M, M)), U.conj()]])
    S = Su @ Ssq
    return 0.5 * S @ S.conj().T


def gbs_kernel(sigma, alpha):
    """(A, gamma, P0) from the complex covariance and the mean vector alpha_full = (alpha,
    alpha^*) (App. A definitions)."""
    sigma = np.asarray(sigma, dtype=complex)
    n2 = sigma.shape[0]
    M = n2 // 2
    alpha = np.asarray(alpha, dtype=complex)
    af = np.concatenate([alpha, alpha.conj()])
    sQ = sigma + 0.5 * np.eye(n2)
    sQinv = np.linalg.inv(sQ)
    O = np.eye(n2) - sQinv
    X = np.block([[np.zeros((M, M)), np.eye(M)], [np.eye(M), np.zeros((M, M))]])
    A = X @ O
    gamma = af.conj() @ sQinv
    P0 = np.exp(-0.5 * (af.conj() @ sQinv @ af)) / np.sqrt(np.linalg.det(sQ))
    return A, gamma, P0


def pattern_prob_mixed(sigma, alpha, n):
    """Eq. mixed_prob with the 2N x 2N matrix A_n: repeat indices i and i+M n_i times, diagonal
    <- gamma_n. Uses the explicit finite difference sieve; intended for N <= 8."""
    A, gamma, P0 = gbs_kernel(sigma, alpha)
    n = [int(x) for x in n]
    reps2 = n + n
    An = expand_pattern(A, gamma, reps2)
    lh = lhaf_fds_dense(An) if An.shape[0] else 1.0
    return (P0 * lh).real / math.prod(math.factorial(k) for k in n)


def pure_kernel_B(U, r, alpha):
    """B (M x M), gamma_B (M,), P0 for the pure state (U, r, alpha): the first diagonal block of
    A and the first M loop weights (Eq. Adef)."""
    sigma = pure_state_sigma(U, r)
    A, gamma, P0 = gbs_kernel(sigma, alpha)
    M = len(r)
    return A[:M, :M], gamma[:M], P0


def pattern_prob_pure(U, r, alpha, n):
    """P(n) = P0 |lhaf(B_n)|^2 / prod n_i!  for the pure state (Eq. mixed_prob with Eq. Adef)."""
    B, gB, P0 = pure_kernel_B(U, r, alpha)
    lh = lhaf_repeated(B, gB, n)
    return float((P0 * abs(lh) ** 2).real / math.prod(math.factorial(int(k)) for k in n)), lh
