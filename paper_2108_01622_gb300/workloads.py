"""Seeded synthetic GBS-shaped inputs for the loop-hafnian hot path.

This module only draws inputs. It holds none of the loop-hafnian arithmetic and is shared by the
tests (oracle side), the GPU parity tests and bench.py. Recipes follow the paper's workloads (Haar
interferometers with squeezed sources, App. A and Sec. V) with these choices:

* Haar unitary: QR of a complex Ginibre matrix with the diagonal-phase fix (Mezzadri 2007).
* Pure-state kernel input B = U diag(tanh r) U^T (a symmetric M x M matrix).
* Loop weights gamma: complex normal with E|gamma|^2 = 0.5 (real and imaginary parts
  N(0, 1/4)), unless stated otherwise.
* Photon patterns: distinct occupied modes plus multinomial extra photons, rejecting counts above
  a cap.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


def haar_unitary(rng: np.random.Generator, M: int) -> np.ndarray:
    Z = (rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    return Q * (d / np.abs(d))


def kernel_from_squeezing(U: np.ndarray, r: np.ndarray) -> np.ndarray:
    """B = U diag(tanh r) U^T: the synthetic symmetric input matrix of the workloads."""
    return (U * np.tanh(r)[None, :]) @ U.T


def complex_normal(rng: np.random.Generator, size, mean_sq: float = 0.5) -> np.ndarray:
    s = np.sqrt(mean_sq / 2.0)
    return rng.normal(scale=s, size=size) + 1j * rng.normal(scale=s, size=size)


def pattern_distinct_plus_multinomial(rng, M, n_modes, n_total, cap) -> np.ndarray:
    """n_modes distinct occupied modes with one photon each, then n_total - n_modes more photons
    spread by a multinomial over those modes; redraw while any count exceeds cap."""
    modes = rng.choice(M, size=n_modes, replace=False)
    while True:
        extra = rng.multinomial(n_total - n_modes, np.ones(n_modes) / n_modes)
        counts = 1 + extra
        if counts.max() <= cap:
            break
    reps = np.zeros(M, dtype=np.int32)
    reps[modes] = counts
    return reps


def pattern_multinomial(rng, M, n_total, cap) -> np.ndarray:
    """n_total photons by a multinomial over all M modes; redraw while any count exceeds cap."""
    while True:
        reps = rng.multinomial(n_total, np.ones(M) / M)
        if reps.max() <= cap:
            return reps.astype(np.int32)


@dataclass
class Problem:
    """One loop hafnian lhaf(B_n): B (M x M), gamma (M,), reps (M,)."""

    B: np.ndarray
    gamma: np.ndarray
    reps: np.ndarray
    name: str = ""
    U: Optional[np.ndarray] = None
    r: Optional[np.ndarray] = None

    @property
    def N(self) -> int:
        return int(self.reps.sum())


def single_lhaf_24(seed: int = 1, M: int = 24, n_photons: int = 24) -> Problem:
    """24-mode Haar kernel, r ~ U[0.5, 1.5], complex-normal loops, one photon per mode
    (collision-free; 2^11 sieve terms after halving)."""
    rng = np.random.default_rng(seed)
    U = haar_unitary(rng, M)
    r = rng.uniform(0.5, 1.5, size=M)
    B = kernel_from_squeezing(U, r)
    gamma = complex_normal(rng, M)
    reps = np.zeros(M, dtype=np.int32)
    reps[:n_photons] = 1
    return Problem(B, gamma, reps, f"collision-free N={n_photons}, M={M}", U, r)


def collision_lhaf_40(seed: int = 2, M: int = 100, n_modes: int = 22, n_photons: int = 40,
                      cap: int = 4) -> Problem:
    """100-mode Haar kernel, r ~ U[1.0, 1.6], gamma = 0; 40 photons over 22 modes with counts in
    1..4 (photon collisions, repeated-pair sieve)."""
    rng = np.random.default_rng(seed)
    U = haar_unitary(rng, M)
    r = rng.uniform(1.0, 1.6, size=M)
    B = kernel_from_squeezing(U, r)
    gamma = np.zeros(M, dtype=complex)
    reps = pattern_distinct_plus_multinomial(rng, M, n_modes, n_photons, cap)
    return Problem(B, gamma, reps, f"collision N={n_photons} over {n_modes} modes, M={M}", U, r)


def large_lhaf_60(seed: int = 5, M: int = 100, n_photons: int = 60) -> Problem:
    """100-mode Haar kernel, r ~ U[1.2, 1.8], complex-normal loops, 60 distinct modes with one
    photon each (2^29 sieve terms after halving)."""
    rng = np.random.default_rng(seed)
    U = haar_unitary(rng, M)
    r = rng.uniform(1.2, 1.8, size=M)
    B = kernel_from_squeezing(U, r)
    gamma = complex_normal(rng, M)
    modes = rng.choice(M, size=n_photons, replace=False)
    reps = np.zeros(M, dtype=np.int32)
    reps[modes] = 1
    return Problem(B, gamma, reps, f"collision-free N={n_photons}, M={M}", U, r)


def lossy_kernel(rng, M: int, r_lo: float, r_hi: float, eta: float):
    """Thermal loss eta folded into each squeezed mode in closed form: quadrature variances
    v_x = (eta e^{-2r} + 1 - eta)/2, v_p = (eta e^{2r} + 1 - eta)/2 (vacuum = 1/2). The state is a
    pure squeezed state with r' = ln(v_p / v_x) / 4 plus classical noise of per-mode variance
    sqrt(v_x v_p) - 1/2, which is drawn into the loop weights gamma."""
    U = haar_unitary(rng, M)
    r = rng.uniform(r_lo, r_hi, size=M)
    vx = (eta * np.exp(-2 * r) + 1 - eta) / 2
    vp = (eta * np.exp(2 * r) + 1 - eta) / 2
    rp = 0.25 * np.log(vp / vx)
    nu = np.sqrt(vx * vp)
    B = kernel_from_squeezing(U, rp)
    noise_var = np.maximum(nu - 0.5, 1e-3)
    return U, rp, B, noise_var


@dataclass
class BlockPair:
    A1: np.ndarray  # n x n complex symmetric
    A2: np.ndarray  # n x n complex symmetric
    C: np.ndarray   # 2n x 2n: A1 on the even indices, A2 on the odd ones, no coupling between them


def block_diagonal_pair(seed: int, n: int) -> BlockPair:
    """Two random complex symmetric n x n matrices (entries (Z + Z^T)/2, Z complex normal with
    E|Z_ij|^2 = 1) and their direct sum as one 2n x 2n matrix whose indices interleave the blocks
    (index 2i is A1's i, 2i + 1 is A2's i), so that consecutive indices, which a one-photon-per-
    mode pattern pairs, always belong to different blocks (the accuracy experiment of App. B.4,
    Fig. glynn_accuracy: lhaf(C) = lhaf(A1) lhaf(A2), loops on the diagonal)."""
    rng = np.random.default_rng(seed)

    def sym():
        Z = complex_normal(rng, (n, n), 1.0)
        return (Z + Z.T) / 2

    A1, A2 = sym(), sym()
    C = np.zeros((2 * n, 2 * n), dtype=complex)
    C[0::2, 0::2] = A1
    C[1::2, 1::2] = A2
    return BlockPair(A1, A2, C)


@dataclass
class MixedState:
    sigma: np.ndarray  # 2M x 2M complex covariance in the basis (a_1..a_M, a_1^dag..a_M^dag)
    alpha: np.ndarray  # M displacements
    U: np.ndarray
    r: np.ndarray
    eta: float


def lossy_state(seed: int, M: int, r_lo: float = 0.3, r_hi: float = 0.9, eta: float = 0.6,
                alpha_mean_sq: float = 0.1) -> MixedState:
    """A lossy displaced squeezed state as a covariance input: single-mode squeezing r ~ U[r_lo,
    r_hi] (a -> a cosh r - a^dag sinh r), a Haar interferometer, then uniform transmission eta on
    every mode, which maps the covariance to eta sigma + (1 - eta) I / 2 and the mean to
    sqrt(eta) alpha. The displacement is complex normal before the loss."""
    rng = np.random.default_rng(seed)
    U = haar_unitary(rng, M)
    r = rng.uniform(r_lo, r_hi, size=M)
    ch, sh = np.diag(np.cosh(r)), np.diag(np.sinh(r))
    Z = np.zeros((M, M))
    S = np.block([[U, Z], [Z, U.conj()]]) @ np.block([[ch, -sh], [-sh, ch]])
    sigma = 0.5 * S @ S.conj().T
    sigma = eta * sigma + 0.5 * (1.0 - eta) * np.eye(2 * M)
    alpha = np.sqrt(eta) * complex_normal(rng, M, alpha_mean_sq)
    return MixedState(sigma.astype(complex), alpha.astype(complex), U, r, eta)


@dataclass
class Batch:
    B: np.ndarray  # shared M x M kernel
    gammas: List[np.ndarray]
    reps: List[np.ndarray]
    name: str = ""
    problems: List[Problem] = field(default_factory=list)


def chain_rule_batch(seed: int = 3, M: int = 50, count: int = 4096, n_lo: int = 10,
                     n_hi: int = 40, cap: int = 3, eta: float = 0.6) -> Batch:
    """Chain-rule-step batch: `count` loop hafnians of uneven size from one 50-mode lossy GBS
    state (r ~ U[0.8, 1.4], eta = 0.6); N ~ U{10..40}, multinomial pattern, counts <= 3; each item
    draws its own loop weights (the displacement-dependent gamma' of the chain-rule sampler)."""
    rng = np.random.default_rng(seed)
    U, rp, B, noise_var = lossy_kernel(rng, M, 0.8, 1.4, eta)
    gammas, reps = [], []
    for _ in range(count):
        N = int(rng.integers(n_lo, n_hi + 1))
        reps.append(pattern_multinomial(rng, M, N, cap))
        g = U @ complex_normal(rng, M, 1.0) * np.sqrt(noise_var)
        gammas.append(g.astype(complex))
    probs = [Problem(B, g, n, f"chain-rule item {i}") for i, (g, n) in enumerate(zip(gammas, reps))]
    return Batch(B, gammas, reps, f"chain-rule batch x{count}, M={M}", probs)


def gradient_batch(seed: int = 4, M: int = 40, count: int = 256, n_photons: int = 32) -> Batch:
    """256 outcomes of 32 photons (multinomial, collisions allowed) from a 40-mode Haar state with
    r ~ U[0.8, 1.4] and complex-normal loops."""
    rng = np.random.default_rng(seed)
    U = haar_unitary(rng, M)
    r = rng.uniform(0.8, 1.4, size=M)
    B = kernel_from_squeezing(U, r)
    gamma = complex_normal(rng, M)
    reps = [pattern_multinomial(rng, M, n_photons, n_photons) for _ in range(count)]
    probs = [Problem(B, gamma, n, f"grad item {i}", U, r) for i, n in enumerate(reps)]
    return Batch(B, [gamma] * count, reps, f"gradient batch x{count}, M={M}", probs)


def random_symmetric(rng, M: int) -> np.ndarray:
    X = rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))
    return (X + X.T) / 2


def small_problem(seed: int, M: int, reps, loops: bool = True, scale: float = 0.5) -> Problem:
    """Random complex symmetric B (entries ~ scale) with an explicit pattern, for parity sweeps."""
    rng = np.random.default_rng(seed)
    B = random_symmetric(rng, M) * scale
    gamma = complex_normal(rng, M) if loops else np.zeros(M, complex)
    return Problem(B, gamma, np.asarray(reps, dtype=np.int32), f"small seed={seed}")
