"""Loop-hafnian oracle (arXiv:2108.01622, App. B). TEST INFRASTRUCTURE ONLY.

Plain CPU restatement of the paper's formulas, written for checking by eye against the paper:

* ``lhaf_bruteforce``  -- the definition: sum over single-pair matchings (App. B, opening
  definition of lhaf).
* ``lhaf_et``          -- eigenvalue-trace inclusion/exclusion (App. B.1, Eq. ET_loop with
  Eq. ET_poly), with the sign reading (-1)^(N/2-|Z|) (the printed (-1)^|Z| is off by the overall
  factor (-1)^(N/2); the brute-force pin shows which is right).
* ``lhaf_fds_dense``   -- finite difference sieve on an explicit matrix (App. B.4, Eq. fdsieve).
* ``matched_reps``     -- greedy choice of repeated pairs (App. B.3, steps 1-5).
* ``lhaf_repeated``    -- finite difference sieve over repeated pairs (App. B.2 and the last
  paragraph of App. B.4): per pair, delta runs from -eta to +eta in steps of 2. Power traces by
  repeated products, or from eigenvalues (App. B.1's route) on request.
* ``lhaf_grad_minor``  -- d lhaf / d B and d lhaf / d gamma from the definition (a derivative of a
  matching sum is the matching sum of a minor).

The per-term function f is Eq. ET_poly written out: traces Tr((C X)^k) and loop terms
v X (C X)^(k-1) v^T by repeated matrix products, then the lambda^(N/2) coefficient of
sum_j (1/j!) (sum_k g_k lambda^k)^j by literal polynomial powers. Sums of terms use
``math.fsum`` (exact rounding of the sum of the fp64 terms).

Precision: complex128 (the paper's precision, App. B.6) unless mpmath numbers are passed to the
brute-force routine.
"""
from __future__ import annotations

import itertools
import math
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

# ---------------------------------------------------------------------------------------------
# Definition
# ---------------------------------------------------------------------------------------------


def lhaf_bruteforce(A):
    """lhaf(A) = sum over single-pair matchings M of [N] of prod_{(i,j) in M} A_ij (App. B).

    A matching groups the indices into singles (loops, weight A_ii) and pairs (weight A_ij).
    Recursion on the lowest remaining index i: it is either a loop, or paired with a j > i.
    Works for any element type with + and * (complex, mpmath.mpc, fractions). Intended for
    N <= 16.
    """
    N = len(A)
    memo = {}

    def rec(mask: int):
        if mask == 0:
            return 1
        if mask in memo:
            return memo[mask]
        i = (mask & -mask).bit_length() - 1
        rest = mask & ~(1 << i)
        total = A[i][i] * rec(rest)
        others = rest
        while others:
            j = (others & -others).bit_length() - 1
            others &= others - 1
            total = total + A[i][j] * rec(rest & ~(1 << j))
        memo[mask] = total
        return total

    return rec((1 << N) - 1)


def expand_pattern(B, gamma, reps):
    """A_n of App. A (Eq. mixed_prob and the chain-rule variant): repeat row/column i of B
    reps[i] times, then put the repeated entries of gamma on the diagonal."""
    B = np.asarray(B, dtype=complex)
    gamma = np.asarray(gamma, dtype=complex)
    idx = [i for i, r in enumerate(reps) for _ in range(int(r))]
    A = B[np.ix_(idx, idx)].copy()
    if len(idx):
        A[np.arange(len(idx)), np.arange(len(idx))] = gamma[idx]
    return A


# ---------------------------------------------------------------------------------------------
# Eq. ET_poly: the per-term function f
# ---------------------------------------------------------------------------------------------


def et_poly_coefficient(g: np.ndarray, h: int) -> np.ndarray:
    """[lambda^h] of sum_{j=1}^{h} (1/j!) (sum_{k=1}^{h} g_k lambda^k)^j  (Eq. ET_poly).

    g has shape (T, h): g[:, k-1] = g_k for a batch of T terms. Returns shape (T,).
    Polynomial powers are formed literally, truncated at degree h.
    """
    T = g.shape[0]
    dt = g.dtype
    if h == 0:
        return np.ones(T, dtype=dt)
    base = np.zeros((T, h + 1), dtype=dt)
    base[:, 1:] = g[:, :h]
    power = np.zeros((T, h + 1), dtype=dt)
    power[:, 0] = 1.0
    total = np.zeros(T, dtype=dt)
    for j in range(1, h + 1):
        new = np.zeros_like(power)
        for d in range(h + 1):  # truncated product power * base
            new[:, d] = np.sum(power[:, : d + 1] * base[:, d::-1], axis=1)
        power = new
        total = total + power[:, h] / dt.type(math.factorial(j))
    return total


def _g_coefficients(C: np.ndarray, v: np.ndarray, Xs: np.ndarray, h: int) -> np.ndarray:
    """g_k = Tr((C X)^k)/(2k) + v X (C X)^(k-1) v^T / 2, k = 1..h (Eq. ET_poly), for a batch of
    pairing matrices Xs (T, n, n). Powers by repeated matrix products."""
    T, n, _ = Xs.shape
    dt = np.result_type(C.dtype, Xs.dtype)
    g = np.zeros((T, h), dtype=dt)
    if n == 0:
        return g
    CX = np.matmul(C[None, :, :], Xs)  # (T, n, n)
    P = np.broadcast_to(np.eye(n, dtype=dt), (T, n, n)).copy()  # (C X)^(k-1)
    vX = np.matmul(v[None, None, :], Xs)[:, 0, :]  # (T, n)
    for k in range(1, h + 1):
        loop = np.einsum("ti,tij,j->t", vX, P, v)
        P = np.matmul(P, CX)  # now (C X)^k
        tr = np.einsum("tii->t", P)
        g[:, k - 1] = tr / dt.type(2 * k) + loop / dt.type(2)
    return g


def _g_coefficients_eig(C: np.ndarray, v: np.ndarray, Xs: np.ndarray, h: int) -> np.ndarray:
    """The same g_k with the traces taken from eigenvalues, the route App. B.1 names:
    Tr((C X)^k) = sum_i lambda_i^k over the eigenvalues of C X (valid for any matrix, defective or
    not); the loop terms v X (C X)^(k-1) v^T by repeated matrix-vector products."""
    T, n, _ = Xs.shape
    g = np.zeros((T, h), dtype=np.complex128)
    if n == 0:
        return g
    CX = np.matmul(C[None, :, :], Xs)
    lam = np.linalg.eigvals(CX)  # (T, n)
    vX = np.matmul(v[None, None, :], Xs)[:, 0, :]  # (T, n)
    w = np.broadcast_to(v, (T, n)).astype(np.complex128)  # (C X)^(k-1) v^T
    power = np.ones_like(lam)
    for k in range(1, h + 1):
        power = power * lam
        tr = power.sum(axis=1)
        loop = np.einsum("ti,ti->t", vX, w)
        w = np.einsum("tij,tj->ti", CX, w)
        g[:, k - 1] = tr / (2 * k) + loop / 2
    return g


def _pairing_matrices(deltas: np.ndarray, dtype=np.complex128) -> np.ndarray:
    """X_delta = [[0, diag(delta)], [diag(delta), 0]] for each row of deltas (App. B.4)."""
    T, H = deltas.shape
    X = np.zeros((T, 2 * H, 2 * H), dtype=dtype)
    ar = np.arange(H)
    X[:, ar, H + ar] = deltas
    X[:, H + ar, ar] = deltas
    return X


def _fsum_complex(values: Iterable[complex]) -> complex:
    vals = list(values)
    return complex(math.fsum(v.real for v in vals), math.fsum(v.imag for v in vals))


def _pad_odd(A: np.ndarray) -> np.ndarray:
    """For odd N: append an index with loop weight 1 and no couplings; it can only be a loop, so
    the loop hafnian is unchanged (the paper states its formulas for even N only)."""
    N = A.shape[0]
    P = np.zeros((N + 1, N + 1), dtype=complex)
    P[:N, :N] = A
    P[N, N] = 1.0
    return P


# ---------------------------------------------------------------------------------------------
# App. B.1: eigenvalue-trace inclusion/exclusion
# ---------------------------------------------------------------------------------------------


def lhaf_et(A) -> complex:
    """Eq. ET_loop: lhaf(A) = sum_{Z subset [N/2]} (-1)^(N/2-|Z|) f(A_Z), where A_Z keeps rows and
    columns i and N/2+i for i in Z, v = diag(A_Z), X pairs i with N/2+i, and f is the
    lambda^(N/2) coefficient of Eq. ET_poly. Intended for N <= 20."""
    A = np.asarray(A, dtype=complex)
    if A.shape[0] % 2:
        A = _pad_odd(A)
    N = A.shape[0]
    h = N // 2
    if h == 0:
        return 1.0 + 0j
    terms = []
    for size in range(0, h + 1):
        for Z in itertools.combinations(range(h), size):
            if size == 0:
                terms.append(0j)  # every trace of the empty matrix is 0, so f = 0
                continue
            keep = list(Z) + [h + i for i in Z]
            C = A[np.ix_(keep, keep)]
            v = np.diag(C).copy()
            X = _pairing_matrices(np.ones((1, size)))
            g = _g_coefficients(C, v, X, h)
            f = et_poly_coefficient(g, h)[0]
            terms.append((-1) ** (h - size) * f)
    return _fsum_complex(terms)


# ---------------------------------------------------------------------------------------------
# App. B.4: finite difference sieve on an explicit matrix
# ---------------------------------------------------------------------------------------------


def lhaf_fds_dense(A, batch: int = 2048) -> complex:
    """Eq. fdsieve: lhaf(A) = 2^(-N/2) sum_{delta in {-1,1}^(N/2)} (prod_k delta_k) f(A X_delta).

    f(A X_delta) is read as Eq. ET_poly with X replaced by X_delta in both the trace and the
    loop terms, and v = diag(A). All 2^(N/2) sign vectors are summed (no halving).
    """
    A = np.asarray(A, dtype=complex)
    if A.shape[0] % 2:
        A = _pad_odd(A)
    N = A.shape[0]
    h = N // 2
    if h == 0:
        return 1.0 + 0j
    v = np.diag(A).copy()
    all_terms = []
    total = 1 << h
    for start in range(0, total, batch):
        idx = np.arange(start, min(total, start + batch))
        bits = (idx[:, None] >> np.arange(h)[None, :]) & 1
        deltas = 1.0 - 2.0 * bits  # bit set -> delta = -1
        g = _g_coefficients(A, v, _pairing_matrices(deltas), h)
        f = et_poly_coefficient(g, h)
        sign = np.prod(deltas, axis=1)
        all_terms.extend((sign * f).tolist())
    return _fsum_complex(all_terms) / 2.0**h


# ---------------------------------------------------------------------------------------------
# App. B.3: greedy matching of repeated pairs
# ---------------------------------------------------------------------------------------------


def matched_reps(reps: Sequence[int]) -> Tuple[List[Tuple[int, int, int]], Optional[int]]:
    """Greedy pairing (App. B.3).

    Returns (pairs, leftover) where pairs is a list of (mode_left, mode_right, eta) and leftover
    is the mode of the one unpaired photon when N is odd (else None).

    Steps: sort counts descending (ties: ascending mode index); if n1 >= 2 n2 make floor(n1/2)
    copies of the pair (m1, m1), else n2 copies of (m1, m2); subtract; drop zero counts; repeat
    while more than one photon remains.
    """
    counts = [(int(c), m) for m, c in enumerate(reps) if int(c) > 0]
    if any(int(c) < 0 for c in reps):
        raise ValueError("negative photon count")
    pairs = []
    while sum(c for c, _ in counts) > 1:
        counts.sort(key=lambda cm: (-cm[0], cm[1]))
        n1, m1 = counts[0]
        n2 = counts[1][0] if len(counts) > 1 else 0
        if n1 >= 2 * n2:
            eta = n1 // 2
            pairs.append((m1, m1, eta))
            counts[0] = (n1 - 2 * eta, m1)
        else:
            m2 = counts[1][1]
            pairs.append((m1, m2, n2))
            counts[0] = (n1 - n2, m1)
            counts[1] = (0, m2)
        counts = [cm for cm in counts if cm[0] > 0]
    leftover = counts[0][1] if counts else None
    return pairs, leftover


def repeated_term_count(reps: Sequence[int]) -> int:
    """prod_i (eta_i + 1) over the greedy pairs (App. B.2): the number of sieve terms before the
    sign-symmetry halving. A leftover photon adds one pair with eta = 1."""
    pairs, leftover = matched_reps(reps)
    t = 1
    for _, _, eta in pairs:
        t *= eta + 1
    if leftover is not None:
        t *= 2
    return t


# ---------------------------------------------------------------------------------------------
# App. B.2 + B.4: finite difference sieve over repeated pairs
# ---------------------------------------------------------------------------------------------

PAD_MODE = -1


def reduced_slot_problem(B, gamma, reps):
    """Reduced 2H x 2H slot matrix for the repeated-pair sieve.

    Slot i (i < H) is the left photon of pair i and slot H+i its right photon (so the fixed
    matching X pairs i with H+i, as in App. B.1). C[s, t] = B[mode(s), mode(t)] for all s, t,
    including s == t: two distinct copies of one slot are two photons of one mode, weight B_mm.
    v[s] = gamma[mode(s)] carries the loops. When N is odd a pad slot (loop weight 1, no
    couplings) is paired with the leftover photon.

    Returns (C, v, etas, h) with h = ceil(N/2).
    """
    B = np.asarray(B, dtype=complex)
    gamma = np.asarray(gamma, dtype=complex)
    pairs, leftover = matched_reps(reps)
    plist = [(a, b, e) for a, b, e in pairs]
    if leftover is not None:
        plist.append((leftover, PAD_MODE, 1))
    H = len(plist)
    modes = [p[0] for p in plist] + [p[1] for p in plist]
    n = 2 * H
    C = np.zeros((n, n), dtype=complex)
    v = np.zeros(n, dtype=complex)
    for s in range(n):
        v[s] = 1.0 if modes[s] == PAD_MODE else gamma[modes[s]]
        for t in range(n):
            if modes[s] != PAD_MODE and modes[t] != PAD_MODE:
                C[s, t] = B[modes[s], modes[t]]
    N = int(sum(int(r) for r in reps))
    h = (N + 1) // 2
    etas = [p[2] for p in plist]
    return C, v, etas, h


def repeated_sieve_terms(B, gamma, reps, start: int = 0, stop: Optional[int] = None,
                         batch: int = 2048, dtype=np.complex128, traces: str = "products") -> list:
    """The signed, weighted sieve terms prod_i C(eta_i,k_i) (-1)^(k_i) f(C X_delta') for the digit
    vectors k number start..stop-1 in itertools.product order (App. B.2, B.4). Used by
    lhaf_repeated (all terms) and by timing on a bounded sample of terms. dtype: complex128 (the
    paper's precision) or np.clongdouble for an extended-precision reference of the same sum."""
    C, v, etas, h = reduced_slot_problem(B, gamma, reps)
    C = C.astype(dtype)
    v = v.astype(dtype)
    total = math.prod(e + 1 for e in etas)
    stop = total if stop is None else min(stop, total)
    digit_ranges = [range(e + 1) for e in etas]
    all_k = np.array(list(itertools.islice(itertools.product(*digit_ranges), start, stop)), dtype=np.int64)
    etas_a = np.array(etas, dtype=np.int64)
    terms: List[complex] = []
    for b0 in range(0, len(all_k), batch):
        ks = all_k[b0 : b0 + batch]
        deltas = (etas_a[None, :] - 2 * ks).astype(float)
        weights = np.array(
            [
                math.prod(math.comb(int(e), int(k)) * (-1) ** int(k) for e, k in zip(etas, row))
                for row in ks
            ],
            dtype=float,
        ).astype(dtype)
        if traces == "eigenvalues":
            g = _g_coefficients_eig(C, v, _pairing_matrices(deltas), h)
        else:
            g = _g_coefficients(C, v, _pairing_matrices(deltas, dtype), h)
        f = et_poly_coefficient(g, h)
        terms.extend(list(weights * f))
    return terms


def lhaf_repeated(B, gamma, reps, batch: int = 2048, dtype=np.complex128, traces: str = "products"):
    """lhaf(A_n) by the finite difference sieve over greedy repeated pairs (App. B.2, B.4).

    For pair i repeated eta_i times, k_i in 0..eta_i copies carry -1, so
    delta'_i = eta_i - 2 k_i with multiplicity C(eta_i, k_i) and sign (-1)^(k_i):
      lhaf = 2^(-h) sum_k prod_i C(eta_i,k_i) (-1)^(k_i) f(C X_delta'),  h = N/2,
    with f the lambda^h coefficient of Eq. ET_poly for the reduced slot matrix. Every digit
    vector is summed (no halving). traces="eigenvalues" takes the power traces from eigenvalues
    (App. B.1) instead of repeated products (complex128 only).
    """
    N = int(sum(int(r) for r in reps))
    if N == 0:
        return 1.0 + 0j
    h = (N + 1) // 2
    terms = repeated_sieve_terms(B, gamma, reps, batch=batch, dtype=dtype, traces=traces)
    if np.dtype(dtype) == np.complex128:
        return _fsum_complex(terms) / 2.0**h
    # extended precision: sum in that precision, smallest magnitudes first
    arr = np.array(terms, dtype=dtype)
    arr = arr[np.argsort(np.abs(arr))]
    return np.sum(arr) / dtype(2) ** h


# ---------------------------------------------------------------------------------------------
# Gradients (from the definition)
# ---------------------------------------------------------------------------------------------


def lhaf_grad_minor(B, gamma, reps, lhaf_fn=None):
    """Derivatives of lhaf(A_n) with respect to the entries of B (as a symmetric variable,
    B_mm' = B_m'm one variable) and gamma, from the definition (App. B): each matching term that
    contains a factor x contributes the matching sum over the remaining indices.

      d lhaf / d B_mm'  = n_m n_m' lhaf(n - e_m - e_m')        (m != m')
      d lhaf / d B_mm   = C(n_m, 2) lhaf(n - 2 e_m)
      d lhaf / d gamma_m = n_m lhaf(n - e_m)

    Returns (dB (M x M, symmetric), dgamma (M,)).
    """
    if lhaf_fn is None:
        lhaf_fn = lhaf_repeated
    B = np.asarray(B, dtype=complex)
    gamma = np.asarray(gamma, dtype=complex)
    reps = [int(r) for r in reps]
    M = len(reps)
    dB = np.zeros((M, M), dtype=complex)
    dg = np.zeros(M, dtype=complex)
    for m in range(M):
        if reps[m] >= 1:
            r = list(reps)
            r[m] -= 1
            dg[m] = reps[m] * lhaf_fn(B, gamma, r)
        for mp in range(m, M):
            if m == mp:
                if reps[m] >= 2:
                    r = list(reps)
                    r[m] -= 2
                    dB[m, m] = math.comb(reps[m], 2) * lhaf_fn(B, gamma, r)
            elif reps[m] >= 1 and reps[mp] >= 1:
                r = list(reps)
                r[m] -= 1
                r[mp] -= 1
                dB[m, mp] = dB[mp, m] = reps[m] * reps[mp] * lhaf_fn(B, gamma, r)
    return dB, dg


# ---------------------------------------------------------------------------------------------
# Helpers used by pins
# ---------------------------------------------------------------------------------------------


def permanent_bruteforce(Bm) -> complex:
    """perm(B) = sum over permutations s of prod_i B[i, s(i)] (textbook definition)."""
    Bm = np.asarray(Bm, dtype=complex)
    n = Bm.shape[0]
    return _fsum_complex(
        math.prod(Bm[i, s[i]] for i in range(n)) for s in itertools.permutations(range(n))
    ) if n else 1.0 + 0j
