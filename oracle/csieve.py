"""Test infrastructure only: ctypes access to the plain C restatement of the repeated-pair sieve
(``lhaf_sieve.c``; App. B.2, B.4 Eq. fdsieve, per-term Eq. ET_poly through a Householder
Hessenberg form, La Budde's recurrence and Newton's identities, or repeated products). It is the
timed CPU baseline (OpenMP over terms) and is pinned against the numpy oracle, brute force and
closed forms in the CPU tests. The slot problem (greedy pairs, reduced matrix, degree) comes from
``lhaf_oracle.reduced_slot_problem``.

Built with gcc (OpenMP when available) into ``oracle/liblhaf_sieve_oracle.so`` on first use."""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

from . import lhaf_oracle as lo

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lhaf_sieve.c")
LIB = os.path.join(HERE, "liblhaf_sieve_oracle.so")
_LIB = None


def build() -> str:
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", LIB, SRC, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP runtime: one thread
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("gcc failed for the C oracle:\n" + r.stderr)
    return LIB


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            build()
        lib = ctypes.CDLL(LIB)
        lib.oracle_sieve_sum.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        lib.oracle_sieve_sum.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def sieve_sum(B, gamma, reps, start: int = 0, stop=None, hess: bool = True, threads: int = 0):
    """Unscaled sum of the weighted sieve terms numbered [start, stop) (every digit vector, in
    itertools.product order as ``lhaf_oracle.repeated_sieve_terms``): (complex, threads used)."""
    C, v, etas, h = lo.reduced_slot_problem(B, gamma, reps)
    H = len(etas)
    total = math.prod(e + 1 for e in etas)
    stop = total if stop is None else min(int(stop), total)
    Cr = np.ascontiguousarray(C, dtype=np.complex128)
    vr = np.ascontiguousarray(v, dtype=np.complex128)
    er = np.ascontiguousarray(np.asarray(etas, dtype=np.int32))
    out = np.zeros(4, np.float64)
    used = _lib().oracle_sieve_sum(H, Cr.ctypes.data, vr.ctypes.data, er.ctypes.data, int(h), int(start), int(stop),
                                   1 if hess else 0, int(threads), out.ctypes.data)
    if used < 0:
        raise ValueError("problem outside the C oracle's sizes (at most 32 pairs)")
    return complex(out[0] + out[1], out[2] + out[3]), used


def lhaf(B, gamma, reps, hess: bool = True, threads: int = 0) -> complex:
    """lhaf(B_n) = 2^-h x (sum over every digit vector) (App. B.4 Eq. fdsieve, no halving)."""
    N = int(sum(int(r) for r in reps))
    if N == 0:
        return 1.0 + 0j
    s, _ = sieve_sum(B, gamma, reps, hess=hess, threads=threads)
    return s / 2.0 ** ((N + 1) // 2)
