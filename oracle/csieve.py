"""Test infrastructure only: ctypes access to the plain C restatement of the repeated-pair sieve
(``lhaf_sieve.c``; App. B.2, B.4 Eq. fdsieve, per-term Eq. ET_poly through a Householder
Hessenberg form, La Budde's recurrence and Newton's identities, or repeated products). It is the
timed CPU baseline (OpenMP over terms) and is pinned against the numpy oracle, brute force and
closed forms in the CPU tests. The slot problem (greedy pairs, reduced matrix, degree) comes from
``lhaf_oracle.reduced_slot_problem``.

Built with gcc (OpenMP when available) into ``oracle/liblhaf_sieve_oracle.so`` on first use, and
with ``LHAF_ORACLE_EXTENDED`` (the same steps in long double complex) into
``oracle/liblhaf_sieve_oracle_ext.so``: the extended-precision reference for ill-conditioned sums."""
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
LIB_EXT = os.path.join(HERE, "liblhaf_sieve_oracle_ext.so")
_LIBS = {}


def _build_one(target: str, defines) -> str:
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared"] + list(defines) + ["-o", target, SRC, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP runtime: one thread
        r = subprocess.run(base, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("gcc failed for the C oracle:\n" + r.stderr)
    return target


def build() -> str:
    _build_one(LIB_EXT, ["-DLHAF_ORACLE_EXTENDED"])
    return _build_one(LIB, [])


def _lib(extended: bool = False):
    path = LIB_EXT if extended else LIB
    if path not in _LIBS:
        if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(SRC):
            _build_one(path, ["-DLHAF_ORACLE_EXTENDED"] if extended else [])
        lib = ctypes.CDLL(path)
        lib.oracle_sieve_sum.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        lib.oracle_sieve_sum.restype = ctypes.c_int
        _LIBS[path] = lib
    return _LIBS[path]


def _sieve(B, gamma, reps, start, stop, hess, threads, extended):
    C, v, etas, h = lo.reduced_slot_problem(B, gamma, reps)
    H = len(etas)
    total = math.prod(e + 1 for e in etas)
    stop = total if stop is None else min(int(stop), total)
    Cr = np.ascontiguousarray(C, dtype=np.complex128)
    vr = np.ascontiguousarray(v, dtype=np.complex128)
    er = np.ascontiguousarray(np.asarray(etas, dtype=np.int32))
    out = np.zeros(5, np.float64)
    used = _lib(extended).oracle_sieve_sum(H, Cr.ctypes.data, vr.ctypes.data, er.ctypes.data, int(h), int(start),
                                           int(stop), 1 if hess else 0, int(threads), out.ctypes.data)
    if used < 0:
        raise ValueError("problem outside the C oracle's sizes (at most 32 pairs)")
    if extended:  # (hi + lo) pairs rebuild the long double sums exactly
        L = np.longdouble
        return np.clongdouble(complex(0.0, 1.0)) * (L(out[2]) + L(out[3])) + (L(out[0]) + L(out[1])), float(out[4]), used
    return complex(out[0] + out[1], out[2] + out[3]), float(out[4]), used


def sieve_sum(B, gamma, reps, start: int = 0, stop=None, hess: bool = True, threads: int = 0,
              extended: bool = False):
    """Unscaled sum of the weighted sieve terms numbered [start, stop) (every digit vector, in
    itertools.product order as ``lhaf_oracle.repeated_sieve_terms``): (complex, threads used).
    extended: the long double build."""
    s, _, used = _sieve(B, gamma, reps, start, stop, hess, threads, extended)
    return s, used


def lhaf_with_condition(B, gamma, reps, extended: bool = True, threads: int = 0):
    """(lhaf, condition number of its sieve sum, sum of |weight * f| / |sum|): an FP64 evaluation of
    the same sum can lose about log10(condition) digits to cancellation (App. B.4's accuracy
    discussion)."""
    N = int(sum(int(r) for r in reps))
    if N == 0:
        return 1.0 + 0j, 1.0
    s, mag, _ = _sieve(B, gamma, reps, 0, None, True, threads, extended)
    return s / 2 ** ((N + 1) // 2), (mag / float(abs(s)) if s != 0 else math.inf)


def lhaf(B, gamma, reps, hess: bool = True, threads: int = 0, extended: bool = False):
    """lhaf(B_n) = 2^-h x (sum over every digit vector) (App. B.4 Eq. fdsieve, no halving); a
    complex, or an np.clongdouble from the extended build."""
    N = int(sum(int(r) for r in reps))
    if N == 0:
        return np.clongdouble(1.0) if extended else 1.0 + 0j
    s, _ = sieve_sum(B, gamma, reps, hess=hess, threads=threads, extended=extended)
    return s / 2 ** ((N + 1) // 2)
