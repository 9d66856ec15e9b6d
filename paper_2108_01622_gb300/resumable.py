"""Long loop hafnians in resumable chunks (checkpoint/resume on the host).

The sieve terms of Eq. fdsieve are independent, so a long sum (the 60-photon collision-free loop
hafnian has 2^29 evaluated terms, about a quarter of an hour on one GPU) splits into contiguous
term ranges whose unscaled double-double partials add (App. B.6 splits the same sum over MPI
ranks). ``lhaf_checkpointed`` evaluates the ranges one ``Context.lhaf_range`` call at a time and,
after each, rewrites a small JSON checkpoint with every finished range and its partial (as exact
hexadecimal floats). Started again with the same checkpoint path and the same inputs, it skips the
finished ranges, so an interrupted sum loses at most the range that was running. The final value
is ``combine`` of the partials in range order (double-double sum, then the exact 2^-h).

Within a range the library's launches are bounded (at most a fixed budget of model flops each)
and reduce their partials in term order, so a resumed sum equals the uninterrupted one bit for bit
when the same team size runs the ranges (the same ``Context``, or ``LHAF_TEAM`` set).
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Callable, List, Optional, Tuple

import numpy as np

from . import combine, plan

_VERSION = 1


def fingerprint(B, gamma, reps, flags: int) -> str:
    """SHA-256 of the inputs that define the sum (a checkpoint is only resumed for the same ones)."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(np.asarray(B, dtype=np.complex128)).tobytes())
    if gamma is not None:
        h.update(b"g")
        h.update(np.ascontiguousarray(np.asarray(gamma, dtype=np.complex128)).tobytes())
    h.update(np.ascontiguousarray(np.asarray(reps, dtype=np.int32)).tobytes())
    h.update(str(int(flags)).encode())
    return h.hexdigest()


def chunk_ranges(T: int, chunk_terms: int) -> List[Tuple[int, int]]:
    """[begin, end) ranges of at most chunk_terms terms covering [0, T) in order."""
    if chunk_terms <= 0:
        raise ValueError("chunk_terms must be positive")
    return [(b, min(b + chunk_terms, T)) for b in range(0, T, chunk_terms)]


def _load(path: str, fp: str, T: int, chunk_terms: int) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        ck = json.load(f)
    if ck.get("version") != _VERSION or ck.get("fingerprint") != fp:
        raise ValueError(f"checkpoint {path} belongs to other inputs")
    if ck.get("T") != T or ck.get("chunk_terms") != chunk_terms:
        raise ValueError(f"checkpoint {path} was written with another term count or chunk size")
    return {int(b): (int(e), [float.fromhex(x) for x in part]) for b, e, part in ck["done"]}


def _save(path: str, fp: str, T: int, h: int, chunk_terms: int, done: dict) -> None:
    ck = {"version": _VERSION, "fingerprint": fp, "T": T, "h": h, "chunk_terms": chunk_terms,
          "done": [[b, e, [float(x).hex() for x in part]] for b, (e, part) in sorted(done.items())]}
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(ck, f)
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)  # atomic: a crash leaves the old or the new checkpoint, never half of one


def _has_loops(B, gamma, r) -> bool:
    g = np.diag(B) if gamma is None else np.asarray(gamma)
    return bool(np.any(g[r > 0] != 0))


def range_checkpointed(ctx, B, gamma, reps, term_begin: int, term_end: int, path: str, chunk_terms: int,
                       flags: int = 0, on_chunk: Optional[Callable[[int, int, int], None]] = None) -> np.ndarray:
    """Unscaled double-double partials (n x 4, in term order) of the sieve terms [term_begin,
    term_end) (host inputs), in chunks of ``chunk_terms`` terms, checkpointed to ``path`` after
    every chunk and resumed from it. ``on_chunk(index, begin, end)`` runs after a chunk is saved.
    Raises ValueError if ``path`` holds another problem's checkpoint."""
    B = np.asarray(B, dtype=np.complex128)
    r = np.ones(B.shape[0], np.int32) if reps is None else np.asarray(reps, dtype=np.int32)
    T, _, h, _ = plan(r, flags, _has_loops(B, gamma, r))
    if not 0 <= term_begin <= term_end <= T:
        raise ValueError("term range outside the sieve")
    fp = fingerprint(B, gamma, r, flags) + f":{term_begin}:{term_end}"
    done = _load(path, fp, T, chunk_terms)
    ranges = [(term_begin + b, term_begin + e) for b, e in chunk_ranges(term_end - term_begin, chunk_terms)]
    for i, (b, e) in enumerate(ranges):
        if b in done and done[b][0] == e:
            continue
        part = np.asarray(ctx.lhaf_range(B, gamma, r, b, e, flags), dtype=np.float64)
        done[b] = (e, [float(x) for x in part])
        _save(path, fp, T, h, chunk_terms, done)
        if on_chunk is not None:
            on_chunk(i, b, e)
    return np.array([done[b][1] for b, _ in ranges], dtype=np.float64).reshape(-1, 4)


def lhaf_checkpointed(ctx, B, gamma, reps, path: str, chunk_terms: int, flags: int = 0,
                      on_chunk: Optional[Callable[[int, int, int], None]] = None) -> complex:
    """lhaf(B_n) (host inputs): every sieve term in chunks of ``chunk_terms``, checkpointed to
    ``path`` and resumed from it (``range_checkpointed`` over all terms), then ``combine``."""
    B = np.asarray(B, dtype=np.complex128)
    r = np.ones(B.shape[0], np.int32) if reps is None else np.asarray(reps, dtype=np.int32)
    if int(r.sum()) == 0:
        return 1.0 + 0j
    T, _, h, _ = plan(r, flags, _has_loops(B, gamma, r))
    parts = range_checkpointed(ctx, B, gamma, r, 0, T, path, chunk_terms, flags, on_chunk)
    return combine(parts, h)
