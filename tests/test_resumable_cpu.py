"""Checkpoint/resume of long sums on CPU: the oracle stands in for the GPU's term-range partials
(App. B.6: the sieve terms are independent, so range partials add). An exception raised on the
host between chunks stands in for an interrupted run; the resumed run must skip the saved chunks
and give the uninterrupted value bit for bit."""
import json

import numpy as np
import pytest

from oracle import lhaf_oracle as lo
from tests.libutil import ensure_built
from tests.test_multirank_cpu import OracleRank


class CountingRank(OracleRank):
    def __init__(self):
        self.calls = []

    def lhaf_range(self, B, gamma, reps, b, e, flags=0):
        self.calls.append((b, e))
        return super().lhaf_range(B, gamma, reps, b, e, flags)


class Interrupted(Exception):
    pass


def _problem():
    rng = np.random.default_rng(41)
    X = rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5))
    g = (rng.normal(size=5) + 1j * rng.normal(size=5)) / 2
    return (X + X.T) / 4, g, np.array([2, 1, 3, 1, 2], np.int32)


def test_checkpointed_equals_oracle_and_resume_is_bit_identical(tmp_path):
    ensure_built()
    from paper_2108_01622_gb300 import resumable

    B, g, reps = _problem()
    ref = lo.lhaf_repeated(B, g, reps)
    whole = resumable.lhaf_checkpointed(CountingRank(), B, g, reps, str(tmp_path / "a.json"), chunk_terms=5)
    assert abs(whole - ref) <= 1e-12 * abs(ref)

    path = str(tmp_path / "b.json")

    def stop_after_two(i, b, e):
        if i == 1:
            raise Interrupted

    first = CountingRank()
    with pytest.raises(Interrupted):
        resumable.lhaf_checkpointed(first, B, g, reps, path, chunk_terms=5, on_chunk=stop_after_two)
    assert len(first.calls) == 2
    saved = json.load(open(path))
    assert [d[0] for d in saved["done"]] == [0, 5]
    second = CountingRank()
    resumed = resumable.lhaf_checkpointed(second, B, g, reps, path, chunk_terms=5)
    assert (0, 5) not in second.calls and (5, 10) not in second.calls
    assert sorted(first.calls + second.calls) == sorted(resumable.chunk_ranges(saved["T"], 5))
    assert resumed == whole  # bit for bit
    # a finished checkpoint resumes without any work
    third = CountingRank()
    assert resumable.lhaf_checkpointed(third, B, g, reps, path, chunk_terms=5) == whole and not third.calls


def test_checkpoint_of_other_inputs_is_refused(tmp_path):
    ensure_built()
    from paper_2108_01622_gb300 import resumable

    B, g, reps = _problem()
    path = str(tmp_path / "c.json")
    resumable.lhaf_checkpointed(CountingRank(), B, g, reps, path, chunk_terms=4)
    with pytest.raises(ValueError):
        resumable.lhaf_checkpointed(CountingRank(), B * 2, g, reps, path, chunk_terms=4)
    with pytest.raises(ValueError):
        resumable.lhaf_checkpointed(CountingRank(), B, g, reps, path, chunk_terms=3)


def test_range_checkpointed_partials_in_term_order(tmp_path):
    ensure_built()
    import paper_2108_01622_gb300 as lg
    from paper_2108_01622_gb300 import resumable

    B, g, reps = _problem()
    T, _, h, _ = lg.plan(reps)
    parts = resumable.range_checkpointed(CountingRank(), B, g, reps, 3, T - 2, str(tmp_path / "d.json"), 4)
    assert parts.shape == (len(resumable.chunk_ranges(T - 5, 4)), 4)
    direct = OracleRank().lhaf_range(B, g, reps, 3, T - 2)
    assert abs(lg.combine(parts, 0) - complex(direct[0] + direct[1], direct[2] + direct[3])) <= 1e-13 * abs(
        complex(direct[0], direct[2]))
    with pytest.raises(ValueError):
        resumable.range_checkpointed(CountingRank(), B, g, reps, 0, T + 1, str(tmp_path / "e.json"), 4)
