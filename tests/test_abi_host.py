"""C-ABI library without a GPU: it loads, exports every function include/lhaf.h declares, and its
host planner (greedy pairing of App. B.3, term counts, limits, errors) agrees with the oracle."""
import ctypes
import itertools
import math

import numpy as np
import pytest

from oracle import lhaf_oracle as lo
from tests.libutil import ensure_built


@pytest.fixture(scope="module")
def lg():
    return ensure_built()


def test_exports_every_declared_function(lg):
    lib = ctypes.CDLL(lg.LIB_PATH)
    names = lg.header_functions()
    assert {"lhaf", "lhaf_range", "lhaf_ctx_create", "lhaf_plan"} <= set(names)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: the header compiles as strict C99 (and as C++), no torch types
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "abi.c"
    src.write_text('#include "include/lhaf.h"\nint main(void) { lhaf_stats s; (void)s; return 0; }\n')
    for lang, std in (("c", "-std=c99"), ("c++", "-std=c++17")):
        r = subprocess.run([gcc, std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-x", lang, "-I", root, "-c",
                            str(src), "-o", str(tmp_path / f"abi_{lang}.o")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    text = open(os.path.join(root, "include", "lhaf.h")).read()
    assert "Tensor" not in text and "at::" not in text and "torch::" not in text


def halved_count(reps, loops):
    """Evaluated terms after the sign-symmetry halving, from the oracle's greedy pairs."""
    pairs, leftover = lo.matched_reps(reps)
    etas = [e for _, _, e in pairs] + ([1] if leftover is not None else [])
    if not etas:
        return 1
    odd = [e for e in etas if e % 2]
    T = math.prod(e + 1 for e in etas)
    if odd:
        return T // 2
    emax = max(etas)
    return (T // (emax + 1)) * (emax // 2 + 1)


def split_count(reps):
    """Evaluated terms of the zero-digit groups: for every subset Z of the even-eta pairs, the pairs
    in Z sit at their middle digit (slots deleted), the other even pairs skip it (eta digits), odd
    pairs take eta + 1 digits; each group is halved once; a group without pairs is dropped."""
    pairs, leftover = lo.matched_reps(reps)
    etas = [e for _, _, e in pairs] + ([1] if leftover is not None else [])
    even = [e for e in etas if e >= 2 and e % 2 == 0]
    odd = [e for e in etas if e % 2]
    if not even:
        return halved_count(reps, True)
    total = 0
    for z in itertools.product([0, 1], repeat=len(even)):
        kept = [e for e, zi in zip(even, z) if not zi]
        if not kept and not odd:
            continue
        total += math.prod(e for e in kept) * math.prod(e + 1 for e in odd) // 2
    return total


@pytest.mark.parametrize("reps", list(itertools.product(range(4), repeat=3)) + [(2, 1, 0, 3), (1,) * 24, (4, 4, 4), (9,)])
def test_plan_matches_oracle_greedy(lg, reps):
    T, nd, h, P = lg.plan(reps, has_loops=True)
    pairs, leftover = lo.matched_reps(reps)
    N = sum(reps)
    if N == 0:
        assert T == 1
        return
    assert P == len(pairs) + (leftover is not None)
    assert h == (N + 1) // 2
    assert nd == 2 * P + 1
    assert T == split_count(reps)
    assert lg.plan(reps, flags=lg.NO_ZERO_SPLIT, has_loops=True)[0] == halved_count(reps, True)
    # without loops the border disappears unless a pad is needed
    T0, nd0, _, _ = lg.plan(reps, has_loops=False)
    assert T0 == T
    assert nd0 == 2 * P + (1 if leftover is not None else 0)


def test_worked_example_halved(lg):
    # App. B.2 example n = (2,1,0,3): 6 terms, 3 after the sign-symmetry halving
    T, nd, h, P = lg.plan([2, 1, 0, 3], has_loops=False)
    assert (T, P, h) == (3, 2, 3)


def test_plan_groups_count(lg):
    # pairs [2, 1] (worked example): one even pair -> 2 groups; no even pair -> no split
    assert lg.plan_groups([2, 1, 0, 3]) == 2
    assert lg.plan_groups([1, 1, 1, 1]) == 0
    assert lg.plan_groups([2, 1, 0, 3], flags=lg.NO_ZERO_SPLIT) == 0
    # (4,): one pair with eta = 2 alone: the group with it at the middle digit is empty (dropped)
    assert lg.plan_groups([4]) == 1 and lg.plan([4])[0] == 1


def test_et_plan_counts(lg):
    # eigenvalue-trace form (App. B.1, B.2): every choice of kept pairs with 1..eta copies each,
    # the empty one excepted; one sieve per number of kept pairs
    for reps in ([1] * 10, [2, 1, 0, 3], [3, 3, 2, 2, 1], [4, 4, 4, 4]):
        T, nd, h, P = lg.plan(reps, flags=lg.ET)
        pairs, left = lo.matched_reps(reps)
        etas = [e for _, _, e in pairs] + ([1] if left is not None else [])
        assert T == math.prod(e + 1 for e in etas) - 1
        assert lg.plan_groups(reps, flags=lg.ET) == P == len(etas)


def test_et_plan_counts_random_patterns(lg):
    # the eigenvalue-trace term count over many random patterns: prod (eta + 1) - 1 over the
    # oracle's greedy pairs (a pad pair for odd N), one sieve per number of kept pairs
    rng = np.random.default_rng(17)
    for _ in range(200):
        M = int(rng.integers(1, 9))
        reps = [int(x) for x in rng.integers(0, 5, size=M)]
        if sum(reps) == 0:
            continue
        pairs, left = lo.matched_reps(reps)
        etas = [e for _, _, e in pairs] + ([1] if left is not None else [])
        T, nd, h, P = lg.plan(reps, flags=lg.ET)
        assert T == math.prod(e + 1 for e in etas) - 1, reps
        assert P == len(etas) and lg.plan_groups(reps, flags=lg.ET) == P


def test_zero_digit_groups_cover_every_digit_vector():
    # every digit vector lies in exactly one group: middle digits of the even pairs pick the group
    for etas in ([2], [2, 2], [4, 1, 2], [3, 2, 2, 1], [6, 4]):
        even = [e for e in etas if e % 2 == 0]
        covered = 0
        for z in itertools.product([0, 1], repeat=len(even)):
            kept = [e for e, zi in zip(even, z) if not zi]
            covered += math.prod(kept) * math.prod(e + 1 for e in etas if e % 2)
        assert covered == math.prod(e + 1 for e in etas)


def test_no_repeat_speedup_gives_duplicated_count(lg):
    T, nd, h, P = lg.plan([2, 1, 0, 3], flags=lg.NO_REPEAT_SPEEDUP, has_loops=False)
    assert T == 2 ** 2 and P == 3


def test_limits_and_errors(lg):
    with pytest.raises(lg.LhafError) as e:
        lg.plan([1] * 70, has_loops=True)  # 35 pairs + border > 64
    assert e.value.status == 2
    with pytest.raises(lg.LhafError) as e:
        lg.plan([1, -1, 2])
    assert e.value.status == 1
    T, nd, h, P = lg.plan([1] * 62, has_loops=True)
    assert nd == 63 and T == 2 ** 30


def test_flop_model_positive_and_cubic(lg):
    f24 = lg.flops_per_term(25, 12, True)
    f48 = lg.flops_per_term(49, 24, True)
    assert f24 > 0 and 6.0 < f48 / f24 < 9.5
    assert lg.flops_per_term(1, 1, False) == 0.0


def test_combine_scales_exactly(lg):
    parts = np.array([[3.0, 1e-20, -1.0, 0.0], [5.0, 0.0, 2.0, -1e-20]])
    assert lg.combine(parts, 3) == complex(1.0, 0.125)


def test_ctx_create_without_gpu_fails_cleanly(lg):
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(lg.LhafError) as e:
        lg.Context(0)
    assert e.value.status == 3


def test_batched_plan_rejects_bad_arguments_without_a_context(lg):
    lib = lg._lib()
    h = ctypes.c_void_p(123)
    B = np.zeros((2, 2), np.complex128)
    R = np.ones((1, 2), np.int32)
    st = lib.lhaf_batched_plan_create(None, 1, 2, B.ctypes.data, None, R.ctypes.data, 0, ctypes.byref(h))
    assert st == 1 and h.value is None
    assert lib.lhaf_batched_plan_create(None, 1, 2, B.ctypes.data, None, R.ctypes.data, 0, None) == 1
    assert lib.lhaf_batched_plan_exec(None, B.ctypes.data, None, B.ctypes.data, None, None) == 1
    lib.lhaf_batched_plan_destroy(None)
