"""The allocation-free entry point lhaf_noalloc, called through the C ABI, against lhaf().

lhaf_noalloc serves callers that cannot call cudaMalloc/cudaFree (another allocator owns the device
memory, or an allocation's implicit synchronisation is not acceptable): its scratch is a fixed
device array inside the library. This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_2108_01622_gb300 import workloads as wl
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lg = ensure_built()
    lib = ctypes.CDLL(lg.LIB_PATH)
    vp = ctypes.c_void_p
    lib.lhaf_noalloc.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp, vp, vp, ctypes.c_uint32, vp]
    lib.lhaf_noalloc.restype = ctypes.c_int
    return torch, lg, lib


def _call(torch, lib, p, flags=0):
    dev = torch.device("cuda", 0)
    B = torch.from_numpy(np.ascontiguousarray(p.B)).to(dev)
    g = torch.from_numpy(np.ascontiguousarray(p.gamma)).to(dev)
    reps = np.ascontiguousarray(p.reps, dtype=np.int32)
    out = torch.full((1,), complex(np.nan, np.nan), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    st = lib.lhaf_noalloc(0, stream, len(reps), B.data_ptr(), g.data_ptr(), reps.ctypes.data, flags,
                          out.data_ptr())
    torch.cuda.synchronize()
    return st, complex(out.cpu()[0])


def test_noalloc_matches_lhaf_on_two_calls_in_a_row(env):
    torch, lg, lib = env
    first = wl.single_lhaf_24(seed=1, n_photons=20)       # working dimension 21 (loop border)
    second = wl.collision_lhaf_40(seed=2, n_modes=10, n_photons=18)  # smaller, no loops
    with lg.Context(0) as ctx:
        for p in (first, second):
            ref = ctx.lhaf(p.B, p.gamma, p.reps)
            st, got = _call(torch, lib, p)
            assert st == 0, lg.STATUS.get(st, st)
            assert abs(got - ref) / abs(ref) < TOL, (got, ref)


def test_noalloc_rejects_too_large(env):
    torch, lg, lib = env
    p = wl.small_problem(3, 70, [1] * 70)  # 35 pairs + loop border > 64
    st, _ = _call(torch, lib, p)
    assert st == 2  # LHAF_ETOOBIG


def test_noalloc_more_terms_than_teams(env):
    # 28 photons, collision-free: 8192 terms for at most 4096 teams, so every team loops over rounds
    torch, lg, lib = env
    p = wl.single_lhaf_24(seed=3, M=28, n_photons=28)
    assert lg.plan(p.reps)[0] == 8192
    with lg.Context(0) as ctx:
        ref = ctx.lhaf(p.B, p.gamma, p.reps)
    for _ in range(2):
        st, got = _call(torch, lib, p)
        assert st == 0 and abs(got - ref) / abs(ref) < TOL, (got, ref)


def test_noalloc_gamma_none_empty_pattern_and_flags(env):
    torch, lg, lib = env
    p = wl.collision_lhaf_40(seed=5, n_modes=8, n_photons=14)
    dev = torch.device("cuda", 0)
    B = torch.from_numpy(np.ascontiguousarray(p.B)).to(dev)
    reps = np.ascontiguousarray(p.reps, dtype=np.int32)
    out = torch.full((1,), complex(np.nan, np.nan), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    with lg.Context(0) as ctx:
        ref = ctx.lhaf(p.B, None, p.reps)  # loops from diag(B)
    st = lib.lhaf_noalloc(0, stream, len(reps), B.data_ptr(), None, reps.ctypes.data, 0, out.data_ptr())
    torch.cuda.synchronize()
    assert st == 0 and abs(complex(out.cpu()[0]) - ref) / abs(ref) < TOL
    # the eigenvalue-trace form is not offered here
    assert lib.lhaf_noalloc(0, stream, len(reps), B.data_ptr(), None, reps.ctypes.data, lg.ET, out.data_ptr()) == 1
    # the empty pattern: lhaf = 1
    zero = np.zeros_like(reps)
    st = lib.lhaf_noalloc(0, stream, len(zero), B.data_ptr(), None, zero.ctypes.data, 0, out.data_ptr())
    torch.cuda.synchronize()
    assert st == 0 and complex(out.cpu()[0]) == 1.0


def test_noalloc_fp32_only_within_its_bound(env):
    # FP32 terms are refused above degree 18 (N = 38 here), and accepted below it
    torch, lg, lib = env
    big = wl.large_lhaf_60(seed=100, n_photons=38)
    st, _ = _call(torch, lib, big, flags=lg.FP32_TERMS)
    assert st == 2
    small = wl.single_lhaf_24(seed=2, n_photons=16)
    with lg.Context(0) as ctx:
        ref = ctx.lhaf(small.B, small.gamma, small.reps)
    st, got = _call(torch, lib, small, flags=lg.FP32_TERMS)
    assert st == 0 and abs(got - ref) <= 1e-2 * abs(ref)
