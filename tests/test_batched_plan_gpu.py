"""GPU parity of the batched plan (patterns planned once, launches replayed from a CUDA graph for
new values of B and gamma) against the oracle and against lhaf_batched."""
import numpy as np
import pytest

from oracle import lhaf_oracle as lo
from paper_2108_01622_gb300 import workloads as wl
from tests.libutil import ensure_built

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def lg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


@pytest.fixture(scope="module")
def ctx(lg):
    c = lg.Context(0)
    yield c
    c.close()


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _mixed(seed, M=6, n=30):
    rng = np.random.default_rng(seed)
    B = wl.random_symmetric(rng, M) * 0.5
    R = np.array([rng.integers(0, 4, size=M) for _ in range(n)] + [np.zeros(M, int), [3, 0, 0, 0, 0, 0]],
                 dtype=np.int32)
    G = np.array([wl.complex_normal(rng, M) for _ in range(len(R))])
    return B, G, R


def test_plan_replays_new_values_against_oracle(ctx, lg):
    B, G, R = _mixed(3)
    with ctx.batched_plan(B, G, R) as plan:
        for seed in (4, 5):
            B2, G2, _ = _mixed(seed)
            G2[7] = 0.0  # an item without loops (the plan keeps its border)
            vals, status = plan.run(B2, G2)
            assert np.all(status == 0)
            for i in range(len(R)):
                ref = lo.lhaf_repeated(B2, G2[i], R[i])
                if abs(ref) < 1e-12:
                    assert abs(vals[i]) < 1e-11
                else:
                    assert rel(vals[i], ref) < TOL, (seed, i, R[i], vals[i], ref)
            same, _ = ctx.lhaf_batched(B2, G2, R)
            assert np.all(np.abs(vals - same) <= 1e-12 * np.maximum(np.abs(same), 1e-300) + 1e-300)


def test_plan_device_pointers_per_item_B_diag_loops(ctx, lg):
    import torch

    rng = np.random.default_rng(8)
    M, n = 7, 24
    Bs = np.array([wl.random_symmetric(rng, M) * 0.4 for _ in range(n)])
    R = np.array([rng.multinomial(int(rng.integers(1, 13)), np.ones(M) / M) for _ in range(n)], np.int32)
    plan = ctx.batched_plan(torch.from_numpy(Bs).cuda(), None, R, flags=lg.BATCH_B_PER_ITEM)
    Bs2 = np.array([wl.random_symmetric(rng, M) * 0.4 for _ in range(n)])
    out, status = plan.run(torch.from_numpy(Bs2).cuda())
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.all(status == 0)
    for i in range(n):
        assert rel(got[i], lo.lhaf_repeated(Bs2[i], np.diag(Bs2[i]).copy(), R[i])) < TOL
    plan.close()
    with pytest.raises(RuntimeError):
        plan.run(torch.from_numpy(Bs2).cuda())


def test_plan_status_and_nonfinite_host_values(ctx, lg):
    rng = np.random.default_rng(9)
    M = 70
    B = wl.random_symmetric(rng, M) * 0.3
    R = np.zeros((4, M), np.int32)
    R[0, :4] = [1, 2, 0, 1]
    R[1, :] = 1              # 35 pairs + border: above the compiled limit
    R[2, :3] = [1, -1, 1]    # invalid pattern
    R[3, 5:9] = [2, 1, 1, 0]
    G = np.array([wl.complex_normal(rng, M) for _ in range(4)])
    plan = ctx.batched_plan(B, G, R)
    vals, status = plan.run(B, G)
    assert list(status) == [0, 2, 1, 0]
    assert np.isnan(vals[1]) and np.isnan(vals[2])
    assert rel(vals[0], lo.lhaf_repeated(B, G[0], R[0])) < TOL
    assert rel(vals[3], lo.lhaf_repeated(B, G[3], R[3])) < TOL
    G2 = G.copy()
    G2[3, 6] = np.nan       # read by item 3 only
    G2[0, 40] = np.inf      # mode 40 is empty in item 0: not read
    vals, status = plan.run(B, G2)
    assert list(status) == [0, 2, 1, 1]
    assert np.isnan(vals[3]) and rel(vals[0], lo.lhaf_repeated(B, G[0], R[0])) < TOL
    with pytest.raises(ValueError):
        plan.run(B, None)
    plan.close()


def test_plan_chain_rule_sample_matches_batched(ctx, lg):
    b = wl.chain_rule_batch(seed=3, count=96)
    R = np.array(b.reps)
    G = np.array(b.gammas)
    with ctx.batched_plan(b.B, G, R) as plan:
        vals, status, st = plan.run(b.B, G, stats=True)
        ref, _ = ctx.lhaf_batched(b.B, G, R)
    assert np.all(status == 0) and st["terms"] > 0 and st["kernel_ms"] > 0
    for i in range(len(R)):
        assert rel(vals[i], ref[i]) < TOL, i
