"""GPU parity of the batched form (one persistent launch for many loop hafnians of uneven size)
against the oracle and against one lhaf() call per item."""
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


def test_batched_small_mixed_against_oracle(ctx, lg):
    rng = np.random.default_rng(17)
    M = 6
    B = wl.random_symmetric(rng, M) * 0.5
    reps = [rng.integers(0, 4, size=M) for _ in range(40)]
    reps += [np.zeros(M, int), np.array([1, 0, 0, 2, 0, 0]), np.array([3, 0, 0, 0, 0, 0])]
    gammas = np.array([wl.complex_normal(rng, M) for _ in reps])
    gammas[5] = 0.0  # one item without loops
    R = np.array(reps, dtype=np.int32)
    vals, status = ctx.lhaf_batched(B, gammas, R)
    assert np.all(status == 0)
    for i in range(len(R)):
        ref = lo.lhaf_repeated(B, gammas[i], R[i])
        if abs(ref) < 1e-12:
            assert abs(vals[i]) < 1e-11
        else:
            assert rel(vals[i], ref) < TOL, (i, R[i], vals[i], ref)


def test_batched_status_per_item(ctx, lg):
    rng = np.random.default_rng(2)
    M = 70
    B = wl.random_symmetric(rng, M) * 0.3
    R = np.zeros((3, M), np.int32)
    R[0, :4] = [1, 2, 0, 1]
    R[1, :] = 1          # 35 pairs + border: above the compiled limit
    R[2, :3] = [1, -1, 1]  # invalid
    vals, status = ctx.lhaf_batched(B, None, R)
    assert list(status) == [0, 2, 1]
    assert np.isnan(vals[1]) and np.isnan(vals[2])
    assert rel(vals[0], lo.lhaf_repeated(B, np.diag(B).copy(), R[0])) < TOL


def test_chain_rule_batch_sample_matches_single_calls(ctx, lg):
    b = wl.chain_rule_batch(seed=3, count=96)
    R = np.array(b.reps)
    G = np.array(b.gammas)
    vals, status, st = ctx.lhaf_batched(b.B, G, R, stats=True)
    assert np.all(status == 0)
    for i in range(len(R)):
        single = ctx.lhaf(b.B, G[i], R[i])
        assert rel(vals[i], single) < TOL, i
    # oracle on the smaller items
    small = [i for i in range(len(R)) if R[i].sum() <= 18][:12]
    for i in small:
        assert rel(vals[i], lo.lhaf_repeated(b.B, G[i], R[i])) < TOL


def test_batched_per_item_B_and_device_pointers(ctx, lg):
    import torch

    rng = np.random.default_rng(5)
    M, n = 8, 20
    Bs = np.array([wl.random_symmetric(rng, M) * 0.4 for _ in range(n)])
    G = np.array([wl.complex_normal(rng, M) for _ in range(n)])
    R = np.array([rng.multinomial(int(rng.integers(2, 14)), np.ones(M) / M) for _ in range(n)], np.int32)
    host, status = ctx.lhaf_batched(Bs, G, R, flags=lg.BATCH_B_PER_ITEM)
    assert np.all(status == 0)
    for i in range(n):
        assert rel(host[i], lo.lhaf_repeated(Bs[i], G[i], R[i])) < TOL
    out, status = ctx.lhaf_batched(torch.from_numpy(Bs).cuda(), torch.from_numpy(G).cuda(), R,
                                   flags=lg.BATCH_B_PER_ITEM)
    torch.cuda.synchronize()
    assert np.all(np.abs(out.cpu().numpy() - host) <= 1e-13 * np.abs(host))


def test_ill_conditioned_chain_rule_items_against_extended_oracle(ctx, lg):
    # The most cancelling items of the 4096-item chain-rule batch (sum |weight f| / |sum| = 8e6 ..
    # 5e7) against the C oracle's long double values (tests/golden, written by the committed
    # script beside them): an FP64 sum of such terms keeps about 16 - log10(condition) digits, so
    # the bound is condition x 2^-52 (the FP64 C oracle itself is 1.8e-10 off on the worst item),
    # for the batched form and for one call per item alike.
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "chain_rule_ill_conditioned.json")) as f:
        gold = json.load(f)["items"]
    b = wl.chain_rule_batch(seed=3, count=4096)
    idx = [it["index"] for it in gold]
    R = np.array([b.reps[i] for i in idx], dtype=np.int32)
    G = np.array([b.gammas[i] for i in idx])
    vals, st = ctx.lhaf_batched(b.B, G, R)
    assert np.all(st == 0)
    for k, it in enumerate(gold):
        ref = complex(*it["value"])
        tol = max(TOL, it["condition"] * 2.0 ** -52)
        assert rel(vals[k], ref) <= tol, (it["index"], rel(vals[k], ref), tol)
        assert rel(ctx.lhaf(b.B, G[k], R[k]), ref) <= tol
        assert rel(complex(*it["fp64_c_oracle"]), ref) <= tol  # the FP64 oracle meets the same bound
