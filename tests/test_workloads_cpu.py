"""The seeded input recipes hold what they state: pattern sizes and count caps,
unitary interferometers, symmetric kernels, physical (lossy) covariances, interleaved block pairs."""
import numpy as np

from paper_2108_01622_gb300 import workloads as wl


def test_haar_unitary_and_symmetric_kernel():
    U = wl.haar_unitary(np.random.default_rng(0), 12)
    assert np.allclose(U @ U.conj().T, np.eye(12), atol=1e-12)
    B = wl.kernel_from_squeezing(U, np.full(12, 0.7))
    assert np.allclose(B, B.T, atol=1e-14)
    # B = U diag(tanh r) U^T: singular values tanh r
    assert np.allclose(np.linalg.svd(B, compute_uv=False), np.tanh(0.7), atol=1e-12)


def test_pattern_recipes():
    p = wl.collision_lhaf_40(seed=2)
    assert p.reps.sum() == 40 and np.count_nonzero(p.reps) == 22 and p.reps.max() <= 4
    assert np.all(p.gamma == 0)
    q = wl.single_lhaf_24(seed=1)
    assert q.reps.sum() == 24 and q.reps.max() == 1
    big = wl.large_lhaf_60(seed=5)
    assert big.reps.sum() == 60 and big.reps.max() == 1
    b = wl.chain_rule_batch(seed=3, count=64)
    for r in b.reps:
        assert 10 <= r.sum() <= 40 and r.max() <= 3


def test_lossy_state_is_physical():
    st = wl.lossy_state(seed=3, M=4, eta=0.6)
    sig = st.sigma
    assert np.allclose(sig, sig.conj().T, atol=1e-14)
    # a physical state: sigma_Q = sigma + I/2 positive definite and sigma - I/2 ... >= 0 in the
    # sense of the uncertainty relation sigma + (1/2) Z >= 0 with Z = diag(I, -I)
    M = 4
    Zs = np.diag(np.concatenate([np.ones(M), -np.ones(M)]))
    assert np.linalg.eigvalsh(sig + 0.5 * np.eye(2 * M)).min() > 0
    assert np.linalg.eigvalsh(sig + 0.5 * Zs).min() > -1e-12
    # no loss: a pure state (symplectic eigenvalues 1/2: det sigma = 4^-M)
    pure = wl.lossy_state(seed=3, M=4, eta=1.0).sigma
    assert np.isclose(np.linalg.det(pure).real, 0.25 ** M, rtol=1e-9)


def test_block_pair_interleaves_blocks():
    bp = wl.block_diagonal_pair(seed=1, n=5)
    assert np.allclose(bp.C[0::2, 0::2], bp.A1) and np.allclose(bp.C[1::2, 1::2], bp.A2)
    assert np.all(bp.C[0::2, 1::2] == 0) and np.all(bp.C[1::2, 0::2] == 0)
    assert np.allclose(bp.A1, bp.A1.T) and np.allclose(bp.A2, bp.A2.T)
