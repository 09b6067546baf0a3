"""Pins for orthogonal iterations, Rayleigh-Ritz and the sign rule
(Algorithm 1, Eq. 5, Eq. 7)."""

import numpy as np
import pytest

from oracle import subspace
from synth import icosphere, SequenceSpec, sinusoid_rigid_motion


def _principal_sines(U1, U2):
    s = np.linalg.svd(U1.T @ U2, compute_uv=False)
    return np.sqrt(np.clip(1.0 - s ** 2, 0.0, None))


def test_start_basis_orthonormal_and_seeded():
    Q = subspace.start_basis(64, 16, 7, 0)
    np.testing.assert_allclose(Q.T @ Q, np.eye(16), atol=1e-14)
    assert not np.allclose(Q, subspace.start_basis(64, 16, 7, 1))
    np.testing.assert_array_equal(Q, subspace.start_basis(64, 16, 7, 0))


@pytest.mark.parametrize("level,F,k", [(0, 12, 3), (1, 24, 5), (1, 32, 8)])
def test_oi_matches_brute_force_eigendecomposition(level, F, k):
    v, t = icosphere(level)
    spec = SequenceSpec(name="tiny", mesh=f"icosphere:{level}", n_frames=F, rank=k,
                        n_anchors=0, seed=11 + level)
    pos = sinusoid_rigid_motion(v, spec)
    for c in range(3):
        A = pos[:, :, c]
        Ub, lam = subspace.brute_force_basis(A, k)
        gap = lam[k] / lam[k - 1]
        U, theta, done, change = subspace.top_k_basis(A, k, seed=5, c=c, sweeps=400, tol=1e-13)
        np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-13)
        assert _principal_sines(U, Ub).max() < 1e-6 or gap > 0.999
        np.testing.assert_allclose(theta, lam[:k], rtol=1e-9, atol=1e-12 * lam[0])
        # Ritz vectors of well-separated eigenvalues equal the eigenvectors
        # themselves (with the same sign rule)
        sep = np.ones(k, dtype=bool)
        rel = np.abs(np.diff(lam[:k + 1])) / lam[0]
        sep[:] = (rel[:k] > 1e-6) & (np.r_[1.0, rel[:k - 1]] > 1e-6)
        np.testing.assert_allclose(U[:, sep], Ub[:, sep], atol=1e-6)


def test_exact_low_rank_trajectories_are_captured():
    r = np.random.default_rng(0)
    F, n, rank = 40, 300, 6
    A = r.normal(size=(F, rank)) @ r.normal(size=(rank, n))
    U, theta, _, _ = subspace.top_k_basis(A, 8, seed=1, c=0, sweeps=60)
    resid = A - U @ (U.T @ A)
    assert np.linalg.norm(resid) < 1e-10 * np.linalg.norm(A)
    assert theta[rank] < 1e-18 * theta[0] + 1e-9


def test_eigenvalues_descending_and_sign_rule():
    r = np.random.default_rng(1)
    A = r.normal(size=(20, 200))
    U, theta, _, _ = subspace.top_k_basis(A, 5, seed=2, c=0, sweeps=200)
    assert np.all(np.diff(theta) <= 0)
    w = np.arange(1, 21)
    assert np.all(w @ U > 0)
    # flipping the input basis does not change the result
    U2 = subspace.sign_rule(-U)
    np.testing.assert_array_equal(U2, U)


def test_sign_rule_fallback_for_balanced_columns():
    u = np.array([[1.0], [-3.0], [1.0], [0.5]])   # weighted sum 1 - 6 + 3 + 2 = 0
    out = subspace.sign_rule(u / np.linalg.norm(u))
    assert out[1, 0] > 0   # largest |entry| made positive


def test_fixed_sweep_count_is_deterministic():
    r = np.random.default_rng(2)
    A = r.normal(size=(16, 100))
    Q0 = subspace.start_basis(16, 4, 3, 0)
    Q1, d1, _ = subspace.orthogonal_iterations(A, Q0, 5)
    Q2, d2, _ = subspace.orthogonal_iterations(A, Q0, 5)
    assert d1 == d2 == 5
    np.testing.assert_array_equal(Q1, Q2)
