"""Pins for the oracle's Alg. 2 (randomized subspace iteration) and its QR convention.

* orthonormal_basis against an independent Cholesky-based construction and the
  defining properties of the positive-diagonal QR;
* projector exactness on exactly low-rank X (nu >= rank X): L^T L X = X and
  X R R^T = X to rounding;
* the power iterations: on X with a known spectrum the principal angle between
  range(L^T) and the leading left singular subspace shrinks like
  (sigma_{nu+1}/sigma_k)^(2q+1); a missing power step (q effectively 0) fails;
* the Eckart-Young lower bound.
"""

import numpy as np
import pytest

import synth
from oracle import subspace


def test_orthonormal_basis_matches_cholesky_route():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((60, 7))
    Q = subspace.orthonormal_basis(Y)
    Rc = np.linalg.cholesky(Y.T @ Y).T          # upper, positive diagonal
    Qc = Y @ np.linalg.inv(Rc)
    np.testing.assert_allclose(Q, Qc, atol=1e-12)
    np.testing.assert_allclose(Q.T @ Q, np.eye(7), atol=1e-13)
    Rq = Q.T @ Y
    assert np.allclose(np.tril(Rq, -1), 0, atol=1e-12) and np.all(np.diag(Rq) > 0)


def _exact_rank(n, m, p, seed):
    X, G0, F0 = synth.lowrank_data(n, m, p, seed)
    return X


@pytest.mark.parametrize("n,m,p,nu,q", [(90, 70, 4, 6, 0), (90, 70, 4, 4, 2), (61, 83, 5, 9, 4)])
def test_projector_exact_on_low_rank(n, m, p, nu, q):
    X = _exact_rank(n, m, p, seed=n + m)
    Om_L, Om_R = synth.gaussian_sketches(n, m, nu, seed=3)
    L, R, XL, XR = subspace.compress(X, nu, q, Om_L, Om_R)
    assert L.shape == (nu, n) and R.shape == (m, nu) and XL.shape == (nu, m) and XR.shape == (n, nu)
    np.testing.assert_allclose(L @ L.T, np.eye(nu), atol=1e-12)
    np.testing.assert_allclose(R.T @ R, np.eye(nu), atol=1e-12)
    nx = np.linalg.norm(X)
    assert np.linalg.norm(X - L.T @ (L @ X)) / nx < 1e-12
    assert np.linalg.norm(X - (X @ R) @ R.T) / nx < 1e-12
    np.testing.assert_allclose(XL, L @ X, atol=1e-12 * nx)
    np.testing.assert_allclose(XR, X @ R, atol=1e-12 * nx)


def _known_spectrum(n, m, sig, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((n, len(sig))))
    V, _ = np.linalg.qr(rng.standard_normal((m, len(sig))))
    return U, V, (U * sig) @ V.T


@pytest.mark.parametrize("q,bound", [(3, 1e-4), (4, 1e-5)])
def test_power_iterations_converge_to_leading_subspace(q, bound):
    n, m, k, nu = 120, 100, 5, 8
    sig = np.concatenate([np.ones(k), 0.1 * np.ones(40)])
    U, V, X = _known_spectrum(n, m, sig, seed=11)
    Om_L, Om_R = synth.gaussian_sketches(n, m, nu, seed=5)
    L, R = subspace.randomized_subspace_iteration(X, nu, q, Om_L, Om_R)
    angle_L = np.linalg.norm(U[:, :k] - L.T @ (L @ U[:, :k]), 2)
    angle_R = np.linalg.norm(V[:, :k] - R @ (R.T @ V[:, :k]), 2)
    assert angle_L < bound and angle_R < bound
    # Without power steps the same sketch is far from the leading subspace.
    L0, R0 = subspace.randomized_subspace_iteration(X, nu, 0, Om_L, Om_R)
    assert np.linalg.norm(U[:, :k] - L0.T @ (L0 @ U[:, :k]), 2) > 10 * bound


def test_eckart_young_lower_bound():
    X, _, _ = synth.lowrank_data(80, 60, 4, seed=2, snr_db=20.0)
    s = np.linalg.svd(X, compute_uv=False)
    for nu, q in [(4, 0), (6, 2), (10, 4)]:
        Om_L, Om_R = synth.gaussian_sketches(80, 60, nu, seed=nu)
        L, R, XL, XR = subspace.compress(X, nu, q, Om_L, Om_R)
        tail = np.sqrt(np.sum(s[nu:] ** 2))
        err_L = np.linalg.norm(X - L.T @ XL)
        err_R = np.linalg.norm(X - XR @ R.T)
        assert err_L >= tail * (1 - 1e-12) and err_R >= tail * (1 - 1e-12)
        if q >= 2:
            assert err_L <= 1.05 * tail and err_R <= 1.05 * tail


def test_rejects_wrong_sketch_shapes():
    X = np.ones((5, 4))
    with pytest.raises(ValueError):
        subspace.randomized_subspace_iteration(X, 2, 1, np.ones((5, 2)), np.ones((2, 5)))
