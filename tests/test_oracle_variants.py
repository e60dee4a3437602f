"""Pins of the compression variants (oracle.subspace.compression_bases).

  * orthonormality of the bases of every orthonormalising variant;
  * exactly low-rank X (rank r <= nu): every orthonormalising variant's
    projectors reproduce X (L^T L X = X, X R R^T = X) to rounding;
  * power iteration spans, in exact arithmetic, the subspace of subspace
    iteration: at q = 1, 2 on a matrix with a clear spectral gap the two
    subspaces agree to ~1e-10 (principal angles);
  * swapped / single: the half-step bases are the orthonormal bases of the
    named products (X^T Q_L, X Q_R^T), so their subspace angles to the leading
    singular subspaces shrink with q like the default's;
  * Gaussian projection: norm preserving in expectation, E ||L x||^2 = ||x||^2.
"""

import numpy as np
import pytest

import synth
from oracle import subspace


def _angle(A, B):
    """Sine of the largest principal angle between the column spaces of A and B
    (equal dimensions): ||(I - Qa Qa^T) Qb||_2, accurate to rounding."""
    Qa = np.linalg.qr(A)[0]
    Qb = np.linalg.qr(B)[0]
    return float(np.linalg.norm(Qb - Qa @ (Qa.T @ Qb), 2))


def _sk(n, m, nu, seed=4):
    return synth.gaussian_sketches(n, m, nu, seed=seed)


@pytest.mark.parametrize("variant", ["subspace", "swapped", "single", "power"])
def test_orthonormal_and_exact_on_low_rank(variant):
    n, m, r, nu, q = 120, 90, 5, 9, 2
    X, _, _ = synth.lowrank_data(n, m, r, seed=2)
    L, R = subspace.compression_bases(X, nu, q, *_sk(n, m, nu), variant=variant)
    assert L.shape == (nu, n) and R.shape == (m, nu)
    np.testing.assert_allclose(L @ L.T, np.eye(nu), atol=1e-10)
    np.testing.assert_allclose(R.T @ R, np.eye(nu), atol=1e-10)
    nx = np.linalg.norm(X)
    assert np.linalg.norm(X - L.T @ (L @ X)) <= 1e-10 * nx
    assert np.linalg.norm(X - (X @ R) @ R.T) <= 1e-10 * nx


@pytest.mark.parametrize("q", [1, 2])
def test_power_iteration_spans_the_subspace_iteration_subspace(q):
    # singular values 1 .. 0.3 over nu columns, well separated from the rest (0.01)
    n, m, nu = 150, 110, 8
    rng = np.random.default_rng(7)
    U = np.linalg.qr(rng.standard_normal((n, n)))[0]
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    s = np.concatenate([np.linspace(1.0, 0.3, nu), np.full(m - nu, 0.01)])
    X = (U[:, :m] * s) @ V.T
    OmL, OmR = _sk(n, m, nu, seed=9)
    Ls, Rs = subspace.compression_bases(X, nu, q, OmL, OmR, "subspace")
    Lp, Rp = subspace.compression_bases(X, nu, q, OmL, OmR, "power")
    assert _angle(Ls.T, Lp.T) <= 1e-10
    assert _angle(Rs, Rp) <= 1e-10


@pytest.mark.parametrize("variant", ["swapped", "single"])
def test_half_step_bases_converge_with_q(variant):
    n, m, nu, p = 200, 160, 10, 4
    X, _, _ = synth.lowrank_data(n, m, p, seed=11, snr_db=15.0)
    U, _, Vt = np.linalg.svd(X, full_matrices=False)
    prev_l = prev_r = 1.0
    for q in (1, 2, 4):
        L, R = subspace.compression_bases(X, nu, q, *_sk(n, m, nu, seed=13), variant=variant)
        al = np.linalg.norm(U[:, :p] - L.T @ (L @ U[:, :p]), 2)
        ar = np.linalg.norm(Vt[:p].T - R @ (R.T @ Vt[:p].T), 2)
        assert al <= prev_l * 1.0001 and ar <= prev_r * 1.0001
        prev_l, prev_r = al, ar
    assert prev_l < 1e-3 and prev_r < 1e-3


def test_swapped_half_steps_are_the_named_products():
    # L = Q~_R^(q) spans X Q_R^(q-1)^T's columns; R = Q~_L^(q) spans X^T Q_L^(q-1)
    n, m, nu, q = 70, 60, 6, 2
    X, _, _ = synth.lowrank_data(n, m, 4, seed=5, snr_db=10.0)
    OmL, OmR = _sk(n, m, nu)
    Ld, Rd = subspace.compression_bases(X, nu, q - 1, OmL, OmR, "subspace")   # Q_L^(q-1)^T, Q_R^(q-1)^T
    L, R = subspace.compression_bases(X, nu, q, OmL, OmR, "swapped")
    assert _angle(L.T, X @ Rd) <= 1e-10
    assert _angle(R, X.T @ Ld.T) <= 1e-10


def test_gaussian_projection_preserves_norm_in_expectation():
    n, m, nu = 400, 300, 20
    x = np.random.default_rng(3).standard_normal(n)
    ratios = []
    for seed in range(200):
        L, R = subspace.compression_bases(np.ones((n, m)), nu, 0, *_sk(n, m, nu, seed=seed), variant="gaussian")
        ratios.append(np.sum((L @ x) ** 2) / np.sum(x ** 2))
    # chi-square with nu dof / nu: mean 1, sd sqrt(2/nu)/sqrt(200) = 0.016
    assert abs(np.mean(ratios) - 1.0) < 0.06
