"""Pins for the oracle's inner Nesterov loop (Sec. 2) against facts it does not compute itself.

* alpha/beta series: closed forms (golden ratio ...) and the identity
  alpha_{k+1}^2 - alpha_{k+1} = alpha_k^2;
* the loop's limit: the unique NNLS minimiser, found by exhaustive active-set
  enumeration (oracle.bruteforce) and by scipy's Lawson-Hanson NNLS;
* the loop's speed: the O(1/k^2) bound of accelerated projected gradient
  (Beck and Teboulle 2009, Thm. 4.4), which a dropped or sign-flipped
  extrapolation violates on an ill-conditioned problem;
* p = 1 closed form, KKT conditions, the stopping test, H = 0.
"""

import math
import os

import numpy as np
import pytest
import scipy.optimize

from oracle import bruteforce, nenmf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_alpha():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "alpha_series.txt")) if l.strip() and not l.startswith("#")]
    return np.array([[float(v) for v in r[1:]] for r in rows])


def test_alpha_series_closed_values():
    tab = _golden_alpha()
    a = nenmf.alpha_sequence(5)
    b = nenmf.extrapolation_weights(5)
    np.testing.assert_allclose(a[:5], tab[:, 0], atol=1e-10)
    np.testing.assert_allclose(b[:5], tab[:, 1], atol=1e-10)
    assert a[1] == pytest.approx((1 + math.sqrt(5)) / 2, abs=1e-15)
    assert b[0] == 0.0


def test_alpha_identity_and_growth():
    a = nenmf.alpha_sequence(200)
    np.testing.assert_allclose(a[1:] ** 2 - a[1:], a[:-1] ** 2, rtol=1e-13)
    k = np.arange(a.size)
    assert np.all(a >= (k + 2) / 2 - 1e-12) and np.all(a <= k + 1 + 1e-12)
    b = nenmf.extrapolation_weights(200)
    assert np.all(np.diff(b) > 0) and np.all(b < 1)


def _spd_problem(rng, p, N, rows=None, cond=None):
    rows = rows or 3 * p
    A = rng.standard_normal((rows, p))
    if cond is not None:
        U, _, Vt = np.linalg.svd(A, full_matrices=False)
        s = np.geomspace(1.0, 1.0 / math.sqrt(cond), p)
        A = U @ np.diag(s) @ Vt
    Xc = rng.standard_normal((rows, N))
    return A, Xc, A.T @ A, A.T @ Xc


@pytest.mark.parametrize("p", [1, 2, 3, 5, 6])
def test_limit_is_bruteforce_nnls(p):
    rng = np.random.default_rng(100 + p)
    A, Xc, H, B = _spd_problem(rng, p, 8)
    Y0 = rng.random((p, 8))
    F, iters, pg = nenmf.nesterov_nnls(H, B, Y0, max_inner=4000)
    assert iters == 4000
    F_bf = bruteforce.nnls_enumerate_columns(H, B)
    np.testing.assert_allclose(F, F_bf, atol=1e-8)
    for j in range(8):
        f_sp, _ = scipy.optimize.nnls(A, Xc[:, j])
        np.testing.assert_allclose(F[:, j], f_sp, atol=1e-8)
    assert pg < 1e-7


def test_p1_closed_form_in_one_step():
    # p = 1: L_c = h, so the first projected step lands on max(0, b/h) exactly.
    h = np.array([[2.5]])
    b = np.array([[3.0, -1.0, 0.0, 7.5]])
    y0 = np.array([[0.3, 4.0, 1.0, 0.0]])
    F, it, pg = nenmf.nesterov_nnls(h, b, y0, max_inner=1)
    np.testing.assert_allclose(F, np.maximum(0.0, b / 2.5), rtol=0, atol=1e-15)
    F5, _, _ = nenmf.nesterov_nnls(h, b, y0, max_inner=5)
    np.testing.assert_allclose(F5, F, atol=1e-15)


def _objective(H, B, F):
    return 0.5 * np.sum(F * (H @ F)) - np.sum(B * F)


def test_accelerated_rate_bound():
    # Beck-Teboulle Thm 4.4 for x_{k+1} = F_k: f(F_k) - f* <= 2 L ||Y0 - F*||^2 / (k+2)^2.
    rng = np.random.default_rng(7)
    p, N = 6, 4
    A, Xc, H, B = _spd_problem(rng, p, N, cond=1e5)
    Fstar = bruteforce.nnls_enumerate_columns(H, B)
    fstar = _objective(H, B, Fstar)
    Y0 = 10.0 * rng.random((p, N))
    L = nenmf.lipschitz_constant(H)
    d2 = np.sum((Y0 - Fstar) ** 2)
    gaps = []
    for K in range(1, 301):
        F, _, _ = nenmf.nesterov_nnls(H, B, Y0, max_inner=K)
        gaps.append(_objective(H, B, F) - fstar)
    gaps = np.array(gaps)
    k = np.arange(300)
    assert np.all(gaps <= 2 * L * d2 / (k + 2) ** 2 * (1 + 1e-9) + 1e-12)
    # The same problem separates acceleration from plain projected gradient,
    # whose O(1/k) decay breaks the bound: the pin can see a dropped momentum term.
    Fpg = Y0.copy()
    worst = 0.0
    for K in range(300):
        Fpg = np.maximum(0.0, Fpg - (H @ Fpg - B) / L)
        worst = max(worst, (_objective(H, B, Fpg) - fstar) / (2 * L * d2 / (K + 2) ** 2))
    assert worst > 1.0


def test_kkt_at_convergence():
    rng = np.random.default_rng(3)
    A, Xc, H, B = _spd_problem(rng, 8, 50)
    F, _, pg = nenmf.nesterov_nnls(H, B, rng.random((8, 50)), max_inner=3000)
    grad = H @ F - B
    assert np.all(F >= 0)
    assert np.max(np.abs(nenmf.projected_gradient(F, grad))) < 1e-8
    assert np.max(np.abs(F * grad)) < 1e-8
    assert np.all(grad[F == 0] >= -1e-8)


def test_stopping_test_stops_at_first_pass():
    rng = np.random.default_rng(4)
    A, Xc, H, B = _spd_problem(rng, 5, 20)
    Y0 = rng.random((5, 20))
    eps = 1e-3
    F, k, pg = nenmf.nesterov_nnls(H, B, Y0, max_inner=1000, eps=eps)
    assert 1 < k < 1000 and pg <= eps
    _, _, pg_prev = nenmf.nesterov_nnls(H, B, Y0, max_inner=k - 1)
    assert pg_prev > eps
    # min_inner forces at least that many iterations even when the test passes.
    _, k2, _ = nenmf.nesterov_nnls(H, B, Y0, max_inner=1000, min_inner=k + 5, eps=eps)
    assert k2 == k + 5


def test_zero_gram_returns_start():
    Y0 = np.array([[1.0, 0.0], [2.0, 3.0]])
    F, k, _ = nenmf.nesterov_nnls(np.zeros((2, 2)), np.zeros((2, 2)), Y0, max_inner=10)
    assert k == 0
    np.testing.assert_array_equal(F, Y0)


def test_projected_gradient_definition():
    F = np.array([[0.0, 0.0, 1.0, 2.0]])
    g = np.array([[-1.0, 3.0, -4.0, 5.0]])
    np.testing.assert_array_equal(nenmf.projected_gradient(F, g), [[-1.0, 0.0, -4.0, 5.0]])


def test_interior_trajectory_follows_golden_weights():
    # Decoupled quadratic whose minimiser is interior and stays so: each
    # coordinate obeys e_k = (1 - h/L) (Y_k - f*), Y_{k+1} - f* = (1 + b_k) e_k - b_k e_{k-1},
    # run here with the golden beta table, so the loop's beta index is pinned.
    tab = _golden_alpha()
    h = np.array([4.0, 1.0, 0.25])
    H = np.diag(h)
    fstar = np.array([5.0, 6.0, 7.0])
    B = (H @ fstar)[:, None]
    Y0 = (fstar + np.array([0.5, -0.7, 0.9]))[:, None]
    Lc = h.max()
    y = Y0[:, 0] - fstar
    e_prev = y.copy()
    for k in range(5):
        e = (1 - h / Lc) * y
        y = e + tab[k, 1] * (e - e_prev)
        e_prev = e
        F, it, _ = nenmf.nesterov_nnls(H, B, Y0, max_inner=k + 1)
        np.testing.assert_allclose(F[:, 0] - fstar, e, atol=1e-9)
