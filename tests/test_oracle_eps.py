"""Pins for the stop threshold eps of the inner loop (Sec. 2, the KKT /
projected-gradient stopping rule).

eps = tol * ||[P grad_G ; P grad_F]||_F at the initial (G0, F0), so every
early stop of a run with tol > 0 depends on the two arrays that
oracle.nenmf.initial_pg_parts_plain / _compressed return. They are checked
here entry by entry against quantities built without their formulas:

* the gradient comes from central differences of the objective itself,
  evaluated as a plain sum of squared residuals. Each objective is a
  quadratic in the coordinate being varied, so a central difference is exact
  up to rounding (no truncation term), for any step h;
* the KKT projection comes from the gradient mapping of projected gradient
  descent, (x - max(0, x - t g)) / t, at a step t small enough that no
  positive coordinate reaches the bound: it equals g where x > 0 and
  min(0, g) where x = 0;
* the compressed case differentiates the two objectives Alg. 1 alternates:
  1/2 ||X_R - G (F R)||^2 in G and 1/2 ||X_L - (L G) F||^2 in F.

The inputs hold exact zeros in G and F with gradients of both signs there,
so both branches of the projection are exercised. Two planted mistakes (an
unprojected gradient, the projection on the wrong side) must fail the same
comparison.
"""

import numpy as np
import pytest

import synth
from oracle import nenmf, subspace


def _objective_plain(X, G, F):
    r = X - G @ F
    return 0.5 * float(np.sum(r * r))


def _central_gradient(f, A, h=1e-3):
    """Entry-wise central differences of the scalar function f at the array A."""
    g = np.zeros_like(A)
    for idx in np.ndindex(A.shape):
        Ap, Am = A.copy(), A.copy()
        Ap[idx] += h
        Am[idx] -= h
        g[idx] = (f(Ap) - f(Am)) / (2.0 * h)
    return g


def _gradient_mapping(x, g):
    """(x - max(0, x - t g)) / t with t below every positive x / |g|."""
    pos = x > 0
    ratios = x[pos] / np.maximum(np.abs(g[pos]), 1e-300)
    t = 0.5 * float(min(1.0, ratios.min() if ratios.size else 1.0))
    return (x - np.maximum(0.0, x - t * g)) / t


def _case(seed, n=7, m=6, p=2):
    rng = np.random.default_rng(seed)
    X, _, _ = synth.lowrank_data(n, m, p, seed=seed, snr_db=10.0)
    G, F = synth.initial_factors(n, m, p, seed=seed + 1)
    G[rng.random(G.shape) < 0.35] = 0.0
    F[rng.random(F.shape) < 0.35] = 0.0
    # scale the product to overshoot the data on average, so residuals (and
    # the gradients at zero entries) take both signs
    s = np.sqrt(1.3 * X.mean() / (G @ F).mean())
    return X, G * s, F * s


def _reference_plain(X, G, F):
    gG = _central_gradient(lambda A: _objective_plain(X, A, F), G)
    gF = _central_gradient(lambda A: _objective_plain(X, G, A), F)
    return _gradient_mapping(G, gG), _gradient_mapping(F, gF), gG, gF


def _reference_compressed(L, R, XL, XR, G, F):
    def obj_G(A):   # eq. (2) with X, F replaced by X_R, F R
        r = XR - A @ (F @ R)
        return 0.5 * float(np.sum(r * r))

    def obj_F(A):   # eq. (3) with X, G replaced by X_L, L G
        r = XL - (L @ G) @ A
        return 0.5 * float(np.sum(r * r))

    gG = _central_gradient(obj_G, G)
    gF = _central_gradient(obj_F, F)
    return _gradient_mapping(G, gG), _gradient_mapping(F, gF), gG, gF


def _compressed_case(seed):
    X, G, F = _case(seed)
    n, m = X.shape
    OmL, OmR = synth.gaussian_sketches(n, m, 3, seed=seed + 2)
    L, R, XL, XR = subspace.compress(X, 3, 1, OmL, OmR)
    return L, R, XL, XR, G, F


def _both_branches(G, F, ref):
    """The case has zero entries with positive gradient (projected to 0) and
    with negative gradient (kept), so both branches of the projection count."""
    _, _, gG, gF = ref
    x = np.concatenate([G.ravel(), F.ravel()])
    g = np.concatenate([gG.ravel(), gF.ravel()])
    assert np.any((x == 0) & (g > 0)) and np.any((x == 0) & (g < 0)) and np.any(x > 0)


def _assert_parts(parts, ref):
    PG, PF, gG, gF = ref
    scale = max(np.abs(gG).max(), np.abs(gF).max())
    np.testing.assert_allclose(parts[0], PG, rtol=1e-8, atol=1e-9 * scale)
    np.testing.assert_allclose(parts[1], PF, rtol=1e-8, atol=1e-9 * scale)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plain_parts_match_central_differences(seed):
    X, G, F = _case(seed)
    parts = nenmf.initial_pg_parts_plain(X, G, F)
    ref = _reference_plain(X, G, F)
    _both_branches(G, F, ref)
    _assert_parts(parts, ref)
    pg = nenmf.initial_pg_plain(X, G, F)
    assert pg == pytest.approx(np.sqrt(np.sum(ref[0] ** 2) + np.sum(ref[1] ** 2)), rel=1e-9)


@pytest.mark.parametrize("seed", [3, 4])
def test_compressed_parts_match_central_differences(seed):
    L, R, XL, XR, G, F = _compressed_case(seed)
    parts = nenmf.initial_pg_parts_compressed(L, R, XL, XR, G, F)
    ref = _reference_compressed(L, R, XL, XR, G, F)
    _both_branches(G, F, ref)
    _assert_parts(parts, ref)
    pg = nenmf.initial_pg_compressed(L, R, XL, XR, G, F)
    assert pg == pytest.approx(np.sqrt(np.sum(ref[0] ** 2) + np.sum(ref[1] ** 2)), rel=1e-9)


def test_eps_of_a_run_is_tol_times_the_pinned_norm():
    X, G, F = _case(5)
    PG, PF, _, _ = _reference_plain(X, G, F)
    _, _, info = nenmf.nenmf_plain(X, G, F, max_outer=1, max_inner=3, tol=1e-3)
    assert info["eps"] == pytest.approx(1e-3 * np.sqrt(np.sum(PG ** 2) + np.sum(PF ** 2)), rel=1e-9)


@pytest.mark.parametrize("mutation", [
    lambda F, g: g,                                          # unprojected gradient
    lambda F, g: np.where(F > 0.0, g, np.maximum(g, 0.0)),   # projection on the wrong side
])
def test_planted_projection_mistakes_are_caught(monkeypatch, mutation):
    monkeypatch.setattr(nenmf, "projected_gradient", mutation)
    for seed in (0, 1, 2):
        X, G, F = _case(seed)
        with pytest.raises(AssertionError):
            _assert_parts(nenmf.initial_pg_parts_plain(X, G, F), _reference_plain(X, G, F))
    L, R, XL, XR, G, F = _compressed_case(3)
    with pytest.raises(AssertionError):
        _assert_parts(nenmf.initial_pg_parts_compressed(L, R, XL, XR, G, F),
                      _reference_compressed(L, R, XL, XR, G, F))
