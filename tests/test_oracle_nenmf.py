"""Pins for the oracle's outer loops: plain NeNMF (eq. 2-3) and compressed NeNMF (Alg. 1).

* nu = n = m makes L and R square orthogonal, so the compressed Gram and
  right-hand-side matrices equal the plain ones and both trajectories agree;
* with exactly solved subproblems NeNMF is block coordinate descent, so the
  objective never increases;
* exactly low-rank X is recovered (RRE -> 0) by both variants;
* the RRE of eq. (4) against the expansion
  ||X - GF||^2 = ||X||^2 - 2 <G^T X, F> + <G^T G, F F^T> and a loop;
* the relative stopping threshold.
"""

import numpy as np

import synth
from oracle import metrics, nenmf, subspace


def test_compressed_equals_plain_when_nothing_is_compressed():
    n = m = 24
    p = 3
    X, _, _ = synth.lowrank_data(n, m, p, seed=1, snr_db=25.0)
    G0, F0 = synth.initial_factors(n, m, p, seed=2)
    Om_L, Om_R = synth.gaussian_sketches(n, m, n, seed=3)
    L, R, XL, XR = subspace.compress(X, n, 1, Om_L, Om_R)
    Gp, Fp, ip = nenmf.nenmf_plain(X, G0, F0, max_outer=15, max_inner=10, tol=1e-6, record=True)
    Gc, Fc, ic = nenmf.nenmf_compressed(L, R, XL, XR, G0, F0, max_outer=15, max_inner=10, tol=1e-6, record=True)
    np.testing.assert_allclose(Gc, Gp, rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(Fc, Fp, rtol=1e-8, atol=1e-10)
    assert ip["inner"] == ic["inner"]
    assert abs(ip["eps"] - ic["eps"]) <= 1e-9 * ip["eps"]


def test_exact_subproblems_never_increase_objective():
    X, _, _ = synth.lowrank_data(40, 30, 4, seed=5, snr_db=15.0)
    G, F = synth.initial_factors(40, 30, 4, seed=6)
    prev = metrics.rre(X, G, F)
    for _ in range(8):
        G, F, _ = nenmf.nenmf_plain(X, G, F, max_outer=1, max_inner=3000)
        cur = metrics.rre(X, G, F)
        assert cur <= prev * (1 + 1e-10)
        prev = cur


def test_recovers_exact_low_rank():
    n, m, p = 50, 40, 3
    X, _, _ = synth.lowrank_data(n, m, p, seed=8)
    G0, F0 = synth.initial_factors(n, m, p, seed=9)
    _, _, info = nenmf.nenmf_plain(X, G0, F0, max_outer=300, max_inner=20, record=True)
    r = metrics.rre_history(X, info["history"])
    assert r[-1] < 1e-3 and r[-1] < 0.05 * r[0]
    Om_L, Om_R = synth.gaussian_sketches(n, m, p + 4, seed=10)
    L, R, XL, XR = subspace.compress(X, p + 4, 2, Om_L, Om_R)
    _, _, infc = nenmf.nenmf_compressed(L, R, XL, XR, G0, F0, max_outer=300, max_inner=20, record=True)
    rc = metrics.rre_history(X, infc["history"])
    assert rc[-1] < 1e-3 and rc[-1] < 0.05 * rc[0]


def test_rre_expansion_and_loop():
    rng = np.random.default_rng(0)
    X, G, F = rng.random((7, 5)), rng.random((7, 2)), rng.random((2, 5))
    expanded = np.sum(X * X) - 2 * np.sum((G.T @ X) * F) + np.sum((G.T @ G) * (F @ F.T))
    loop = 0.0
    for i in range(7):
        for j in range(5):
            loop += (X[i, j] - sum(G[i, k] * F[k, j] for k in range(2))) ** 2
    nx = np.sqrt(sum(X[i, j] ** 2 for i in range(7) for j in range(5)))
    assert abs(metrics.rre(X, G, F) - np.sqrt(loop) / nx) < 1e-14
    assert abs(metrics.rre(X, G, F) - np.sqrt(expanded) / nx) < 1e-13


def test_relative_threshold_and_early_stop():
    X, _, _ = synth.lowrank_data(30, 25, 3, seed=11)
    G0, F0 = synth.initial_factors(30, 25, 3, seed=12)
    pg0 = nenmf.initial_pg_plain(X, G0, F0)
    _, _, info = nenmf.nenmf_plain(X, G0, F0, max_outer=20, max_inner=200, tol=1e-4)
    assert abs(info["eps"] - 1e-4 * pg0) <= 1e-12 * pg0
    assert any(kg < 200 or kf < 200 for kg, kf in info["inner"])
    _, _, info_abs = nenmf.nenmf_plain(X, G0, F0, max_outer=1, max_inner=5, tol=0.5, tol_mode="abs")
    assert info_abs["eps"] == 0.5
    _, _, info_off = nenmf.nenmf_plain(X, G0, F0, max_outer=2, max_inner=7, tol=0.0)
    assert info_off["eps"] is None and info_off["inner"] == [(7, 7), (7, 7)]


def test_factors_stay_nonnegative_under_semi_nmf_compression():
    # X_L, X_R, G_L and F_R may be negative (Sec. 3); only G and F are projected.
    X, _, _ = synth.lowrank_data(60, 50, 4, seed=13, snr_db=30.0)
    G0, F0 = synth.initial_factors(60, 50, 4, seed=14)
    Om_L, Om_R = synth.gaussian_sketches(60, 50, 9, seed=15)
    L, R, XL, XR = subspace.compress(X, 9, 2, Om_L, Om_R)
    assert XL.min() < 0 or XR.min() < 0
    G, F, _ = nenmf.nenmf_compressed(L, R, XL, XR, G0, F0, max_outer=10, max_inner=10)
    assert G.min() >= 0 and F.min() >= 0
