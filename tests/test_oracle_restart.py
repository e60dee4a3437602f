"""Pins of the optional adaptive restart of the inner loop (oracle.nenmf.nesterov_nnls(restart=True)).

Restart acts only where a column's objective rises, so:
  * on a problem whose plain trajectory never raises any column's objective,
    restart changes nothing (bit for bit);
  * right after a restart the column takes a plain projected-gradient step
    (momentum weight beta_0 = 0), which cannot raise the objective (descent
    lemma of the projected gradient step with step 1/L_c from a feasible point);
  * with many iterations the restarted loop still reaches the brute-force
    NNLS solution.
"""

import numpy as np
import pytest

from oracle import bruteforce, nenmf


def _ill_conditioned(p, N, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((p, p)))[0]
    H = Q @ np.diag(np.geomspace(1.0, 1.0 / cond, p)) @ Q.T
    B = H @ rng.standard_normal((p, N)) + 0.05 * rng.standard_normal((p, N))
    return H, B, np.abs(rng.standard_normal((p, N)))


def test_no_rise_means_no_change():
    # the first five iterations of this problem raise no column objective
    rng = np.random.default_rng(1)
    W = rng.random((3, 40)) + 2.0
    H = W @ W.T / 40
    B = rng.random((3, 25))
    Y0 = rng.random((3, 25))
    trace = []
    F_r, k_r, _ = nenmf.nesterov_nnls(H, B, Y0, 5, restart=True, trace=trace)
    assert not any(mask.any() for _, mask in trace)
    F_p, k_p, _ = nenmf.nesterov_nnls(H, B, Y0, 5)
    np.testing.assert_array_equal(F_r, F_p)


def test_restart_happens_and_is_followed_by_descent():
    H, B, Y0 = _ill_conditioned(6, 40, seed=3)
    trace = []
    nenmf.nesterov_nnls(H, B, Y0, 60, restart=True, trace=trace)
    objs = np.array([o for o, _ in trace])
    masks = np.array([m for _, m in trace])
    assert masks.sum() > 0                      # the momentum overshoots on this problem
    k_idx, col = np.nonzero(masks[:-1])
    # after restarting at k the step k+1 is a projected gradient step from F_k
    assert np.all(objs[k_idx + 1, col] <= objs[k_idx, col] + 1e-12 * np.abs(objs[k_idx, col]))


def test_plain_run_rises_where_restart_acts():
    # the same problem without restart: some column objective rises somewhere
    H, B, Y0 = _ill_conditioned(6, 40, seed=3)
    Lc = nenmf.lipschitz_constant(H)
    beta = nenmf.extrapolation_weights(60)
    Y, Fp, prev = Y0.copy(), Y0.copy(), None
    rises = 0
    for k in range(60):
        F = np.maximum(0.0, Y - (H @ Y - B) / Lc)
        obj = 0.5 * np.sum(F * (H @ F), axis=0) - np.sum(B * F, axis=0)
        if prev is not None:
            rises += int(np.sum(obj > prev))
        prev = obj
        Y = F + beta[k] * (F - Fp)
        Fp = F
    assert rises > 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_restarted_loop_reaches_bruteforce_nnls(seed):
    H, B, Y0 = _ill_conditioned(4, 8, seed=seed, cond=50.0)
    F, _, _ = nenmf.nesterov_nnls(H, B, Y0, 5000, restart=True)
    for j in range(B.shape[1]):
        ref = bruteforce.nnls_enumerate(H, B[:, j])
        np.testing.assert_allclose(F[:, j], ref, atol=1e-8)
