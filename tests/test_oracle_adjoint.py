"""Pins of the oracle's reverse-mode derivative (oracle/adjoint.py) by central finite differences.

Directional derivatives <grad, d> are compared with (f(x + h d) - f(x - h d)) / 2h
at h = 1e-6 in float64 (truncation ~h^2, rounding ~1e-16 / h, both far below
the 1e-6 relative bound). The map is smooth only where no projection
max(0, z) switches sign inside [x - h d, x + h d]: such directions are
skipped (the signs of every z_k are compared at x and x +- h d), and most
directions must remain.
"""

import numpy as np
import pytest

import synth
from oracle import adjoint, subspace
from oracle.nenmf import lipschitz_constant


def _central(f, h=1e-6):
    return (f(h) - f(-h)) / (2 * h)


def test_lambda_max_derivative():
    rng = np.random.default_rng(4)
    W = rng.random((5, 9))
    H = W @ W.T
    E = rng.standard_normal((5, 5))
    E = E + E.T
    v = adjoint.top_eigenvector(H)
    fd = _central(lambda t: lipschitz_constant(H + t * E))
    assert fd == pytest.approx(float(v @ E @ v), rel=1e-7)


@pytest.mark.parametrize("K", [1, 2, 5, 12])
def test_inner_loop_adjoint(K):
    rng = np.random.default_rng(K)
    p, N = 4, 30
    W = rng.random((p, 7))
    H = W @ W.T
    B = W @ rng.random((7, N))
    Y0 = rng.random((p, N))
    C = rng.standard_normal((p, N))          # a fixed linear functional of the output
    f = lambda H_, B_, Y_: float(np.sum(C * adjoint.nnls_forward(H_, B_, Y_, K)[0]))
    out, tape = adjoint.nnls_forward(H, B, Y0, K)
    dY0, dH, dB = adjoint.nnls_adjoint(H, B, tape, C)
    signs = [z > 0 for z in tape["z"]]
    checked = 0
    for i in range(12):
        dYd = rng.standard_normal((p, N))
        dBd = rng.standard_normal((p, N))
        E = rng.standard_normal((p, p))
        E = E + E.T
        h = 1e-6
        same = all(np.array_equal(s, z > 0) for sgn in (1, -1)
                   for s, z in zip(signs, adjoint.nnls_forward(H + sgn * h * E, B + sgn * h * dBd,
                                                               Y0 + sgn * h * dYd, K)[1]["z"]))
        if not same:
            continue
        fd = _central(lambda t: f(H + t * E, B + t * dBd, Y0 + t * dYd), h)
        an = float(np.sum(dY0 * dYd) + np.sum(dB * dBd) + np.sum(dH * E))
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9), (i, an, fd)
        checked += 1
    assert checked >= 9


def _problem(n, m, p, nu, q, seed):
    X, _, _ = synth.lowrank_data(n, m, p, seed=seed, snr_db=20.0)
    G0, F0 = synth.initial_factors(n, m, p, seed=seed + 1)
    OmL, OmR = synth.gaussian_sketches(n, m, nu, seed=seed + 2)
    L, R, _, _ = subspace.compress(X, nu, q, OmL, OmR)
    return X, L, R, G0, F0


@pytest.mark.parametrize("T,K", [(1, 1), (4, 5), (2, 10)])
def test_unrolled_compressed_nenmf_gradient(T, K):
    # The small differentiated configuration: n = 64, m = 48, p = 4, 20 directions.
    n, m, p, nu, q = 64, 48, 4, 8, 2
    X, L, R, G0, F0 = _problem(n, m, p, nu, q, seed=21)
    loss, dX, dG0, dF0 = adjoint.loss_and_gradient(X, L, R, G0, F0, T, K)
    base = adjoint.projection_signs(X, L, R, G0, F0, T, K)
    dirs = synth.random_directions((n * m + n * p + p * m,), 20, seed=5)
    h = 1e-6
    checked = 0
    for d in dirs:
        dXd = d[:n * m].reshape(n, m)
        dGd = d[n * m:n * m + n * p].reshape(n, p)
        dFd = d[n * m + n * p:].reshape(p, m)
        at = lambda t: (X + t * dXd, G0 + t * dGd, F0 + t * dFd)
        smooth = all(all(np.array_equal(a, b) for a, b in zip(base, adjoint.projection_signs(*at(s * h)[:1], L, R,
                                                                                              *at(s * h)[1:], T, K)))
                     for s in (1, -1))
        if not smooth:
            continue

        def f(t):
            Xt, Gt, Ft = at(t)
            return adjoint.loss_and_gradient(Xt, L, R, Gt, Ft, T, K)[0]

        fd = _central(f, h)
        an = float(np.sum(dX * dXd) + np.sum(dG0 * dGd) + np.sum(dF0 * dFd))
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-8 * abs(loss)), (an, fd)
        checked += 1
    assert checked >= 15


def test_gradient_of_a_fixed_point():
    # With G0, F0 the exact nonnegative factors of a noise-free X and nu = n = m
    # (L, R orthogonal), every inner step maps the factors to themselves and
    # the loss is 0: its gradient vanishes.
    n, m, p = 12, 10, 2
    X, G0, F0 = synth.lowrank_data(n, m, p, seed=3)
    L = np.linalg.qr(np.random.default_rng(0).standard_normal((n, n)))[0].T
    R = np.linalg.qr(np.random.default_rng(1).standard_normal((m, m)))[0]
    loss, dX, dG0, dF0 = adjoint.loss_and_gradient(X, L, R, G0, F0, 3, 4)
    assert loss < 1e-20
    assert np.abs(dX).max() < 1e-8 and np.abs(dG0).max() < 1e-8 and np.abs(dF0).max() < 1e-8
