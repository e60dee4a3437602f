"""GPU parity of nenmf_backward (reverse-mode derivative of the compressed solve) against the FP64 oracle.

Both sides start from the same float32 X, L, R, X_L, X_R, G0, F0. The GPU
forward is nenmf_solve with the stop test off and snapshots on; the
oracle's is oracle.adjoint.compressed_forward. Each side forms the
cotangents of the loss ||X - G_T F_T||_F^2 from its own (G_T, F_T) and runs
its backward; compared are dX_L, dX_R, dG0, dF0 and the total dX
(2 (X - G_T F_T) + L^T dX_L + dX_R R^T), in relative Frobenius norm.

Tolerance: the GPU computes in float32 (unit roundoff u = 2^-24); every one
of the 2 T K adjoint steps is a p-term matrix-vector product applied to a
cotangent of unit scale, so the rounding it adds is ~p u relative, and the
steps compose (each is non-expansive up to the projection mask) to a bound of
~2 T K p u: at most 4e-5 for the small cases, 2e-4 for the 4096 x 4096 one.
The forward trajectories themselves differ by float32 rounding, which moves
a projection's activity only where |z| sits within ~1e-6 of 0; the tests
take 2e-4 (small cases) and 1e-3 (the 4096 x 4096 case, 13 million z's).
"""

import numpy as np
import pytest

import synth
from oracle import adjoint, subspace

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _check(gpu, ora, tol):
    # Each gradient's error against tol times its own norm, floored at 1% of
    # the whole gradient's norm: a gradient that nearly vanishes (dX_L at
    # p = nu = 1) carries float32 rounding of the terms that cancel in it.
    scale = np.sqrt(sum(np.sum(b * b) for b in ora))
    errs = {}
    for name, a, b in zip(("dXL", "dXR", "dG0", "dF0", "dX"), gpu, ora):
        err = np.linalg.norm(a - b)
        errs[name] = err / max(np.linalg.norm(b), 1e-300)
        assert err <= tol * (np.linalg.norm(b) + 1e-2 * scale), (name, errs)
    print(errs)


def _inputs(n, m, p, nu, q, seed):
    X, _, _ = synth.lowrank_data(n, m, p, seed=seed, snr_db=20.0, dtype=np.float32)
    G0, F0 = synth.initial_factors(n, m, p, seed=seed + 1)
    OmL, OmR = synth.gaussian_sketches(n, m, nu, seed=seed + 2)
    L, R, XL, XR = (a.astype(np.float32) for a in subspace.compress(X.astype(np.float64), nu, q, OmL, OmR))
    return X, L, R, XL, XR, G0.astype(np.float32), F0.astype(np.float32)


def _gpu(nmf, X, L, R, XL, XR, G0, F0, p, T, K):
    import torch
    n, m = X.shape
    prob = nmf.compressed_problem(_t(L), _t(R), _t(XL), _t(XR), p)
    G, F = _t(G0), _t(F0)
    rec = nmf.SolveRecord(G=torch.empty((T, n, p), device="cuda"), F=torch.empty((T, p, m), device="cuda"))
    if T > 0:
        nmf.solve(prob, G, F, T, K, tol=0.0, record=rec)
    Gd, Fd = _np(G), _np(F)
    E = X.astype(np.float64) - Gd @ Fd
    dXL, dXR, dG0, dF0, dX = nmf.backward(prob, _t(G0), _t(F0), rec, _t(-2.0 * E @ Fd.T), _t(-2.0 * Gd.T @ E),
                                          T, K, want_dX=True)
    return _np(dXL), _np(dXR), _np(dG0), _np(dF0), 2.0 * E + _np(dX)


def _oracle(X, L, R, XL, XR, G0, F0, T, K):
    G, F, tape = adjoint.compressed_forward(L, R, XL, XR, G0, F0, T, K)
    E = X.astype(np.float64) - G @ F
    dXL, dXR, dG0, dF0 = adjoint.compressed_backward(L, R, XL, XR, tape, -2.0 * E @ F.T, -2.0 * G.T @ E)
    Ld, Rd = L.astype(np.float64), R.astype(np.float64)
    return dXL, dXR, dG0, dF0, 2.0 * E + Ld.T @ dXL + dXR @ Rd.T


@pytest.mark.parametrize("n,m,p,nu,q,T,K", [
    (64, 48, 4, 8, 2, 3, 5),        # the finite-difference configuration of the oracle's pins
    (200, 150, 5, 10, 2, 4, 5),
    (300, 257, 12, 20, 1, 3, 10),
    (130, 90, 1, 1, 1, 2, 3),
    (96, 80, 16, 26, 2, 2, 1),
    (150, 140, 20, 30, 1, 2, 4),
])
def test_backward_matches_oracle(nmf, n, m, p, nu, q, T, K):
    args = _inputs(n, m, p, nu, q, seed=n + p)
    _check(_gpu(nmf, *args, p, T, K), _oracle(*args, T, K), 2e-4)


def test_backward_full_size(nmf):
    # n = m = 4096, p = 16, nu = 26, q = 2; 20 outer x 5 inner
    args = _inputs(4096, 4096, 16, 26, 2, seed=4)
    _check(_gpu(nmf, *args, 16, 20, 5), _oracle(*args, 20, 5), 1e-3)


def test_zero_outer_iterations(nmf):
    X, L, R, XL, XR, G0, F0 = _inputs(50, 40, 3, 6, 1, seed=2)
    import torch
    prob = nmf.compressed_problem(_t(L), _t(R), _t(XL), _t(XR), 3)
    dG, dF = _t(np.ones((50, 3))), _t(np.full((3, 40), 2.0))
    rec = nmf.SolveRecord(G=None, F=None)
    dXL, dXR, dG0, dF0, _ = nmf.backward(prob, _t(G0), _t(F0), rec, dG, dF, 0, 5)
    torch.cuda.synchronize()
    assert float(dXL.abs().max()) == 0.0 and float(dXR.abs().max()) == 0.0
    np.testing.assert_array_equal(_np(dG0), np.ones((50, 3)))
    np.testing.assert_array_equal(_np(dF0), np.full((3, 40), 2.0))


def test_backward_is_deterministic(nmf):
    args = _inputs(180, 120, 6, 12, 1, seed=7)
    a = _gpu(nmf, *args, 6, 3, 5)
    b = _gpu(nmf, *args, 6, 3, 5)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
