"""GPU parity of the float64 twins (nmf_compress_f64, nenmf_solve_f64) against the FP64 oracle.

Both sides compute in float64 (unit roundoff u = 2^-53 ~ 1.1e-16) from the
same inputs. They differ in summation order (LAPACK/BLAS against the
kernels' sequential loops) and in the QR method (Householder with a sign
fix against three CholeskyQR passes), so the bars are rounding bars:
 * compression: the CholeskyQR basis differs from the Householder one by
   ~u cond(Y) per orthonormalisation; the noisy low-rank inputs here keep
   cond(Y) below ~1e4, so 1e-9 of the largest entry leaves a margin of
   ~1e3; orthonormality 1e-12; X_L, X_R against the products of the
   returned bases 1e-13 (products of length <= 500 in float64);
 * exactly rank-p X with nu > p (rank-deficient sketches, shifted first
   pass): only the span is defined, so the projectors L^T L X and X R R^T
   must reproduce X to 1e-12;
 * solve with a fixed number of iterations (tol = 0): T K projected
   gradient steps, each non-expansive up to the momentum factor (1 + beta
   < 2), from u-level differences per step: 1e-9 relative (Frobenius) at
   T K <= 100;
 * with the stop test: the same inner iteration counts (the squared
   projected-gradient norms sit far from eps^2 relative to u), and the
   results to 1e-8.
"""

import numpy as np
import pytest

import synth
from oracle import adjoint, nenmf, philox, subspace

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _np(t):
    return t.detach().cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,m,nu,q", [(300, 257, 12, 2), (257, 300, 9, 1), (500, 400, 10, 4), (120, 100, 20, 0)])
def test_compress_f64_matches_oracle(nmf, n, m, nu, q):
    X, _, _ = synth.lowrank_data(n, m, 5, seed=n + q, snr_db=30.0)
    OmL, OmR = synth.gaussian_sketches(n, m, nu, seed=3)
    L, R, XL, XR = (_np(a) for a in nmf.compress_f64(_t(X), nu, q, omega_L=_t(OmL), omega_R=_t(OmR)))
    Lo, Ro, XLo, XRo = subspace.compress(X, nu, q, OmL, OmR)
    np.testing.assert_allclose(L @ L.T, np.eye(nu), atol=1e-12)
    np.testing.assert_allclose(R.T @ R, np.eye(nu), atol=1e-12)
    errs = (np.abs(L - Lo).max() / np.abs(Lo).max(), np.abs(R - Ro).max() / np.abs(Ro).max())
    print("basis errors", errs)
    assert max(errs) <= 1e-9
    assert _rel(XL, L @ X) <= 1e-13 and _rel(XR, X @ R) <= 1e-13
    assert _rel(XL, XLo) <= 1e-9 and _rel(XR, XRo) <= 1e-9


def test_compress_f64_exact_low_rank(nmf):
    n, m, p, nu, q = 333, 222, 6, 10, 2
    X, _, _ = synth.lowrank_data(n, m, p, seed=3)
    OmL, OmR = synth.gaussian_sketches(n, m, nu, seed=11)
    L, R, XL, XR = (_np(a) for a in nmf.compress_f64(_t(X), nu, q, omega_L=_t(OmL), omega_R=_t(OmR)))
    np.testing.assert_allclose(L @ L.T, np.eye(nu), atol=1e-10)
    np.testing.assert_allclose(R.T @ R, np.eye(nu), atol=1e-10)
    nx = np.linalg.norm(X)
    assert np.linalg.norm(X - L.T @ (L @ X)) <= 1e-12 * nx
    assert np.linalg.norm(X - (X @ R) @ R.T) <= 1e-12 * nx


def test_compress_f64_seeded_draw(nmf):
    # NULL sketches: the library's float32 draw (nmf_gaussian_sketch, streams
    # 0 and 1) widened to float64, so the result equals the call given those
    # sketches, bit for bit. (oracle.philox reproduces the draw only to
    # float32 rounding of its logarithm and sine, which the weaker basis
    # directions amplify; the oracle parity of the bases is the test above.)
    n, m, nu, q, seed = 240, 180, 8, 1, 7
    X, _, _ = synth.lowrank_data(n, m, 4, seed=1, snr_db=30.0)
    a = nmf.compress_f64(_t(X), nu, q, seed=seed)
    OmL = nmf.gaussian_sketch(m, nu, seed, 0).double()
    OmR = nmf.gaussian_sketch(nu, n, seed, 1).double()
    b = nmf.compress_f64(_t(X), nu, q, omega_L=OmL, omega_R=OmR)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(_np(x), _np(y))
    # and the draw is the documented one to float32 rounding
    PL, PR = philox.sketches(n, m, nu, seed)
    np.testing.assert_allclose(_np(OmL), PL, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(_np(OmR), PR, rtol=1e-5, atol=1e-5)


def _problem(nmf, mode, n, m, p, nu, q, seed):
    X, _, _ = synth.lowrank_data(n, m, p, seed=seed, snr_db=30.0)
    if mode == "plain":
        return X, nmf.plain_problem_f64(_t(X), p), None
    OmL, OmR = synth.gaussian_sketches(n, m, nu, seed=seed + 1)
    L, R, XL, XR = subspace.compress(X, nu, q, OmL, OmR)
    return X, nmf.compressed_problem_f64(_t(L), _t(R), _t(XL), _t(XR), p), (L, R, XL, XR)


def _oracle(mode, X, comp, G0, F0, T, K, **kw):
    if mode == "plain":
        return nenmf.nenmf_plain(X, G0, F0, T, K, **kw)
    return nenmf.nenmf_compressed(*comp, G0, F0, T, K, **kw)


@pytest.mark.parametrize("mode", ["plain", "compressed"])
@pytest.mark.parametrize("restart", [False, True])
def test_solve_f64_fixed_iterations(nmf, mode, restart):
    n, m, p, nu, q, T, K = 200, 150, 5, 10, 2, 10, 10
    X, pr, comp = _problem(nmf, mode, n, m, p, nu, q, seed=4)
    G0, F0 = synth.initial_factors(n, m, p, seed=5)
    G, F = _t(G0), _t(F0)
    st = nmf.read_stats(nmf.solve_f64(pr, G, F, T, K, restart=restart))
    Go, Fo, _ = _oracle(mode, X, comp, G0, F0, T, K, restart=restart)
    print(mode, restart, _rel(_np(G), Go), _rel(_np(F), Fo))
    assert _rel(_np(G), Go) <= 1e-9 and _rel(_np(F), Fo) <= 1e-9
    assert st.status == 0 and st.outer_done == T
    assert list(st.total_inner) == [T * K, T * K]


@pytest.mark.parametrize("mode", ["plain", "compressed"])
@pytest.mark.parametrize("tol", [1e-3, 1e-5])
def test_solve_f64_stop_test(nmf, mode, tol):
    n, m, p, nu, q, T, K = 180, 160, 4, 9, 2, 15, 60
    X, pr, comp = _problem(nmf, mode, n, m, p, nu, q, seed=6)
    G0, F0 = synth.initial_factors(n, m, p, seed=7)
    G, F = _t(G0), _t(F0)
    st = nmf.read_stats(nmf.solve_f64(pr, G, F, T, K, tol=tol))
    Go, Fo, info = _oracle(mode, X, comp, G0, F0, T, K, tol=tol)
    kG = sum(k for k, _ in info["inner"])
    kF = sum(k for _, k in info["inner"])
    assert list(st.total_inner) == [kG, kF]
    assert list(st.last_inner) == list(info["inner"][-1])
    assert abs(st.eps - info["eps"]) <= 1e-12 * info["eps"]
    assert _rel(_np(G), Go) <= 1e-8 and _rel(_np(F), Fo) <= 1e-8


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_config_c1_plain_fp64(nmf, seed):
    # plain NeNMF in float64: n = 500, m = 400, p = 5, X = G0 F0 exactly,
    # initial factors Uniform[0, 1], 50 outer x <= 10 inner, tol 1e-6
    n, m, p, T, K = 500, 400, 5, 50, 10
    X, _, _ = synth.lowrank_data(n, m, p, seed=seed)
    G0, F0 = synth.initial_factors(n, m, p, seed=100 + seed)
    G, F = _t(G0), _t(F0)
    st = nmf.read_stats(nmf.solve_f64(nmf.plain_problem_f64(_t(X), p), G, F, T, K, tol=1e-6))
    Go, Fo, info = nenmf.nenmf_plain(X, G0, F0, T, K, tol=1e-6)
    rre = np.linalg.norm(X - _np(G) @ _np(F)) / np.linalg.norm(X)
    rre_o = np.linalg.norm(X - Go @ Fo) / np.linalg.norm(X)
    print(seed, rre, rre_o)
    assert abs(rre - rre_o) <= 1e-9 * max(rre_o, 1e-12) + 1e-13
    assert list(st.total_inner) == [sum(k for k, _ in info["inner"]), sum(k for _, k in info["inner"])]


def test_zero_outer_iterations_f64(nmf):
    n, m, p = 60, 50, 3
    X, _, _ = synth.lowrank_data(n, m, p, seed=2)
    G0, F0 = synth.initial_factors(n, m, p, seed=3)
    G, F = _t(G0), _t(F0)
    st = nmf.read_stats(nmf.solve_f64(nmf.plain_problem_f64(_t(X), p), G, F, 0, 5))
    np.testing.assert_array_equal(_np(G), G0)
    np.testing.assert_array_equal(_np(F), F0)
    assert st.outer_done == 0


def test_f64_twin_is_deterministic(nmf):
    n, m, p, nu, q = 150, 120, 4, 8, 1
    X, pr, _ = _problem(nmf, "compressed", n, m, p, nu, q, seed=9)
    G0, F0 = synth.initial_factors(n, m, p, seed=10)
    out = []
    for _ in range(2):
        G, F = _t(G0), _t(F0)
        nmf.solve_f64(pr, G, F, 5, 10, tol=1e-4, restart=True)
        out.append((_np(G), _np(F)))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def _backward_case(nmf, n, m, p, nu, q, seed):
    X, _, _ = synth.lowrank_data(n, m, p, seed=seed, snr_db=20.0)
    G0, F0 = synth.initial_factors(n, m, p, seed=seed + 1)
    OmL, OmR = synth.gaussian_sketches(n, m, nu, seed=seed + 2)
    L, R, _, _ = subspace.compress(X, nu, q, OmL, OmR)
    return X, L, R, G0, F0


def _gpu_loss_and_gradient(nmf, X, L, R, G0, F0, T, K):
    # loss ||X - G_T F_T||^2 with X_L = L X, X_R = X R (L, R fixed), every step on the GPU in float64
    pr = nmf.compressed_problem_f64(_t(L), _t(R), _t(L @ X), _t(X @ R), G0.shape[1])
    G, F = _t(G0), _t(F0)
    nmf.solve_f64(pr, G, F, T, K)
    Gd, Fd = _np(G), _np(F)
    E = X - Gd @ Fd
    dXL, dXR, dG0, dF0, dX = nmf.backward_f64(pr, _t(G0), _t(F0), _t(-2.0 * E @ Fd.T), _t(-2.0 * Gd.T @ E), T, K,
                                               want_dX=True)
    return float(np.sum(E * E)), 2.0 * E + _np(dX), _np(dG0), _np(dF0)


@pytest.mark.parametrize("T,K", [(1, 1), (4, 5), (2, 10)])
def test_backward_f64_matches_oracle(nmf, T, K):
    n, m, p, nu, q = 64, 48, 4, 8, 2
    X, L, R, G0, F0 = _backward_case(nmf, n, m, p, nu, q, seed=21)
    loss, dX, dG0, dF0 = _gpu_loss_and_gradient(nmf, X, L, R, G0, F0, T, K)
    lo, dXo, dG0o, dF0o = adjoint.loss_and_gradient(X, L, R, G0, F0, T, K)
    assert abs(loss - lo) <= 1e-12 * lo
    for a, b in ((dX, dXo), (dG0, dG0o), (dF0, dF0o)):
        assert _rel(a, b) <= 1e-10, _rel(a, b)


def test_backward_f64_central_differences(nmf):
    # the GPU float64 gradient against central differences of the GPU float64
    # forward (h = 1e-6: truncation ~h^2, rounding ~1e-16 / h), along random
    # directions that keep every projection's sign
    n, m, p, nu, q, T, K = 64, 48, 4, 8, 2, 4, 5
    X, L, R, G0, F0 = _backward_case(nmf, n, m, p, nu, q, seed=21)
    loss, dX, dG0, dF0 = _gpu_loss_and_gradient(nmf, X, L, R, G0, F0, T, K)
    base = adjoint.projection_signs(X, L, R, G0, F0, T, K)
    h = 1e-6
    checked = 0
    for d in synth.random_directions((n * m + n * p + p * m,), 12, seed=5):
        dXd = d[:n * m].reshape(n, m)
        dGd = d[n * m:n * m + n * p].reshape(n, p)
        dFd = d[n * m + n * p:].reshape(p, m)
        if not all(all(np.array_equal(a, b) for a, b in zip(
                base, adjoint.projection_signs(X + s * h * dXd, L, R, G0 + s * h * dGd, F0 + s * h * dFd, T, K)))
                   for s in (1, -1)):
            continue
        lp = _gpu_loss_and_gradient(nmf, X + h * dXd, L, R, G0 + h * dGd, F0 + h * dFd, T, K)[0]
        lm = _gpu_loss_and_gradient(nmf, X - h * dXd, L, R, G0 - h * dGd, F0 - h * dFd, T, K)[0]
        fd = (lp - lm) / (2 * h)
        an = float(np.sum(dX * dXd) + np.sum(dG0 * dGd) + np.sum(dF0 * dFd))
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-8 * loss), (an, fd)
        checked += 1
    assert checked >= 8


def test_full_sketch_reduces_to_plain_f64(nmf):
    # nu = n = m: L and R are square orthogonal, so G_L^T G_L = G^T G,
    # G_L^T X_L = G^T X (and likewise for F): the compressed trajectory is the
    # plain one up to float64 rounding
    n = m = 64
    p, T, K = 3, 6, 10
    X, _, _ = synth.lowrank_data(n, m, p, seed=8, snr_db=30.0)
    OmL, OmR = synth.gaussian_sketches(n, m, n, seed=9)
    L, R, XL, XR = nmf.compress_f64(_t(X), n, 0, omega_L=_t(OmL), omega_R=_t(OmR))
    np.testing.assert_allclose(_np(L) @ _np(L).T, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(_np(R).T @ _np(R), np.eye(n), atol=1e-12)
    G0, F0 = synth.initial_factors(n, m, p, seed=10)
    Gc, Fc = _t(G0), _t(F0)
    nmf.solve_f64(nmf.compressed_problem_f64(L, R, XL, XR, p), Gc, Fc, T, K)
    Gp, Fp = _t(G0), _t(F0)
    nmf.solve_f64(nmf.plain_problem_f64(_t(X), p), Gp, Fp, T, K)
    assert _rel(_np(Gc), _np(Gp)) <= 1e-10 and _rel(_np(Fc), _np(Fp)) <= 1e-10


@pytest.mark.parametrize("n,m,p,nu", [(33, 17, 1, 1), (80, 90, 32, 40), (70, 50, 2, 50)])
def test_solve_f64_rank_limits(nmf, n, m, p, nu):
    X, pr, comp = _problem(nmf, "compressed", n, m, p, nu, 1, seed=n)
    G0, F0 = synth.initial_factors(n, m, p, seed=m)
    G, F = _t(G0), _t(F0)
    st = nmf.read_stats(nmf.solve_f64(pr, G, F, 5, 8, tol=1e-4))
    Go, Fo, info = _oracle("compressed", X, comp, G0, F0, 5, 8, tol=1e-4)
    assert st.status == 0
    assert list(st.total_inner) == [sum(k for k, _ in info["inner"]), sum(k for _, k in info["inner"])]
    assert _rel(_np(G), Go) <= 1e-8 and _rel(_np(F), Fo) <= 1e-8
