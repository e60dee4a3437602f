"""GPU parity of nenmf_solve (plain NeNMF, eq. 2-3; compressed NeNMF, Alg. 1) against the FP64 oracle.

Inputs are float32 on both sides (the oracle computes in float64 on the same
float32 values). Compared per outer iteration: the RRE of eq. (4), bound
|RRE_gpu - RRE_oracle| <= 1e-5 for the float32 paths (the target tolerance);
after one outer iteration the factors themselves, entry by entry.

Per-entry bound on the factors after one outer iteration: each inner step
forms an O(p)-term gradient H y - b in float32, so an entry's error is a few
units of 2^-24 times the scale of its column's terms, carried through <= 10
non-expansive projected steps (the extrapolation adds at most a factor 2 per
step to a difference, and the contraction of the step removes most of it):
    |gpu - oracle| <= ftol * (|oracle| + s),
s the root-mean-square of the oracle's factor (an entry held at 0 by the
projection on one side and at a rounding-level positive value on the other
differs by rounding of that scale), ftol = 1e-4 for the float32 paths and
2e-2 where the X products take bfloat16 inputs (relative 2^-9 per input).
"""

import numpy as np
import pytest

from _parity import assert_entrywise
import synth
from oracle import metrics, nenmf, subspace

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _record(nmf, T, n, m, p):
    import torch
    return nmf.SolveRecord(G=torch.empty((T, n, p), device="cuda"), F=torch.empty((T, p, m), device="cuda"),
                           times=torch.zeros(T + 1, dtype=torch.int64, device="cuda"))


def _gpu_rre_history(X, rec):
    Gs, Fs = _np(rec.G), _np(rec.F)
    return metrics.rre_history(X, list(zip(Gs, Fs)))


def _inputs(n, m, p, seed, snr=30.0):
    X, _, _ = synth.lowrank_data(n, m, p, seed=seed, snr_db=snr, dtype=np.float32)
    G0, F0 = synth.initial_factors(n, m, p, seed=seed + 1)
    return X, G0.astype(np.float32), F0.astype(np.float32)


@pytest.mark.parametrize("n,m,p,T,inner,tol", [
    (300, 257, 5, 20, 10, 0.0),
    (500, 400, 5, 50, 10, 1e-6),     # the small plain configuration
    (129, 700, 12, 10, 10, 1e-3),    # early stops happen
    (64, 40, 1, 10, 5, 0.0),
    (200, 300, 32, 5, 10, 0.0),
])
@pytest.mark.parametrize("prec", [0, 1])
def test_plain_solve_matches_oracle(nmf, n, m, p, T, inner, tol, prec):
    # prec 1 rounds X and the factor operands of the two X products to
    # bfloat16 (relative 2^-9): the bfloat16 tolerance 1e-3 applies there.
    X, G0, F0 = _inputs(n, m, p, seed=n + p)
    Xd = X.astype(np.float64)
    G, F = _t(G0), _t(F0)
    rec = _record(nmf, T, n, m, p)
    st = nmf.read_stats(nmf.solve(nmf.plain_problem(_t(X), p, prec), G, F, T, inner, tol=tol, record=rec))
    assert st.status == 0 and st.outer_done == T
    Go, Fo, info = nenmf.nenmf_plain(Xd, G0, F0, T, inner, tol=tol, record=True)
    r_gpu = _gpu_rre_history(Xd, rec)
    r_ora = metrics.rre_history(Xd, info["history"])
    assert np.max(np.abs(r_gpu - r_ora)) <= (1e-5 if prec == 0 else 1e-3), (r_gpu - r_ora)
    if tol > 0:
        assert st.eps == pytest.approx(info["eps"], rel=1e-4 if prec == 0 else 2e-2)
    # after the first outer iteration the factors agree closely
    G1, F1 = info["history"][0]
    ftol = 1e-4 if prec == 0 else 2e-2
    assert_entrywise(_np(rec.G[0]), G1, ftol, "G after one outer iteration")
    assert_entrywise(_np(rec.F[0]), F1, ftol, "F after one outer iteration")
    np.testing.assert_array_equal(_np(G), _np(rec.G[T - 1]))
    np.testing.assert_array_equal(_np(F), _np(rec.F[T - 1]))
    assert (_np(G) >= 0).all() and (_np(F) >= 0).all()


@pytest.mark.parametrize("n,m,p,nu,q,T,inner,tol", [
    (300, 257, 5, 12, 2, 20, 10, 1e-6),
    (640, 384, 10, 20, 4, 30, 10, 0.0),
    (129, 700, 12, 22, 1, 10, 10, 1e-3),
    (100, 90, 1, 1, 1, 10, 5, 0.0),
    (200, 190, 32, 64, 1, 5, 10, 0.0),
])
def test_compressed_solve_matches_oracle(nmf, n, m, p, nu, q, T, inner, tol):
    # Isolates Alg. 1: both sides get the same (float32) L, R, X_L, X_R.
    X, G0, F0 = _inputs(n, m, p, seed=n + nu)
    OmL, OmR = synth.gaussian_sketches(n, m, nu, seed=3)
    L, R, XL, XR = (a.astype(np.float32) for a in subspace.compress(X.astype(np.float64), nu, q, OmL, OmR))
    G, F = _t(G0), _t(F0)
    rec = _record(nmf, T, n, m, p)
    prob = nmf.compressed_problem(_t(L), _t(R), _t(XL), _t(XR), p)
    st = nmf.read_stats(nmf.solve(prob, G, F, T, inner, tol=tol, record=rec))
    assert st.status == 0
    Go, Fo, info = nenmf.nenmf_compressed(L, R, XL, XR, G0, F0, T, inner, tol=tol, record=True)
    Xd = X.astype(np.float64)
    r_gpu = _gpu_rre_history(Xd, rec)
    r_ora = metrics.rre_history(Xd, info["history"])
    assert np.max(np.abs(r_gpu - r_ora)) <= 1e-5, (r_gpu - r_ora)
    G1, F1 = info["history"][0]
    assert_entrywise(_np(rec.G[0]), G1, 1e-4, "G after one outer iteration")
    assert_entrywise(_np(rec.F[0]), F1, 1e-4, "F after one outer iteration")
    assert st.total_inner[0] + st.total_inner[1] == pytest.approx(sum(a + b for a, b in info["inner"]), abs=2)


@pytest.mark.parametrize("mode", ["plain", "compressed"])
@pytest.mark.parametrize("inner,tol", [(10, 0.0), (30, 1e-6)])
def test_adaptive_restart_matches_oracle(nmf, mode, inner, tol):
    # NMF Gram matrices are ill-conditioned (one dominant eigenvalue), so the
    # momentum overshoots and restarts happen; the trajectories agree per outer iteration.
    n, m, p, nu, T = 300, 240, 12, 22, 8
    X, G0, F0 = _inputs(n, m, p, seed=31)
    Xd = X.astype(np.float64)
    G, F = _t(G0), _t(F0)
    rec = _record(nmf, T, n, m, p)
    if mode == "plain":
        prob = nmf.plain_problem(_t(X), p, 0)
        _, _, info = nenmf.nenmf_plain(Xd, G0, F0, T, inner, tol=tol, record=True, restart=True)
    else:
        OmL, OmR = synth.gaussian_sketches(n, m, nu, seed=3)
        L, R, XL, XR = (a.astype(np.float32) for a in subspace.compress(Xd, nu, 2, OmL, OmR))
        prob = nmf.compressed_problem(_t(L), _t(R), _t(XL), _t(XR), p)
        _, _, info = nenmf.nenmf_compressed(L, R, XL, XR, G0, F0, T, inner, tol=tol, record=True, restart=True)
    st = nmf.read_stats(nmf.solve(prob, G, F, T, inner, tol=tol, record=rec, restart=True))
    assert st.status == 0
    r_gpu = _gpu_rre_history(Xd, rec)
    r_ora = metrics.rre_history(Xd, info["history"])
    assert np.max(np.abs(r_gpu - r_ora)) <= 1e-5, (r_gpu - r_ora)


def test_timestamps_are_monotone(nmf):
    n, m, p = 256, 256, 4
    X, G0, F0 = _inputs(n, m, p, seed=5)
    rec = _record(nmf, 6, n, m, p)
    nmf.solve(nmf.plain_problem(_t(X), p, 1), _t(G0), _t(F0), 6, 10, record=rec)
    t = rec.times.cpu().numpy()
    assert np.all(np.diff(t) > 0) and t[0] > 0


def test_zero_outer_iterations_is_identity(nmf):
    X, G0, F0 = _inputs(70, 80, 3, seed=8)
    G, F = _t(G0), _t(F0)
    nmf.solve(nmf.plain_problem(_t(X), 3, 0), G, F, 0, 10)
    np.testing.assert_array_equal(_np(G), G0)
    np.testing.assert_array_equal(_np(F), F0)


def test_zero_factor_is_a_fixed_point(nmf):
    # F = 0 makes H_G = F F^T = 0 (L_c = 0): the G update returns G unchanged,
    # as in the oracle; the F update then proceeds from it.
    X, G0, _ = _inputs(60, 50, 3, seed=9)
    F0 = np.zeros((3, 50), dtype=np.float32)
    G, F = _t(G0), _t(F0)
    nmf.solve(nmf.plain_problem(_t(X), 3, 0), G, F, 1, 10)
    Go, Fo, _ = nenmf.nenmf_plain(X.astype(np.float64), G0, F0, 1, 10)
    np.testing.assert_allclose(_np(G), Go, rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(_np(F), Fo, rtol=1e-4, atol=1e-6)


def test_nothing_compressed_equals_plain_on_gpu(nmf):
    # nu = n = m: L and R are square orthogonal and Alg. 1 reduces to plain NeNMF.
    n = m = 48
    p = 4
    X, G0, F0 = _inputs(n, m, p, seed=12)
    L, R, XL, XR = nmf.compress(_t(X), n, 1, prec=0, seed=1)
    Gc, Fc = _t(G0), _t(F0)
    nmf.solve(nmf.compressed_problem(L, R, XL, XR, p), Gc, Fc, 10, 10)
    Gp, Fp = _t(G0), _t(F0)
    nmf.solve(nmf.plain_problem(_t(X), p, 0), Gp, Fp, 10, 10)
    Xd = X.astype(np.float64)
    assert abs(metrics.rre(Xd, _np(Gc), _np(Fc)) - metrics.rre(Xd, _np(Gp), _np(Fp))) < 1e-5
