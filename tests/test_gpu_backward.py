"""GPU parity of nenmf_backward (reverse-mode derivative of the compressed solve) against the FP64 oracle.

Both sides start from the same float32 X, L, R, X_L, X_R, G0, F0. The GPU
forward is nenmf_solve with the stop test off and snapshots on; the
oracle's is oracle.adjoint.compressed_forward. Each side forms the
cotangents of the loss ||X - G_T F_T||_F^2 from its own (G_T, F_T) and runs
its backward; compared are dX_L, dX_R, dG0, dF0 and the total dX
(2 (X - G_T F_T) + L^T dX_L + dX_R R^T), entry by entry.

Per-entry bound. The GPU computes in float32 (u = 2^-24). Every one of the
2 T K adjoint steps is a p-term matrix-vector product applied to a cotangent
of the block's scale, so each entry's rounding error is ~p u times the
scale of the terms that make it, not times the entry itself (an entry that
is small by cancellation carries the error of its terms). Bound per entry:
    |gpu - oracle| <= tol * (|oracle| + s),
with s the root-mean-square of that block's oracle values (its own scale;
no borrowing from other blocks) and tol ~ 2 T K p u: 2e-4 for the small
cases, 1e-3 for the 4096 x 4096 one (see below).

Mask stability. The forward trajectories differ by float32 rounding, which
moves a projection's activity only where a pre-projection value z sits
within ~1e-6 of 0 relative to its column. The small cases assert that the
oracle's trajectory keeps every |z| above 1e-6 of its column's largest |z|
(re-seeded where it did not), so both sides take the same projections. The
4096 x 4096 case (13 million z's, margin ~3e-8) cannot meet that; it is
checked per block in relative norm at 1e-3 and by the share of entries
outside the entry-wise bound. The p = nu = 1 case, whose exact dG0 is 0 and
whose dX_L, dX_R are small by cancellation, has a test of its own.
"""

import numpy as np
import pytest

from _parity import entrywise_ratio
import synth
from oracle import adjoint, subspace

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _check(gpu, ora, tol):
    errs = {name: entrywise_ratio(a, b) for name, a, b in zip(("dXL", "dXR", "dG0", "dF0", "dX"), gpu, ora)}
    print({k: f"{v:.2e}" for k, v in errs.items()})
    for name, r in errs.items():
        assert r <= tol, (name, errs)


def _mask_margin(L, R, XL, XR, G0, F0, T, K):
    """Smallest |z| of the oracle's forward relative to its column's largest |z|."""
    _, _, tape = adjoint.compressed_forward(L, R, XL, XR, G0, F0, T, K)
    margin = np.inf
    for s in tape:
        for t in (s["tG"], s["tF"]):
            for z in t.get("z", []):
                col = np.abs(z).max(axis=0, keepdims=True) + 1e-300
                margin = min(margin, float((np.abs(z) / col).min()))
    return margin


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


@pytest.mark.parametrize("n,m,p,nu,q,T,K,seed", [
    (64, 48, 4, 8, 2, 3, 5, 68),        # the finite-difference configuration of the oracle's pins
    (200, 150, 5, 10, 2, 4, 5, 205),
    (300, 257, 12, 20, 1, 3, 10, 314),  # re-seeded: the first seed's margin was 6e-7
    (96, 80, 16, 26, 2, 2, 1, 112),
    (150, 140, 20, 30, 1, 2, 4, 170),
])
def test_backward_matches_oracle(nmf, n, m, p, nu, q, T, K, seed):
    args = _inputs(n, m, p, nu, q, seed=seed)
    margin = _mask_margin(*args[1:], T, K)
    print("mask margin", margin)
    assert margin > 1e-6
    _check(_gpu(nmf, *args, p, T, K), _oracle(*args, T, K), 2e-4)


def test_backward_exact_one_dimensional_solves(nmf):
    # p = nu = 1: every inner solve is a 1-D problem solved exactly by its
    # first step (z = b / h), so G_T does not depend on G0 and the exact dG0 is
    # 0; dX_L and dX_R are small by cancellation (~1e-5 against a loss
    # gradient of ~4e-2), so their entries carry rounding of terms of the
    # cotangents' scale, not of their own. Bounds: dX (no cancellation) per
    # entry at the adjoint's 2e-4; every other block within 2e-2 of the
    # largest cotangent fed in (max |dG_T|, |dF_T|): the steps after the
    # first sit at the 1-D fixed point, where the adjoint carries factors
    # (1 - h / L_c) that vanish exactly but are ~u in float32 (h summed in
    # float32, L_c by a float-float Rayleigh quotient) and are amplified by
    # the extrapolation weights, so these cancellation-sized blocks keep
    # errors of ~1e-2 of the cotangent scale (measured 6e-3 for dX_L).
    n, m, p, nu, q, T, K = 130, 90, 1, 1, 1, 2, 3
    X, L, R, XL, XR, G0, F0 = _inputs(n, m, p, nu, q, seed=131)
    gpu = _gpu(nmf, X, L, R, XL, XR, G0, F0, p, T, K)
    ora = _oracle(X, L, R, XL, XR, G0, F0, T, K)
    assert np.abs(ora[2]).max() == 0.0                  # the oracle's dG0 vanishes exactly
    assert entrywise_ratio(gpu[4], ora[4]) <= 2e-4      # dX
    G, F, _ = adjoint.compressed_forward(L, R, XL, XR, G0, F0, T, K)
    E = X.astype(np.float64) - G @ F
    cot = max(np.abs(2.0 * E @ F.T).max(), np.abs(2.0 * G.T @ E).max())
    errs = {name: float(np.abs(a - b).max() / cot) for name, a, b in zip(("dXL", "dXR", "dG0", "dF0"), gpu[:4], ora[:4])}
    print("errors relative to the cotangent scale", errs)
    for name, e in errs.items():
        assert e <= 2e-2, (name, errs)


def test_backward_full_size(nmf):
    # n = m = 4096, p = 16, nu = 26, q = 2; 20 outer x 5 inner. With 13
    # million pre-projection values the oracle's trajectory has values within
    # ~1e-7 of 0 relative to their column (the margin printed), so float32
    # rounding flips a few projections and the entries downstream of a flip
    # differ by O(1) of their size: an entry-wise comparison is not defined
    # here. Checked instead: each block's relative Frobenius error (no floor
    # borrowed from other blocks) and the share of entries outside the
    # small-case entry-wise bound.
    args = _inputs(4096, 4096, 16, 26, 2, seed=4)
    print("mask margin", _mask_margin(*args[1:], 20, 5))
    gpu, ora = _gpu(nmf, *args, 16, 20, 5), _oracle(*args, 20, 5)
    for name, a, b in zip(("dXL", "dXR", "dG0", "dF0", "dX"), gpu, ora):
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        s = np.sqrt(np.mean(b * b))
        outside = float(np.mean(np.abs(a - b) > 1e-3 * (np.abs(b) + s)))
        print(name, f"relative {rel:.2e}, entries outside 1e-3 (|ref| + rms): {outside:.2e}")
        assert rel <= 1e-3, (name, rel)
        assert outside <= 1e-2, (name, outside)


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
