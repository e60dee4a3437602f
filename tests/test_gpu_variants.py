"""GPU parity of nmf_compress_variant (the compression variants) against the FP64 oracle.

Both sides get the same host-drawn sketches; tolerances as for nmf_compress
(float32 path: 2^-24-scale errors amplified by the conditioning of the sketch
products; bfloat16 path: X and the bases rounded to 8 significant bits).
* swapped, single: orthonormality, the subspace of the leading p directions,
  the leading p basis vectors entrywise (the same orthonormalisation as the
  default), exact projectors on exactly low-rank X;
* power iteration: the columns between products are only rescaled, so a
  direction with singular value s_i keeps a share (s_i / s_1)^(2q+1) of the
  product; below the working precision (2^-24, bfloat16 2^-9) it is lost,
  which is the variant's known weakness against subspace iteration. Its test
  uses a spectrum the precision resolves (s from 1 to 0.3 over nu directions)
  and compares the leading subspace and the captured energy;
* Gaussian projection: L, R are the scaled sketches (entrywise), X_L and X_R
  the products (float64 products of the library's own L, R).
"""

import numpy as np
import pytest

from _parity import assert_product, bf16_round
import synth
from oracle import subspace

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _final_pass(XL, XR, L, R, X, prec):
    """X_L = L X and X_R = X R entry by entry against float64 products of the
    operands the last pass multiplied (bfloat16-rounded for prec 1)."""
    if prec == 1:
        Ld, Rd, Xd = bf16_round(L), bf16_round(R), bf16_round(X)
    else:
        Ld, Rd, Xd = (np.asarray(a, dtype=np.float64) for a in (L, R, X))
    assert_product(XL, Ld, Xd, "X_L")
    assert_product(XR, Xd, Rd, "X_R")


def _max_angle(Q1, Q2):
    return np.linalg.norm(Q1 - Q2 @ (Q2.T @ Q1), 2)


def _run(nmf, X, nu, q, prec, variant, seed=7):
    n, m = X.shape
    OmL, OmR = (a.astype(np.float32) for a in synth.gaussian_sketches(n, m, nu, seed=seed))
    gpu = [_np(t) for t in nmf.compress(_t(X), nu, q, prec=prec, omega_L=_t(OmL), omega_R=_t(OmR), variant=variant)]
    ora = subspace.compress_variant(X.astype(np.float64), nu, q, OmL.astype(np.float64), OmR.astype(np.float64),
                                    variant)
    return gpu, ora


@pytest.mark.parametrize("variant", ["swapped", "single"])
@pytest.mark.parametrize("n,m,p,nu,q", [(300, 257, 5, 12, 2), (257, 300, 4, 9, 1), (640, 384, 10, 20, 3)])
@pytest.mark.parametrize("prec", [0, 1])
def test_orthonormalising_variants(nmf, variant, n, m, p, nu, q, prec):
    X, _, _ = synth.lowrank_data(n, m, p, seed=n + q, snr_db=30.0, dtype=np.float32)
    (L, R, XL, XR), (Lo, Ro, XLo, XRo) = _run(nmf, X, nu, q, prec, variant)
    np.testing.assert_allclose(L @ L.T, np.eye(nu), atol=2e-5)
    np.testing.assert_allclose(R.T @ R, np.eye(nu), atol=2e-5)
    ang_tol = 1e-3 if prec == 0 else 5e-2
    assert _max_angle(L.T[:, :p], Lo.T) < ang_tol
    assert _max_angle(R[:, :p], Ro) < ang_tol
    lead = 2e-4 if prec == 0 else 3e-2
    np.testing.assert_allclose(L[:p], Lo[:p], atol=lead * np.abs(Lo[:p]).max())
    np.testing.assert_allclose(R[:, :p], Ro[:, :p], atol=lead * np.abs(Ro[:, :p]).max())
    Xd = X.astype(np.float64)
    _final_pass(XL, XR, L, R, X, prec)
    e_gpu = np.linalg.norm(XL) / np.linalg.norm(Xd)
    e_ora = np.linalg.norm(XLo) / np.linalg.norm(Xd)
    assert abs(e_gpu - e_ora) < (1e-5 if prec == 0 else 1e-3)


@pytest.mark.parametrize("variant", ["swapped", "single"])
@pytest.mark.parametrize("prec", [0, 1])
def test_variants_exact_on_low_rank(nmf, variant, prec):
    n, m, p, nu, q = 333, 222, 6, 10, 2
    X, _, _ = synth.lowrank_data(n, m, p, seed=3, dtype=np.float32)
    (L, R, XL, XR), _ = _run(nmf, X, nu, q, prec, variant, seed=11)
    Xd = X.astype(np.float64)
    tol = 1e-5 if prec == 0 else 1e-2
    nx = np.linalg.norm(Xd)
    assert np.linalg.norm(Xd - L.T @ (L @ Xd)) <= tol * nx
    assert np.linalg.norm(Xd - (Xd @ R) @ R.T) <= tol * nx


def _spectrum_matrix(n, m, nu, seed):
    # singular values 1 .. 0.3 over nu directions, 1e-3 beyond: resolvable by
    # q <= 2 power steps in float32 and q = 1 in bfloat16
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.standard_normal((n, m)))[0]
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    s = np.concatenate([np.linspace(1.0, 0.3, nu), np.full(m - nu, 1e-3)])
    return ((U * s) @ V.T).astype(np.float32)


@pytest.mark.parametrize("prec,q", [(0, 1), (0, 2), (1, 1)])
def test_power_iteration(nmf, prec, q):
    n, m, nu, p = 400, 300, 10, 6
    X = _spectrum_matrix(n, m, nu, seed=q)
    (L, R, XL, XR), (Lo, Ro, XLo, XRo) = _run(nmf, X, nu, q, prec, "power")
    np.testing.assert_allclose(L @ L.T, np.eye(nu), atol=2e-5)
    np.testing.assert_allclose(R.T @ R, np.eye(nu), atol=2e-5)
    ang_tol = 1e-3 if prec == 0 else 5e-2
    assert _max_angle(L.T[:, :p], Lo.T) < ang_tol
    assert _max_angle(R[:, :p], Ro) < ang_tol
    Xd = X.astype(np.float64)
    e_gpu = np.linalg.norm(XL) / np.linalg.norm(Xd)
    e_ora = np.linalg.norm(XLo) / np.linalg.norm(Xd)
    assert abs(e_gpu - e_ora) < (1e-5 if prec == 0 else 1e-3)


@pytest.mark.parametrize("prec", [0, 1])
def test_gaussian_projection(nmf, prec):
    n, m, p, nu = 400, 350, 8, 20
    X, _, _ = synth.lowrank_data(n, m, p, seed=5, snr_db=30.0, dtype=np.float32)
    (L, R, XL, XR), (Lo, Ro, _, _) = _run(nmf, X, nu, 0, prec, "gaussian")
    np.testing.assert_allclose(L, Lo, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(R, Ro, rtol=1e-6, atol=1e-7)
    _final_pass(XL, XR, L, R, X, prec)


def test_library_sketch_variants_match_default_draw(nmf):
    # With the sketches drawn by the library (seed), the subspace variant equals nmf_compress
    import torch
    n, m, nu, q = 256, 200, 8, 2
    X, _, _ = synth.lowrank_data(n, m, 4, seed=9, snr_db=30.0, dtype=np.float32)
    a = nmf.compress(_t(X), nu, q, prec=0, seed=5)
    b = nmf.compress(_t(X), nu, q, prec=0, seed=5, variant="subspace")
    for x, y in zip(a, b):
        assert bool(torch.equal(x, y))
    g1 = nmf.compress(_t(X), nu, 0, prec=0, seed=5, variant="gaussian")
    g2 = nmf.compress(_t(X), nu, 0, prec=0, seed=5, variant="gaussian")
    for x, y in zip(g1, g2):
        assert bool(torch.equal(x, y))


@pytest.mark.parametrize("variant", ["subspace", "power"])
def test_compress_batched_equals_one_by_one(nmf, variant):
    # nmf_compress_batched runs each item's compression on its own lane; every
    # item here has at most 12 tiles, which fit one lane's share of the SMs,
    # so it equals nmf_compress_variant with the same seed, bit for bit
    import torch
    shapes = [(300, 200, 8), (128, 400, 5), (257, 129, 12), (90, 90, 4), (500, 333, 20), (64, 70, 3),
              (211, 150, 9), (180, 260, 7), (99, 101, 6), (77, 300, 10)]
    Xs = [_t(synth.lowrank_data(n, m, 4, seed=i, snr_db=20.0, dtype=np.float32)[0]) for i, (n, m, _) in
          enumerate(shapes)]
    nus = [nu for _, _, nu in shapes]
    outs = nmf.compress_batched(Xs, nus, 2, prec=1, seeds=list(range(40, 50)), variant=variant)
    torch.cuda.synchronize()
    for i, (X, nu) in enumerate(zip(Xs, nus)):
        ref = nmf.compress(X, nu, 2, prec=1, seed=40 + i, variant=variant)
        for a, b in zip(outs[i], ref):
            assert bool(torch.equal(a, b)), i


def test_compress_batched_large_item_matches_to_rounding(nmf):
    # With eight items a lane's X passes are planned for about 1/6 of the
    # SMs (24 of 152); an item of 9 x 8 = 72 tiles then gets fewer split-K
    # parts than alone (the
    # same products summed in another order). Its leading p basis vectors
    # (well separated: rank-4 data at 20 dB), the leading p singular values
    # of X_L and X_R and their norms agree with the one-by-one call to
    # float32 rounding; the trailing directions (noise, after q = 2) are ill
    # conditioned and are not compared one by one.
    import torch
    shapes = [(1100, 900, 12)] + [(200 + 10 * i, 150 + 7 * i, 6) for i in range(7)]
    Xs = [_t(synth.lowrank_data(n, m, 4, seed=60 + i, snr_db=20.0, dtype=np.float32)[0]) for i, (n, m, _) in
          enumerate(shapes)]
    nus = [nu for _, _, nu in shapes]
    outs = nmf.compress_batched(Xs, nus, 2, prec=1, seeds=list(range(70, 78)))
    torch.cuda.synchronize()
    L, R, XL, XR = (_np(a) for a in outs[0])
    Lr, Rr, XLr, XRr = (_np(a) for a in nmf.compress(Xs[0], nus[0], 2, prec=1, seed=70))
    np.testing.assert_allclose(L[:4], Lr[:4], atol=1e-4)
    np.testing.assert_allclose(R[:, :4], Rr[:, :4], atol=1e-4)
    for a, b in ((XL, XLr), (XR, XRr)):
        sa, sb = np.linalg.svd(a, compute_uv=False), np.linalg.svd(b, compute_uv=False)
        np.testing.assert_allclose(sa[:4], sb[:4], rtol=1e-4)
        assert abs(np.linalg.norm(a) - np.linalg.norm(b)) <= 1e-4 * np.linalg.norm(b)
    for i in range(1, len(shapes)):
        ref = nmf.compress(Xs[i], nus[i], 2, prec=1, seed=70 + i)
        for a, b in zip(outs[i], ref):
            assert bool(torch.equal(a, b)), i
