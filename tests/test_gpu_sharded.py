"""The row-sharded schedule's per-GPU steps on one GB300, through the C ABI.

* nmf_gram: the float-float Gram of float32 rows against float64;
* nmf_orth_apply: one CholeskyQR pass with a given Gram (R^T R = S), and two
  passes against the oracle's Householder basis;
* nenmf_nnls_block: every iterate of a block against the oracle's inner loop
  run for that many iterations, the recorded ||P grad||^2 against float64 on
  the returned iterates, and a block split (0..3, 4..9) identical to one
  block; kb = 0 evaluates at Y;
* the whole sharded schedule (paper_1812_04315_gb300.sharded with
  CudaBackend) on one rank against the oracle's Alg. 2 + Alg. 1: RRE after
  every outer iteration within 1e-5, the float32 bar of the single-GPU path.
The schedule's collectives over two ranks are tests/test_sharded.py (CPU).
"""

import numpy as np
import pytest

import synth
from oracle import metrics, nenmf, subspace

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("N,nu", [(1000, 20), (257, 1), (3000, 64)])
def test_gram_matches_float64(nmf, N, nu):
    rng = np.random.default_rng(N + nu)
    Y = rng.standard_normal((N, nu)).astype(np.float32)
    S = nmf.gram(_t(Y)).cpu().numpy()
    Yd = Y.astype(np.float64)
    ref = Yd.T @ Yd
    # float-float sums of exact products: ~N 2^-46 of the terms' magnitude
    assert np.all(np.abs(S - ref) <= 1e-11 * (np.abs(Yd).T @ np.abs(Yd)))
    np.testing.assert_array_equal(S, S.T)


def test_orth_apply_one_and_two_passes(nmf):
    import torch
    rng = np.random.default_rng(5)
    N, nu = 2000, 16
    Y = (rng.standard_normal((N, nu)) @ np.diag(np.logspace(0, 3, nu))).astype(np.float32)
    Yg = _t(Y)
    S = nmf.gram(Yg)
    Q1 = nmf.orth_apply(Yg, S)
    # Q1 R = Y with R^T R = S (the float64 Cholesky of the same Gram)
    U = np.linalg.cholesky(S.cpu().numpy()).T
    np.testing.assert_allclose(_np(Q1) @ U, Y.astype(np.float64), atol=2e-5 * np.abs(Y).max())
    Q2 = nmf.orth_apply(Q1, nmf.gram(Q1))
    Q2n = _np(Q2)
    assert np.abs(Q2n.T @ Q2n - np.eye(nu)).max() <= 1e-5
    np.testing.assert_allclose(Q2n, subspace.orthonormal_basis(Y.astype(np.float64)), atol=1e-5)
    # aliasing Q with Y is allowed
    Z = Q1.clone()
    nmf.orth_apply(Z, nmf.gram(Z), out=Z)
    np.testing.assert_array_equal(_np(Z), Q2n)
    assert torch.isfinite(Z).all()


@pytest.mark.parametrize("p,N", [(7, 500), (1, 33), (16, 300), (32, 129)])
def test_nnls_block_matches_the_inner_loop(nmf, p, N):
    rng = np.random.default_rng(p * 100 + N)
    W = rng.random((p, p + 5)).astype(np.float32)
    H = (W.astype(np.float64) @ W.T.astype(np.float64)).astype(np.float32)
    B = (rng.random((p, N)) * 2.0 - 0.3).astype(np.float32)
    Y0 = rng.random((p, N)).astype(np.float32)
    K = 10
    Y, Fp = _t(Y0), _t(Y0)
    keep, pg2, lc = nmf.nnls_block(_t(H), _t(B), Y, Fp, 0, K, K)
    Hd, Bd = H.astype(np.float64), B.astype(np.float64)
    assert abs(float(lc.item()) - np.linalg.eigvalsh(Hd)[-1]) <= 1e-5 * np.linalg.eigvalsh(Hd)[-1]
    for i in range(K):
        ref, _, _ = nenmf.nesterov_nnls(Hd, Bd, Y0, i + 1)
        got = _np(keep[i])
        s = np.sqrt(np.mean(ref * ref))
        assert np.all(np.abs(got - ref) <= 1e-4 * (np.abs(ref) + s)), (i, np.abs(got - ref).max())
        pg = np.sum(nenmf.projected_gradient(got, Hd @ got - Bd) ** 2)
        assert abs(float(pg2[i].item()) - pg) <= 1e-4 * pg + 1e-12
    # the same ten iterations as two blocks
    Y2, Fp2 = _t(Y0), _t(Y0)
    ka, _, _ = nmf.nnls_block(_t(H), _t(B), Y2, Fp2, 0, 4, K)
    kb, _, _ = nmf.nnls_block(_t(H), _t(B), Y2, Fp2, 4, 6, K)
    np.testing.assert_array_equal(_np(ka), _np(keep[:4]))
    np.testing.assert_array_equal(_np(kb), _np(keep[4:]))
    np.testing.assert_array_equal(_np(Y2), _np(Y))
    # kb = 0: ||P grad||^2 at Y, no step
    Ye = _t(Y0)
    _, pe, _ = nmf.nnls_block(_t(H), _t(B), Ye, _t(Y0), 0, 0, 1)
    Yd = Y0.astype(np.float64)
    pref = np.sum(nenmf.projected_gradient(Yd, Hd @ Yd - Bd) ** 2)
    assert abs(float(pe[0].item()) - pref) <= 1e-4 * pref
    np.testing.assert_array_equal(_np(Ye), Y0.astype(np.float64))


@pytest.mark.parametrize("tol", [0.0, 1e-4])
def test_sharded_schedule_on_one_gpu(nmf, tol):
    from paper_1812_04315_gb300 import sharded
    n, m, p, nu, q, T, K = 900, 700, 6, 14, 2, 12, 20
    X, _, _ = synth.lowrank_data(n, m, p, seed=31, snr_db=30.0, dtype=np.float32)
    G0, F0 = (a.astype(np.float32) for a in synth.initial_factors(n, m, p, seed=32))
    OmL, OmR = (a.astype(np.float32) for a in synth.gaussian_sketches(n, m, nu, seed=33))
    be, comm = sharded.CudaBackend(), sharded.Collective()
    assert comm.world == 1
    Xg = _t(X)
    Lt, R, XLt, XR = sharded.compress(be, comm, Xg, nu, q, _t(OmL), _t(OmR.T))
    G, F, info = sharded.solve(be, comm, Lt, R, XLt, XR, _t(G0), _t(F0), T, K, 1, tol, record=True)
    r_gpu = np.array([nmf.rre(Xg, g.contiguous(), f.contiguous()) for g, f in info["history"]])
    Xd = X.astype(np.float64)
    L, Ro, XL, XRo = subspace.compress(Xd, nu, q, OmL.astype(np.float64), OmR.astype(np.float64))
    _, _, ref = nenmf.nenmf_compressed(L, Ro, XL, XRo, G0, F0, T, K, tol=tol, record=True)
    r_ora = metrics.rre_history(Xd, ref["history"])
    assert np.max(np.abs(r_gpu - r_ora)) <= 1e-5, np.abs(r_gpu - r_ora).max()
    np.testing.assert_allclose(_np(R), Ro, atol=1e-4)
    if tol > 0:
        assert abs(info["eps"] - ref["eps"]) <= 1e-4 * ref["eps"]
        for (kg, kf), (og, of) in zip(info["inner"], ref["inner"]):
            assert abs(kg - og) <= 1 and abs(kf - of) <= 1
