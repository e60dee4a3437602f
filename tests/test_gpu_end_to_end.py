"""End-to-end parity: GPU compression + GPU compressed NeNMF against the FP64
oracle's Alg. 2 + Alg. 1 on the same seeded inputs and sketches.

The target tolerance: RRE within 1e-5 of the oracle's on the float32 path and
within 1e-3 on the bfloat16 path, at every recorded outer iteration.
The full-size case is the benchmark's workload (n = m = 10^4, p = 10, nu = 20,
q = 4, 30 dB, 100 outer iterations of at most 10 inner ones), run in the
configuration the benchmark times; its RRE is checked at sampled iterations.
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


def _run(nmf, X, G0, F0, p, nu, q, T, inner, tol, prec, OmL, OmR, keep=None):
    import torch
    n, m = X.shape
    Xg = _t(X)
    L, R, XL, XR = nmf.compress(Xg, nu, q, prec=prec, omega_L=_t(OmL), omega_R=_t(OmR))
    G, F = _t(G0), _t(F0)
    keep = list(range(T)) if keep is None else keep
    rec = nmf.SolveRecord(G=torch.empty((T, n, p), device="cuda"), F=torch.empty((T, p, m), device="cuda"))
    st = nmf.read_stats(nmf.solve(nmf.compressed_problem(L, R, XL, XR, p), G, F, T, inner, tol=tol, record=rec))
    assert st.status == 0 and st.outer_done == T
    r = []
    for t in keep:
        r.append(nmf.rre(Xg, rec.G[t].contiguous(), rec.F[t].contiguous()))
    return np.array(r), st


@pytest.mark.parametrize("prec,tol_rre", [(0, 1e-5), (1, 1e-3)])
@pytest.mark.parametrize("n,m,p,nu,q", [(1000, 1000, 10, 20, 4), (777, 1500, 8, 18, 2)])
def test_compressed_nenmf_end_to_end(nmf, prec, tol_rre, n, m, p, nu, q):
    T, inner, tol = 40, 10, 1e-6
    X, _, _ = synth.lowrank_data(n, m, p, seed=21, snr_db=30.0, dtype=np.float32)
    G0, F0 = (a.astype(np.float32) for a in synth.initial_factors(n, m, p, seed=22))
    OmL, OmR = (a.astype(np.float32) for a in synth.gaussian_sketches(n, m, nu, seed=23))
    r_gpu, st = _run(nmf, X, G0, F0, p, nu, q, T, inner, tol, prec, OmL, OmR)
    Xd = X.astype(np.float64)
    L, R, XL, XR = subspace.compress(Xd, nu, q, OmL.astype(np.float64), OmR.astype(np.float64))
    _, _, info = nenmf.nenmf_compressed(L, R, XL, XR, G0, F0, T, inner, tol=tol, record=True)
    r_ora = metrics.rre_history(Xd, info["history"])
    assert np.max(np.abs(r_gpu - r_ora)) <= tol_rre, np.abs(r_gpu - r_ora).max()


@pytest.mark.parametrize("prec,tol_rre", [(1, 1e-3), (0, 1e-5)])
def test_full_size_workload(nmf, prec, tol_rre):
    n = m = 10000
    p, nu, q, T, inner, tol = 10, 20, 4, 100, 10, 1e-6
    X, _, _ = synth.lowrank_data(n, m, p, seed=0, snr_db=30.0, dtype=np.float32)
    G0, F0 = (a.astype(np.float32) for a in synth.initial_factors(n, m, p, seed=1))
    OmL, OmR = (a.astype(np.float32) for a in synth.gaussian_sketches(n, m, nu, seed=2))
    keep = [0, 9, 49, 99]
    r_gpu, st = _run(nmf, X, G0, F0, p, nu, q, T, inner, tol, prec, OmL, OmR, keep=keep)
    Xd = X.astype(np.float64)
    L, R, XL, XR = subspace.compress(Xd, nu, q, OmL.astype(np.float64), OmR.astype(np.float64))
    Go, Fo, info = nenmf.nenmf_compressed(L, R, XL, XR, G0, F0, T, inner, tol=tol, record=True)
    r_ora = np.array([metrics.rre(Xd, *info["history"][t]) for t in keep])
    assert np.max(np.abs(r_gpu - r_ora)) <= tol_rre, (r_gpu, r_ora)


def test_largest_configuration(nmf):
    # n = 5e4, m = 2e4 (X 4 GB float32), p = 32, nu = 42, q = 4, 40 dB, 10%
    # of G0's entries zero, bfloat16 compression. With the stop test on, the
    # solve has more vectors than one co-resident grid holds and runs on the
    # batched kernel; properties at full size, and the single-problem kernel
    # (stop test off, which needs no co-residency) against the batched kernel
    # on the same compressed inputs.
    import torch
    n, m, p, nu, q = 50000, 20000, 32, 42, 4
    X, _, _ = synth.lowrank_data_device(n, m, p, seed=5, snr_db=40.0, zero_frac=0.1)
    L, R, XL, XR = nmf.compress(X, nu, q, prec=nmf.PREC_BF16, seed=6)
    assert float((L @ L.T - torch.eye(nu, device="cuda")).abs().max()) < 2e-5
    assert float((R.T @ R - torch.eye(nu, device="cuda")).abs().max()) < 2e-5
    G0, F0 = (_t(a) for a in synth.initial_factors(n, m, p, seed=7))
    prob = nmf.compressed_problem(L, R, XL, XR, p)
    G, F = G0.clone(), F0.clone()
    st = nmf.read_stats(nmf.solve(prob, G, F, 60, 10, tol=1e-6))
    torch.cuda.synchronize()
    assert st.status == 0 and st.outer_done == 60
    assert bool(torch.isfinite(G).all()) and bool((G >= 0).all()) and bool((F >= 0).all())
    r0, r1 = nmf.rre(X, G0, F0), nmf.rre(X, G, F)
    assert r1 < 0.05 and r1 < r0 / 10, (r0, r1)   # 40 dB: the noise floor is about 0.01
    # two kernels, one method: stop test off, 5 outer iterations
    G1, F1 = G0.clone(), F0.clone()
    nmf.solve(prob, G1, F1, 5, 10)
    G2, F2 = G0.clone(), F0.clone()
    nmf.solve_batched([prob], [G2], [F2], 5, 10, cluster=8)
    assert abs(nmf.rre(X, G1, F1) - nmf.rre(X, G2, F2)) <= 1e-5


@pytest.mark.parametrize("prec,tol_rre", [(1, 1e-3), (0, 1e-5)])
def test_largest_configuration_shape_against_oracle(nmf, prec, tol_rre):
    # The largest configuration's regime at a size the oracle finishes in
    # seconds: p = 32 (the widest register tile of the solve kernel),
    # nu = 42 (the 48-wide MMA of the tensor-core pass), q = 4, 40 dB noise,
    # 10 % of G0's entries zero (sparse sources); n x m = 5000 x 2000 keeps
    # the 5 : 2 aspect. GPU compression + solve against the oracle's Alg. 2 +
    # Alg. 1 on the same sketches, RRE at every outer iteration.
    n, m, p, nu, q, T, inner, tol = 5000, 2000, 32, 42, 4, 100, 10, 1e-6
    X, _, _ = synth.lowrank_data(n, m, p, seed=5, snr_db=40.0, dtype=np.float32, zero_frac=0.1)
    G0, F0 = (a.astype(np.float32) for a in synth.initial_factors(n, m, p, seed=7))
    OmL, OmR = (a.astype(np.float32) for a in synth.gaussian_sketches(n, m, nu, seed=6))
    r_gpu, st = _run(nmf, X, G0, F0, p, nu, q, T, inner, tol, prec, OmL, OmR)
    Xd = X.astype(np.float64)
    L, R, XL, XR = subspace.compress(Xd, nu, q, OmL.astype(np.float64), OmR.astype(np.float64))
    _, _, info = nenmf.nenmf_compressed(L, R, XL, XR, G0, F0, T, inner, tol=tol, record=True)
    r_ora = metrics.rre_history(Xd, info["history"])
    print("max |RRE gpu - RRE oracle|", np.abs(r_gpu - r_ora).max(), "final", r_gpu[-1], r_ora[-1])
    assert np.max(np.abs(r_gpu - r_ora)) <= tol_rre, np.abs(r_gpu - r_ora).max()
