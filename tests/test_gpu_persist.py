"""The persistent compressed solve (all outer iterations of Alg. 1 in one
cooperative launch) against the per-update launches of the same method.

Both paths run the same arithmetic in the same order: the per-CTA shares of
the p x nu products, their fixed-order sums, H, L_c, B, the inner loop of
Sec. 2 with its stop test, eps from the projected gradients at (G0, F0).
(For p <= 6 at padded rank 8 and p in 9..10 at rank 12 the persistent
inner loop leaves out two padding rows, which hold exact zeros.) So their
factors, statistics and snapshots agree bit for bit; the oracle parity of
the default (persistent) path is tests/test_gpu_solve.py's. Cases cover
ragged tiles, n != m (CTAs idle on one side), p = 1, nu = 1, p = 32, both
shortened loop ranks, the stop test with early stops, min_inner, adaptive
restart, snapshots, zero outer iterations and a zero factor (L_c = 0).
"""

import numpy as np
import pytest

import synth
from oracle import subspace

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _case(n, m, p, nu, seed):
    X, _, _ = synth.lowrank_data(n, m, p, seed=seed, snr_db=30.0, dtype=np.float32)
    G0, F0 = (a.astype(np.float32) for a in synth.initial_factors(n, m, p, seed=seed + 1))
    OmL, OmR = synth.gaussian_sketches(n, m, nu, seed=seed + 2)
    L, R, XL, XR = (a.astype(np.float32) for a in subspace.compress(X.astype(np.float64), nu, 1, OmL, OmR))
    return (L, R, XL, XR), G0, F0


def _run(nmf, comp, G0, F0, p, T, inner, per_update, **kw):
    import torch
    n, m = G0.shape[0], F0.shape[1]
    nmf.set_kernel_path(per_update_solve=per_update)
    try:
        G, F = _t(G0), _t(F0)
        rec = nmf.SolveRecord(G=torch.zeros((max(T, 1), n, p), device="cuda"),
                              F=torch.zeros((max(T, 1), p, m), device="cuda"),
                              times=torch.zeros(T + 1, dtype=torch.int64, device="cuda"))
        st = nmf.solve(nmf.compressed_problem(*(_t(a) for a in comp), p), G, F, T, inner, record=rec, **kw)
        torch.cuda.synchronize()
    finally:
        nmf.set_kernel_path()
    return G, F, nmf.read_stats(st), rec


CASES = [
    # n, m, p, nu, T, inner, kwargs
    (1000, 1000, 10, 20, 12, 10, dict(tol=1e-6)),
    (777, 1500, 8, 18, 10, 10, dict(tol=1e-4)),
    (1500, 333, 5, 12, 8, 10, dict(tol=0.0)),
    (129, 700, 12, 22, 10, 10, dict(tol=1e-3, min_inner=3)),
    (300, 257, 1, 1, 6, 5, dict(tol=1e-6)),
    (200, 190, 32, 40, 4, 10, dict(tol=1e-5)),
    (640, 384, 12, 20, 6, 30, dict(tol=1e-6, restart=True)),
    (500, 400, 6, 10, 5, 10, dict(tol=0.0, restart=True)),
    (64, 40, 4, 6, 5, 10, dict(tol=1e-6)),
    (300, 300, 6, 12, 0, 10, dict(tol=1e-6)),
    (900, 1100, 6, 14, 8, 10, dict(tol=1e-5)),
    (600, 500, 9, 19, 6, 20, dict(tol=1e-6, restart=True)),
]


@pytest.mark.parametrize("n,m,p,nu,T,inner,kw", CASES)
def test_persistent_equals_per_update(nmf, n, m, p, nu, T, inner, kw):
    import torch
    comp, G0, F0 = _case(n, m, p, nu, seed=n + m + p)
    Ga, Fa, sa, ra = _run(nmf, comp, G0, F0, p, T, inner, False, **kw)
    Gb, Fb, sb, rb = _run(nmf, comp, G0, F0, p, T, inner, True, **kw)
    assert sa.status == 0 and sb.status == 0
    assert bool(torch.equal(Ga, Gb)) and bool(torch.equal(Fa, Fb))
    assert (sa.outer_done, tuple(sa.last_inner), tuple(sa.total_inner)) == \
        (sb.outer_done, tuple(sb.last_inner), tuple(sb.total_inner))
    assert sa.eps == sb.eps and tuple(sa.pg_norm) == tuple(sb.pg_norm) and tuple(sa.lipschitz) == tuple(sb.lipschitz)
    if T > 0:
        assert bool(torch.equal(ra.G[:T], rb.G[:T])) and bool(torch.equal(ra.F[:T], rb.F[:T]))
        ts = ra.times.cpu().numpy()
        assert np.all(np.diff(ts) > 0)   # one stamp per outer iteration, increasing
        np.testing.assert_array_equal(ra.G[T - 1].cpu().numpy(), Ga.cpu().numpy())


def test_zero_factor_keeps_the_other(nmf):
    import torch
    comp, G0, F0 = _case(400, 300, 5, 10, seed=9)
    F0 = np.zeros_like(F0)   # H_G = 0: the G update keeps G (L_c = 0)
    Ga, Fa, sa, _ = _run(nmf, comp, G0, F0, 5, 3, 10, False, tol=1e-6)
    Gb, Fb, sb, _ = _run(nmf, comp, G0, F0, 5, 3, 10, True, tol=1e-6)
    assert sa.status == sb.status
    assert bool(torch.equal(Ga, Gb)) and bool(torch.equal(Fa, Fb))
