"""GPU checks of nmf_project and of the torch.autograd.Function around the
compressed solve and its adjoint (nenmf_backward), against the FP64 oracle.

nmf_project computes X_L = L X and X_R = X R in float32 (products of length
n or m with float32 accumulation: 1e-5 relative) or from bfloat16 X and
bases (8 significant bits: 1e-2). The autograd gradient of
||X - G_T F_T||^2 is compared with oracle.adjoint.loss_and_gradient under
the tolerance of the GPU backward's own parity test (2e-4 relative, each
gradient floored at 1% of the whole gradient's norm).
"""

import numpy as np
import pytest

from _parity import assert_entrywise, assert_product, bf16_round
import synth
from oracle import adjoint, subspace

pytestmark = pytest.mark.gpu


def _t(a, grad=False):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda", requires_grad=grad)


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _bases(n, m, p, nu, q, seed):
    X, _, _ = synth.lowrank_data(n, m, p, seed=seed, snr_db=20.0, dtype=np.float32)
    OmL, OmR = synth.gaussian_sketches(n, m, nu, seed=seed + 2)
    L, R, _, _ = subspace.compress(X.astype(np.float64), nu, q, OmL, OmR)
    return X, L.astype(np.float32), R.astype(np.float32)


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-2)])
@pytest.mark.parametrize("n,m,nu", [(300, 257, 12), (129, 400, 7)])
def test_project(nmf, n, m, nu, prec, tol):
    X, L, R = _bases(n, m, 4, nu, 1, seed=n)
    XL, XR = nmf.project(_t(X), _t(L), _t(R), prec=prec)
    Xd, Ld, Rd = X.astype(np.float64), L.astype(np.float64), R.astype(np.float64)
    if prec == 1:  # the tensor cores multiply the bfloat16-rounded operands
        Xd, Ld, Rd = bf16_round(X), bf16_round(L), bf16_round(R)
    assert_product(_np(XL), Ld, Xd, "X_L")
    assert_product(_np(XR), Xd, Rd, "X_R")


@pytest.mark.parametrize("n,m,p,nu,q,T,K", [(200, 150, 5, 10, 2, 4, 5), (96, 80, 3, 6, 1, 2, 10)])
def test_autograd_gradient_matches_oracle(nmf, n, m, p, nu, q, T, K):
    X, L, R = _bases(n, m, p, nu, q, seed=n + p)
    G0, F0 = (a.astype(np.float32) for a in synth.initial_factors(n, m, p, seed=3))
    Xt, Gt, Ft = _t(X, True), _t(G0, True), _t(F0, True)
    G, F = nmf.compressed_nenmf(Xt, Gt, Ft, _t(L), _t(R), T, K)
    loss = ((Xt - G @ F) ** 2).sum()
    loss.backward()
    lo, dXo, dG0o, dF0o = adjoint.loss_and_gradient(X.astype(np.float64), L.astype(np.float64),
                                                    R.astype(np.float64), G0.astype(np.float64),
                                                    F0.astype(np.float64), T, K)
    assert abs(float(loss.detach()) - lo) <= 1e-4 * lo
    # per entry, with the adjoint's bound (tests/test_gpu_backward.py)
    for name, a, b in zip(("dX", "dG0", "dF0"), (Xt.grad, Gt.grad, Ft.grad), (dXo, dG0o, dF0o)):
        assert_entrywise(_np(a), b, 2e-4, name)


def test_autograd_forward_equals_solve(nmf):
    import torch
    n, m, p, nu, q, T, K = 150, 120, 4, 8, 1, 3, 5
    X, L, R = _bases(n, m, p, nu, q, seed=5)
    G0, F0 = (a.astype(np.float32) for a in synth.initial_factors(n, m, p, seed=6))
    G, F = nmf.compressed_nenmf(_t(X), _t(G0), _t(F0), _t(L), _t(R), T, K)
    XL, XR = nmf.project(_t(X), _t(L), _t(R))
    G2, F2 = _t(G0), _t(F0)
    nmf.solve(nmf.compressed_problem(_t(L), _t(R), XL, XR, p), G2, F2, T, K)
    assert bool(torch.equal(G, G2)) and bool(torch.equal(F, F2))
