"""GPU parity of the building blocks through the C ABI against the oracle or exact references.

* Gaussian sketch: element-by-element against the oracle's Philox/Box-Muller;
* one pass, two products (nmf_dual_product): float32 path against float64
  products (tensor cores on three bfloat16 parts up to 32 columns, CUDA
  cores beyond, and the two against each other); bfloat16 path against
  float64 products of the bfloat16-rounded inputs (only the float32
  accumulation differs);
* RRE (eq. 4) against float64.

Tolerances. A float32 dot product of length K has error below
K * 2^-24 * sum|x_i a_i| (worst case); the tests use the bound with K replaced
by 4 sqrt(K) against the row's sum of |products| (random-sign rounding), which
the summation order of any split-K kernel satisfies with a wide margin.
"""

import numpy as np
import pytest

import synth
from oracle import philox

pytestmark = pytest.mark.gpu


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("rows,cols,seed,stream", [(37, 11, 5, 0), (20, 10000, 2**40 + 3, 1), (1, 3, 0, 7)])
def test_gaussian_sketch_matches_oracle(nmf, rows, cols, seed, stream):
    z = _np(nmf.gaussian_sketch(rows, cols, seed, stream))
    ref = philox.gaussian_matrix(rows, cols, seed, stream)
    np.testing.assert_allclose(z, ref, rtol=2e-6, atol=2e-6)


def _bf16_round(a):
    import torch
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


@pytest.mark.parametrize("n,m,k", [(300, 517, 20), (64, 64, 1), (129, 1000, 10), (1000, 77, 42), (5, 7, 3),
                                   (2000, 3000, 20), (3100, 2600, 42), (2500, 4100, 64), (4000, 1000, 10)])
@pytest.mark.parametrize("prec", [0, 1])
def test_dual_product(nmf, n, m, k, prec):
    rng = np.random.default_rng(n * 31 + m + k)
    X = rng.random((n, m)).astype(np.float32)
    A = rng.standard_normal((m, k)).astype(np.float32)
    B = rng.standard_normal((n, k)).astype(np.float32)
    YN, YT = nmf.dual_product(_t(X), _t(A), _t(B), prec=prec)
    Xd, Ad, Bd = X.astype(np.float64), A.astype(np.float64), B.astype(np.float64)
    if prec == 1:
        Xd, Ad, Bd = _bf16_round(X), _bf16_round(A), _bf16_round(B)
    refN, refT = Xd @ Ad, Xd.T @ Bd
    boundN = 4 * np.sqrt(m) * 2.0 ** -24 * (np.abs(Xd) @ np.abs(Ad)) + 1e-30
    boundT = 4 * np.sqrt(n) * 2.0 ** -24 * (np.abs(Xd).T @ np.abs(Bd)) + 1e-30
    assert np.all(np.abs(_np(YN) - refN) <= boundN)
    assert np.all(np.abs(_np(YT) - refT) <= boundT)
    # one product alone
    YN2, YT2 = nmf.dual_product(_t(X), _t(A), None, prec=prec)
    assert YT2 is None
    np.testing.assert_array_equal(_np(YN2), _np(YN))


@pytest.mark.parametrize("n,m,k", [(2000, 3000, 20), (1000, 77, 42), (3333, 2222, 64)])
def test_tensor_core_path_matches_cuda_core_path(nmf, n, m, k):
    # Same bfloat16 inputs on both kernels: only the float32 summation order differs.
    rng = np.random.default_rng(k)
    X = _t(rng.random((n, m)))
    A = _t(rng.standard_normal((m, k)))
    B = _t(rng.standard_normal((n, k)))
    tcN, tcT = nmf.dual_product(X, A, B, prec=1)
    nmf.set_kernel_path(True)
    try:
        scN, scT = nmf.dual_product(X, A, B, prec=1)
    finally:
        nmf.set_kernel_path(False)
    for a, b, K in ((tcN, scN, m), (tcT, scT, n)):
        a, b = _np(a), _np(b)
        scale = np.abs(b).max()
        assert np.max(np.abs(a - b)) <= 8 * np.sqrt(K) * 2.0 ** -24 * np.sqrt(K) * scale


@pytest.mark.parametrize("n,m,k", [(2000, 3000, 20), (129, 1000, 10), (5, 7, 3), (300, 517, 32), (640, 384, 16)])
def test_float32_tensor_core_path_matches_cuda_cores(nmf, n, m, k):
    # Float32 X and operands: the tensor cores take three bfloat16 parts of
    # each (up to 32 columns), the CUDA-core kernel plain float32. Both sit
    # inside the float32 bound of test_dual_product; their difference is the
    # two summation orders, bounded by twice that bound.
    rng = np.random.default_rng(n + 7 * m + k)
    X = rng.random((n, m)).astype(np.float32)
    A = rng.standard_normal((m, k)).astype(np.float32)
    B = rng.standard_normal((n, k)).astype(np.float32)
    tcN, tcT = nmf.dual_product(_t(X), _t(A), _t(B), prec=0)
    nmf.set_kernel_path(True)
    try:
        scN, scT = nmf.dual_product(_t(X), _t(A), _t(B), prec=0)
    finally:
        nmf.set_kernel_path(False)
    Xd, Ad, Bd = X.astype(np.float64), A.astype(np.float64), B.astype(np.float64)
    for got, alt, ref, absprod, K in ((tcN, scN, Xd @ Ad, np.abs(Xd) @ np.abs(Ad), m),
                                      (tcT, scT, Xd.T @ Bd, np.abs(Xd).T @ np.abs(Bd), n)):
        bound = 4 * np.sqrt(K) * 2.0 ** -24 * absprod + 1e-30
        got, alt = _np(got), _np(alt)
        assert np.all(np.abs(got - ref) <= bound)
        assert np.all(np.abs(alt - ref) <= bound)
        assert np.all(np.abs(got - alt) <= 2 * bound)
        # the three-part products are far closer than bfloat16 inputs would be
        assert np.max(np.abs(got - ref) / (absprod + 1e-30)) < 2.0 ** -20


def test_float32_tensor_core_path_keeps_small_residuals(nmf):
    # X = 1 + d with |d| ~ 2^-12: bfloat16 keeps only 1, the three parts keep
    # d to 2^-27; X A - 1 A isolates the residual part of the product.
    n, m, k = 256, 384, 8
    rng = np.random.default_rng(3)
    d = (rng.random((n, m)) * 2.0 ** -12).astype(np.float32)
    X = (np.float32(1.0) + d).astype(np.float32)
    A = rng.standard_normal((m, k)).astype(np.float32)
    YN, _ = nmf.dual_product(_t(X), _t(A), None, prec=0)
    Xd, Ad = X.astype(np.float64), A.astype(np.float64)
    ref = Xd @ Ad
    assert np.all(np.abs(_np(YN) - ref) <= 4 * np.sqrt(m) * 2.0 ** -24 * (np.abs(Xd) @ np.abs(Ad)))


def test_dual_product_is_deterministic(nmf):
    rng = np.random.default_rng(1)
    X = _t(rng.random((777, 555)))
    A = _t(rng.standard_normal((555, 24)))
    B = _t(rng.standard_normal((777, 24)))
    for prec in (1, 0):
        a1, b1 = nmf.dual_product(X, A, B, prec=prec)
        a2, b2 = nmf.dual_product(X, A, B, prec=prec)
        assert bool((a1 == a2).all()) and bool((b1 == b2).all())


@pytest.mark.parametrize("n,m,p", [(300, 200, 5), (1, 1, 1), (513, 257, 32)])
def test_rre_kernel(nmf, n, m, p):
    rng = np.random.default_rng(n + m + p)
    X = rng.random((n, m)).astype(np.float32)
    G = rng.random((n, p)).astype(np.float32)
    F = rng.random((p, m)).astype(np.float32) / p
    terms = _np(nmf.rre_terms(_t(X), _t(G), _t(F)))
    Xd, Gd, Fd = X.astype(np.float64), G.astype(np.float64), F.astype(np.float64)
    ref_e = np.sum((Xd - Gd @ Fd) ** 2)
    ref_x = np.sum(Xd ** 2)
    # per-entry residual error <= p * 2^-24 * sum|G F| + rounding of x: relative 1e-5 on the sums
    assert abs(terms[0] - ref_e) <= 1e-5 * ref_e + 1e-9
    assert abs(terms[1] - ref_x) <= 1e-7 * ref_x


def test_rre_kernel_beyond_the_grid_row_limit(nmf):
    # 64 x 65535 rows fill the grid's y extent; with 100 rows more, the last
    # block walks a second row block (the same fixed summation order per block).
    n, m, p = 64 * 65535 + 100, 3, 2
    rng = np.random.default_rng(17)
    X = rng.random((n, m)).astype(np.float32)
    G = rng.random((n, p)).astype(np.float32)
    F = rng.random((p, m)).astype(np.float32) / p
    terms = _np(nmf.rre_terms(_t(X), _t(G), _t(F)))
    Xd, Gd, Fd = X.astype(np.float64), G.astype(np.float64), F.astype(np.float64)
    ref_e = np.sum((Xd - Gd @ Fd) ** 2)
    ref_x = np.sum(Xd ** 2)
    assert abs(terms[0] - ref_e) <= 1e-5 * ref_e
    assert abs(terms[1] - ref_x) <= 1e-7 * ref_x
