"""Entry-wise comparison helpers shared by the GPU parity tests.

* entrywise: |got - ref| <= tol (|ref| + s), s the root-mean-square of ref.
  An entry's float32 rounding error scales with the terms that make it, and
  for an entry that is small by cancellation (or held at 0 by a projection
  on one side only) those terms are of the array's scale, not the entry's.
* product_bound: a float32 dot product of length K has error below
  K u sum|a_i b_i| (u = 2^-24) in the worst case; with rounding errors of
  random sign the tests take 4 sqrt(K) u sum|a_i b_i| per entry, which any
  fixed summation order (split-K included) meets with a wide margin.
"""

import numpy as np


def bf16_round(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def entrywise_ratio(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    s = np.sqrt(np.mean(ref * ref)) if ref.size else 0.0
    return float((np.abs(got - ref) / (np.abs(ref) + s + 1e-300)).max()) if ref.size else 0.0


def assert_entrywise(got, ref, tol, what=""):
    r = entrywise_ratio(got, ref)
    assert r <= tol, (what, r, tol)


def assert_product(got, A, B, what=""):
    """got ~= A @ B (float64 A, B: the operands the kernel multiplied) within the dot-product bound."""
    K = A.shape[1]
    ref = A @ B
    bound = 4 * np.sqrt(K) * 2.0 ** -24 * (np.abs(A) @ np.abs(B)) + 1e-30
    worst = float((np.abs(np.asarray(got, dtype=np.float64) - ref) / bound).max())
    assert worst <= 1.0, (what, worst)
