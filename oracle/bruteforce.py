"""Exhaustive nonnegative least squares for tiny problems (a pin for the oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

min_{f >= 0} 1/2 f^T H f - b^T f with H symmetric positive definite has one
minimiser, characterised by the KKT conditions: on the passive set P
(f_P > 0) the gradient vanishes, H_PP f_P = b_P; on the rest f = 0 and the
gradient (H f - b) is >= 0. Enumerating all 2^p passive sets and keeping the
one that satisfies these conditions gives the minimiser with no iteration at
all, so it is independent of the Nesterov loop it checks.
"""

from __future__ import annotations

import itertools

import numpy as np


def nnls_enumerate(H: np.ndarray, b: np.ndarray, rtol: float = 1e-10) -> np.ndarray:
    H = np.asarray(H, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    p = b.size
    scale = max(1.0, float(np.max(np.abs(b))), float(np.max(np.abs(H))))
    best = None
    best_obj = np.inf
    for size in range(p + 1):
        for P in itertools.combinations(range(p), size):
            f = np.zeros(p)
            if P:
                idx = list(P)
                f[idx] = np.linalg.solve(H[np.ix_(idx, idx)], b[idx])
                if np.any(f[idx] <= 0.0):
                    continue
            g = H @ f - b
            Z = [i for i in range(p) if i not in P]
            if Z and np.any(g[Z] < -rtol * scale):
                continue
            obj = 0.5 * f @ H @ f - b @ f
            if obj < best_obj:
                best, best_obj = f, obj
    if best is None:
        raise RuntimeError("no KKT point found (H not positive definite?)")
    return best


def nnls_enumerate_columns(H: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Column-wise minimiser for B with several right-hand sides (p x N)."""
    B = np.asarray(B, dtype=np.float64)
    return np.stack([nnls_enumerate(H, B[:, j]) for j in range(B.shape[1])], axis=1)
