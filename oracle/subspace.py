"""Randomized subspace iteration for NMF (Alg. 2), FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Shapes (Sec. 3): L is nu x n, R is m x nu, X_L = L X is nu x m, X_R = X R is
n x nu, with p <= nu << min(n, m).

Readings of points the paper leaves open:
  * an orthonormal basis from a QR decomposition = the Q factor of the thin
    Householder QR with the signs fixed so that diag(R) > 0 (unique when the
    input has full column rank). A wide input (nu x m, orthonormal rows
    wanted) is orthonormalised through its transpose.
  * Alg. 2's output step reads L = Q~_L^(q), R = Q~_R^(q), which has the wrong
    shapes (Q~_L^(q) is m x nu while L must be nu x n). The oracle takes the
    last full-step bases: L = (Q_L^(q))^T and R = (Q_R^(q))^T, so that
    L L^T = I and R^T R = I (Sec. 3 asks for orthonormal columns of one basis
    and rows of the other; here rows and columns are swapped to match the
    shapes).
"""

from __future__ import annotations

import numpy as np


def orthonormal_basis(Y: np.ndarray) -> np.ndarray:
    """Q of the thin QR Y = Q R with diag(R) >= 0 (Y tall: rows >= columns)."""
    Q, Rf = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
    s = np.sign(np.diag(Rf))
    s[s == 0.0] = 1.0
    return Q * s


def orthonormal_rows(Z: np.ndarray) -> np.ndarray:
    """Orthonormal basis of the row space of a wide Z, as rows (via Z^T)."""
    return orthonormal_basis(np.asarray(Z).T).T


def randomized_subspace_iteration(X, nu: int, q: int, Omega_L, Omega_R):
    """Alg. 2 with given Gaussian Omega_L (m x nu) and Omega_R (nu x n).

    Returns (L, R) with L = (Q_L^(q))^T (nu x n) and R = (Q_R^(q))^T (m x nu).
    """
    X = np.asarray(X, dtype=np.float64)
    n, m = X.shape
    Omega_L = np.asarray(Omega_L, dtype=np.float64)
    Omega_R = np.asarray(Omega_R, dtype=np.float64)
    if Omega_L.shape != (m, nu) or Omega_R.shape != (nu, n):
        raise ValueError("Omega_L must be m x nu and Omega_R nu x n")
    QL = orthonormal_basis(X @ Omega_L)          # Q_L^(0), n x nu
    QR = orthonormal_rows(Omega_R @ X)           # Q_R^(0), nu x m
    for _ in range(q):
        QtL = orthonormal_basis(X.T @ QL)        # Q~_L^(k), m x nu
        QtR = orthonormal_rows(QR @ X.T)         # Q~_R^(k), nu x n
        QL = orthonormal_basis(X @ QtL)          # Q_L^(k), n x nu
        QR = orthonormal_rows(QtR @ X)           # Q_R^(k), nu x m
    return QL.T, QR.T


def compress(X, nu: int, q: int, Omega_L, Omega_R):
    """L, R from Alg. 2, then X_L = L X and X_R = X R (the compression step of Alg. 1)."""
    X = np.asarray(X, dtype=np.float64)
    L, R = randomized_subspace_iteration(X, nu, q, Omega_L, Omega_R)
    return L, R, L @ X, X @ R


def gaussian_projection(Omega_L_rows, Omega_R_cols):
    """Plain random projection of Sec. 3 (footnote): L = Omega / sqrt(nu), R likewise.

    Omega_L_rows is nu x n, Omega_R_cols is m x nu.
    """
    nu = Omega_L_rows.shape[0]
    return np.asarray(Omega_L_rows) / np.sqrt(nu), np.asarray(Omega_R_cols) / np.sqrt(nu)


VARIANTS = ("subspace", "swapped", "single", "power", "gaussian")


def _unit_columns(Y: np.ndarray) -> np.ndarray:
    """Y with every column scaled to unit norm (the span is unchanged)."""
    nrm = np.linalg.norm(Y, axis=0)
    nrm[nrm == 0.0] = 1.0
    return Y / nrm


def compression_bases(X, nu: int, q: int, Omega_L, Omega_R, variant: str = "subspace"):
    """(L, R) of one compression variant, L nu x n and R m x nu.

    subspace  Alg. 2 as read in the module docstring (the default);
    swapped   Alg. 2's output step with the tildes swapped, the other
              dimensionally valid reading: L = Q~_R^(q) (nu x n, orthonormal
              rows), R = Q~_L^(q) (m x nu, orthonormal columns); needs q >= 1;
    single    one chain (Omega_L only): Q_L^(q) as in Alg. 2 gives L, and the
              next half-step basis orth(X^T Q_L^(q)) gives R;
    power     randomized power iteration (structured random projection,
              Sec. 3): the same products with no orthonormalisation between
              them, columns only rescaled to unit norm (span unchanged,
              magnitudes bounded), one orthonormalisation at the end;
    gaussian  plain random projection (Sec. 3 footnote): L = Omega_R / sqrt(nu)
              (nu x n), R = Omega_L / sqrt(nu) (m x nu), no pass over X.
    """
    X = np.asarray(X, dtype=np.float64)
    n, m = X.shape
    Omega_L = np.asarray(Omega_L, dtype=np.float64)
    Omega_R = np.asarray(Omega_R, dtype=np.float64)
    if Omega_L.shape != (m, nu) or Omega_R.shape != (nu, n):
        raise ValueError("Omega_L must be m x nu and Omega_R nu x n")
    if variant == "subspace":
        return randomized_subspace_iteration(X, nu, q, Omega_L, Omega_R)
    if variant == "swapped":
        if q < 1:
            raise ValueError("the swapped reading needs q >= 1")
        QL = orthonormal_basis(X @ Omega_L)
        QR = orthonormal_rows(Omega_R @ X)
        for _ in range(q):
            QtL = orthonormal_basis(X.T @ QL)
            QtR = orthonormal_rows(QR @ X.T)
            QL = orthonormal_basis(X @ QtL)
            QR = orthonormal_rows(QtR @ X)
        return QtR, QtL
    if variant == "single":
        QL = orthonormal_basis(X @ Omega_L)
        for _ in range(q):
            QL = orthonormal_basis(X @ orthonormal_basis(X.T @ QL))
        return QL.T, orthonormal_basis(X.T @ QL)
    if variant == "power":
        YL = _unit_columns(X @ Omega_L)              # n x nu
        YR = _unit_columns(X.T @ Omega_R.T)          # m x nu: the R chain transposed
        for _ in range(q):
            YL = _unit_columns(X @ _unit_columns(X.T @ YL))
            YR = _unit_columns(X.T @ _unit_columns(X @ YR))
        return orthonormal_basis(YL).T, orthonormal_basis(YR)
    if variant == "gaussian":
        return gaussian_projection(Omega_R, Omega_L)
    raise ValueError(f"unknown variant {variant!r}")


def compress_variant(X, nu: int, q: int, Omega_L, Omega_R, variant: str = "subspace"):
    """L, R of a variant, then X_L = L X and X_R = X R."""
    X = np.asarray(X, dtype=np.float64)
    L, R = compression_bases(X, nu, q, Omega_L, Omega_R, variant)
    return L, R, L @ X, X @ R
