"""NeNMF and compressed NeNMF, FP64, following the paper step by step.

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never
imports this module.

Notation (Sec. 1-3): X is n x m and nonnegative, G is n x p, F is p x m,
X ~= G F (eq. 1). NeNMF alternately solves eq. (2) for G and eq. (3) for F,
each with an inner Nesterov loop (Sec. 2). Compressed NeNMF (Alg. 1) solves
eq. (2) with X, F replaced by X_R = X R, F_R = F R, and eq. (3) with X, G
replaced by X_L = L X, G_L = L G.

Every inner subproblem is written in one form: columns of an unknown p x N
matrix are independent nonnegative least-squares problems
    min_{F >= 0}  1/2 ||X - G F||_F^2,
whose gradient is  grad = H F - B  with  H = G^T G  (p x p),  B = G^T X.
The G-subproblem of eq. (2) is put in this form by transposition:
    min_{G >= 0} 1/2 ||X - G F||^2 = min_{G^T >= 0} 1/2 ||X^T - F^T G^T||^2,
so  H = F F^T  and  B = F X^T, and the unknown is G^T.

Readings of points the paper leaves open:
  * step size 1/L_c with L_c = lambda_max(H), the Lipschitz constant of the
    gradient (Sec. 2 cites Guan et al. 2012, whose step this is);
  * the inner loop returns the projected iterate F_k, not Y_K (the text's
    "F^{t+1} = Y_K" would break F >= 0 of eq. 3);
  * alpha and Y restart at every inner solve (Sec. 2: Y_0 = F^t, alpha_0 = 1);
  * projected gradient P_ij = grad_ij if F_ij > 0 else min(0, grad_ij), tested
    at the returned F_k as ||P||_F <= eps once k+1 >= min_inner; tol <= 0
    switches the test off;
  * eps = tol * ||[P grad_G ; P grad_F]||_F at the initial (G0, F0) of the
    objective being solved ("rel"), or eps = tol ("abs");
  * if H == 0 (lambda_max = 0) the subproblem is constant and Y_0 is returned
    after zero iterations;
  * adaptive restart (the remedy the paper suggests for non-monotone RRE,
    after O'Donoghue and Candes 2015), optional, function-value scheme per
    column: the columns are independent problems, so each column tracks its
    own objective f_j(F_k) = 1/2 F_k^T H F_k - B_j^T F_k and, when it rises
    (k >= 1), drops its momentum: that extrapolation uses beta_0 = 0 and
    the column's weights start again from beta_1. A rise counts when it
    exceeds RESTART_TOL times the objective's term scale
    sum_c |F_c| (|grad_c| + |B_c|), so that rounding of a float32
    evaluation near convergence does not trigger it.
"""

from __future__ import annotations

import numpy as np


RESTART_TOL = 1e-5


def alpha_sequence(K: int) -> np.ndarray:
    """alpha_0 = 1, alpha_{k+1} = (1 + sqrt(4 alpha_k^2 + 1)) / 2 (Sec. 2); K+1 values."""
    a = [1.0]
    for _ in range(K):
        a.append((1.0 + np.sqrt(4.0 * a[-1] * a[-1] + 1.0)) / 2.0)
    return np.array(a)


def extrapolation_weights(K: int) -> np.ndarray:
    """beta_k = (alpha_k - 1) / alpha_{k+1}, the weight sliding F_k away from F_{k-1} (Sec. 2)."""
    a = alpha_sequence(K + 1)
    return (a[:-1] - 1.0) / a[1:]


def lipschitz_constant(H: np.ndarray) -> float:
    """L_c = largest eigenvalue of the symmetric PSD Gram matrix H."""
    return float(np.linalg.eigvalsh(H)[-1])


def projected_gradient(F: np.ndarray, grad: np.ndarray) -> np.ndarray:
    """KKT projected gradient: grad where F > 0, min(0, grad) where F == 0."""
    return np.where(F > 0.0, grad, np.minimum(grad, 0.0))


def nesterov_nnls(H, B, Y0, max_inner: int, min_inner: int = 1, eps: float | None = None,
                  restart: bool = False, trace: list | None = None):
    """Inner Nesterov loop of NeNMF (Sec. 2) for min_{F>=0} 1/2 ||X - G F||^2.

    H = G^T G (p x p), B = G^T X (p x N), Y0 = F^t (p x N).
    With `restart`, a column whose objective rises drops its momentum (see
    the module docstring). `trace`, if given, receives per iteration the
    column objectives and the restart mask.
    Returns (F, iterations, ||P grad(F)||_F).
    """
    if max_inner < 1:
        raise ValueError("max_inner must be >= 1")
    H = np.asarray(H, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    Y = np.array(Y0, dtype=np.float64, copy=True)
    Lc = lipschitz_constant(H)
    if Lc <= 0.0:
        return Y, 0, float(np.linalg.norm(projected_gradient(Y, -B)))
    beta = extrapolation_weights(max_inner)   # beta_k = (alpha_k - 1) / alpha_{k+1}
    F_prev = Y.copy()            # F_{-1}; irrelevant because beta_0 = 0
    F_k = Y
    r = np.zeros(Y.shape[1], dtype=np.int64)   # per column: iterations since its last restart
    obj_prev = None
    for k in range(max_inner):
        grad_Y = H @ Y - B                           # gradient at Y_k
        F_k = np.maximum(0.0, Y - grad_Y / Lc)       # one projected gradient step
        if restart:
            grad_F = H @ F_k - B
            obj = 0.5 * np.sum(F_k * (H @ F_k), axis=0) - np.sum(B * F_k, axis=0)
            scale = np.sum(np.abs(F_k) * (np.abs(grad_F) + np.abs(B)), axis=0)
            rising = ((obj - obj_prev > RESTART_TOL * scale) if obj_prev is not None
                      else np.zeros_like(obj, dtype=bool))
            r[rising] = 0
            if trace is not None:
                trace.append((obj, rising))
            obj_prev = obj
        Y = F_k + beta[r] * (F_k - F_prev)           # slide away from F_{k-1}
        r += 1
        F_prev = F_k
        if eps is not None and k + 1 >= min_inner:
            pg = float(np.linalg.norm(projected_gradient(F_k, H @ F_k - B)))
            if pg <= eps:
                return F_k, k + 1, pg
    pg = float(np.linalg.norm(projected_gradient(F_k, H @ F_k - B)))
    return F_k, max_inner, pg


def _threshold(tol: float, tol_mode: str, initial_pg: float) -> float | None:
    if tol is None or tol <= 0.0:
        return None
    if tol_mode == "abs":
        return float(tol)
    if tol_mode == "rel":
        return float(tol) * initial_pg
    raise ValueError("tol_mode must be 'rel' or 'abs'")


def initial_pg_parts_plain(X, G, F):
    """(P grad_G, P grad_F) of 1/2||X - GF||^2 at (G, F): n x p and p x m."""
    gG = G @ (F @ F.T) - X @ F.T
    gF = (G.T @ G) @ F - G.T @ X
    return projected_gradient(G, gG), projected_gradient(F, gF)


def initial_pg_parts_compressed(L, R, XL, XR, G, F):
    """(P grad_G, P grad_F) of the two compressed objectives of Alg. 1 at (G, F):
    1/2||X_R - G F R||^2 in G and 1/2||X_L - L G F||^2 in F."""
    FR = F @ R
    gG = G @ (FR @ FR.T) - XR @ FR.T
    GL = L @ G
    gF = (GL.T @ GL) @ F - GL.T @ XL
    return projected_gradient(G, gG), projected_gradient(F, gF)


def _joint_norm(parts) -> float:
    return float(np.sqrt(sum(np.sum(a * a) for a in parts)))


def initial_pg_plain(X, G, F) -> float:
    """||[P grad_G ; P grad_F]||_F of 1/2||X - GF||^2 at (G, F)."""
    return _joint_norm(initial_pg_parts_plain(X, G, F))


def initial_pg_compressed(L, R, XL, XR, G, F) -> float:
    """Same norm for the compressed objectives of Alg. 1 at (G, F)."""
    return _joint_norm(initial_pg_parts_compressed(L, R, XL, XR, G, F))


def nenmf_plain(X, G0, F0, max_outer: int, max_inner: int, min_inner: int = 1,
                tol: float = 0.0, tol_mode: str = "rel", record: bool = False, restart: bool = False):
    """Plain NeNMF: alternate eq. (2) then eq. (3), each by the Nesterov loop.

    Returns (G, F, info); info["history"] holds (G, F) after every outer
    iteration when `record` is set.
    """
    X = np.asarray(X, dtype=np.float64)
    G = np.array(G0, dtype=np.float64, copy=True)
    F = np.array(F0, dtype=np.float64, copy=True)
    eps = _threshold(tol, tol_mode, initial_pg_plain(X, G, F) if tol and tol > 0 else 0.0)
    info = {"eps": eps, "inner": [], "history": []}
    for _ in range(max_outer):
        # eq. (2) with F fixed, as a problem in G^T: H = F F^T, B = F X^T.
        Gt, kG, _ = nesterov_nnls(F @ F.T, F @ X.T, G.T, max_inner, min_inner, eps, restart)
        G = Gt.T
        # eq. (3) with G fixed: H = G^T G, B = G^T X.
        F, kF, _ = nesterov_nnls(G.T @ G, G.T @ X, F, max_inner, min_inner, eps, restart)
        info["inner"].append((kG, kF))
        if record:
            info["history"].append((G.copy(), F.copy()))
    return G, F, info


def nenmf_compressed(L, R, XL, XR, G0, F0, max_outer: int, max_inner: int, min_inner: int = 1,
                     tol: float = 0.0, tol_mode: str = "rel", record: bool = False, restart: bool = False):
    """Compressed NeNMF, Alg. 1: X_L = L X and X_R = X R are given.

    repeat: F_R = F R; solve eq. (2) with (X, F) -> (X_R, F_R);
            G_L = L G; solve eq. (3) with (X, G) -> (X_L, G_L).
    """
    L = np.asarray(L, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    XL = np.asarray(XL, dtype=np.float64)
    XR = np.asarray(XR, dtype=np.float64)
    G = np.array(G0, dtype=np.float64, copy=True)
    F = np.array(F0, dtype=np.float64, copy=True)
    eps = _threshold(tol, tol_mode,
                     initial_pg_compressed(L, R, XL, XR, G, F) if tol and tol > 0 else 0.0)
    info = {"eps": eps, "inner": [], "history": []}
    for _ in range(max_outer):
        FR = F @ R                                                   # p x nu
        Gt, kG, _ = nesterov_nnls(FR @ FR.T, FR @ XR.T, G.T, max_inner, min_inner, eps, restart)
        G = Gt.T
        GL = L @ G                                                   # nu x p
        F, kF, _ = nesterov_nnls(GL.T @ GL, GL.T @ XL, F, max_inner, min_inner, eps, restart)
        info["inner"].append((kG, kF))
        if record:
            info["history"].append((G.copy(), F.copy()))
    return G, F, info
