"""Reverse-mode derivative of unrolled compressed NeNMF (Alg. 1 with the inner loop of Sec. 2), FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring): the CUDA library never
imports this module.

The differentiated map is (X_L, X_R, G0, F0) -> (G_T, F_T): T outer
iterations of Alg. 1, each inner solve run for exactly K iterations (no stop
test), with L and R held fixed (they enter as constants; X reaches the map
only through X_L = L X and X_R = X R, so dX = L^T dX_L + dX_R R^T).

Readings (the paper gives no derivative; these are the standard ones):
  * max(0, z) has derivative 1[z > 0], so 0 at z = 0;
  * L_c = lambda_max(H) has derivative v v^T for the unit eigenvector v of a
    simple largest eigenvalue;
  * everything else is differentiated exactly, step by step in the order the
    forward computes it.

Inner loop (nesterov_nnls with K iterations, columns of a p x N unknown):
    z_k = Y_k - (H Y_k - B) / L_c,   F_k = max(0, z_k),
    Y_{k+1} = F_k + beta_k (F_k - F_{k-1}),   F_{-1} = Y_0,   output F_{K-1}.
Its adjoint runs k = K-1 .. 0:
    dF_k += (1 + beta_k) dY_{k+1};  dF_{k-1} += -beta_k dY_{k+1};
    dz_k = 1[z_k > 0] dF_k;
    dY_k = dz_k - H dz_k / L_c;  dH -= dz_k Y_k^T / L_c;  dB += dz_k / L_c;
    dL_c += <H Y_k - B, dz_k> / L_c^2 = <Y_k - z_k, dz_k> / L_c;
and dY_0 gains dF_{-1}; finally dH += dL_c v v^T. H is symmetric by
construction (W W^T), so only the symmetric part of dH carries meaning; it
reaches W as (dH + dH^T) W.
"""

from __future__ import annotations

import numpy as np

from .nenmf import extrapolation_weights, lipschitz_constant


def top_eigenvector(H: np.ndarray) -> np.ndarray:
    """Unit eigenvector of the largest eigenvalue of the symmetric H."""
    return np.linalg.eigh(H)[1][:, -1]


def nnls_forward(H, B, Y0, K: int):
    """K iterations of the inner loop; returns (F_{K-1}, tape)."""
    H = np.asarray(H, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    Y = np.array(Y0, dtype=np.float64, copy=True)
    Lc = lipschitz_constant(H)
    if Lc <= 0.0:
        return Y, {"Lc": 0.0}
    beta = extrapolation_weights(K)
    F_prev = Y.copy()
    Ys, zs = [], []
    F_k = Y
    for k in range(K):
        z = Y - (H @ Y - B) / Lc
        F_k = np.maximum(0.0, z)
        Ys.append(Y)
        zs.append(z)
        Y = F_k + beta[k] * (F_k - F_prev)
        F_prev = F_k
    return F_k, {"Lc": Lc, "beta": beta, "Y": Ys, "z": zs}


def nnls_adjoint(H, B, tape, dOut):
    """(dY_0, dH, dB) of the inner loop given dOut = d/dF_{K-1}."""
    H = np.asarray(H, dtype=np.float64)
    dOut = np.asarray(dOut, dtype=np.float64)
    Lc = tape["Lc"]
    if Lc <= 0.0:
        # zero iterations: the output is Y_0 itself
        return dOut.copy(), np.zeros_like(H), np.zeros_like(np.asarray(B, dtype=np.float64))
    beta, Ys, zs = tape["beta"], tape["Y"], tape["z"]
    K = len(zs)
    dF = [np.zeros_like(dOut) for _ in range(K)]
    dF[K - 1] = dOut.copy()
    dF_minus1 = np.zeros_like(dOut)
    dY_next = np.zeros_like(dOut)      # adjoint of Y_K, which the output does not use
    dH = np.zeros_like(H)
    dB = np.zeros_like(dOut)
    dL = 0.0
    for k in range(K - 1, -1, -1):
        dF[k] += (1.0 + beta[k]) * dY_next
        if k >= 1:
            dF[k - 1] -= beta[k] * dY_next
        else:
            dF_minus1 -= beta[k] * dY_next
        dz = np.where(zs[k] > 0.0, dF[k], 0.0)
        dY_next = dz - H @ dz / Lc
        dH -= dz @ Ys[k].T / Lc
        dB += dz / Lc
        dL += float(np.sum((Ys[k] - zs[k]) * dz)) / Lc
    v = top_eigenvector(H)
    dH += dL * np.outer(v, v)
    return dY_next + dF_minus1, dH, dB


def compressed_forward(L, R, XL, XR, G0, F0, T: int, K: int):
    """Alg. 1 for T outer iterations of K inner iterations; returns (G_T, F_T, tape)."""
    L, R, XL, XR = (np.asarray(a, dtype=np.float64) for a in (L, R, XL, XR))
    G = np.array(G0, dtype=np.float64, copy=True)
    F = np.array(F0, dtype=np.float64, copy=True)
    tape = []
    for _ in range(T):
        FR = F @ R                               # p x nu
        HG, BG = FR @ FR.T, FR @ XR.T            # the G problem as columns of G^T
        Gt, tG = nnls_forward(HG, BG, G.T, K)
        Gn = Gt.T
        GL = L @ Gn                              # nu x p
        HF, BF = GL.T @ GL, GL.T @ XL
        Fn, tF = nnls_forward(HF, BF, F, K)
        tape.append(dict(F=F, FR=FR, HG=HG, BG=BG, tG=tG, GL=GL, HF=HF, BF=BF, tF=tF))
        G, F = Gn, Fn
    return G, F, tape


def compressed_backward(L, R, XL, XR, tape, dG_T, dF_T):
    """(dX_L, dX_R, dG0, dF0) given the cotangents of (G_T, F_T)."""
    L, R, XL, XR = (np.asarray(a, dtype=np.float64) for a in (L, R, XL, XR))
    dG = np.array(dG_T, dtype=np.float64, copy=True)
    dF = np.array(dF_T, dtype=np.float64, copy=True)
    dXL = np.zeros_like(XL)
    dXR = np.zeros_like(XR)
    for s in reversed(tape):
        # F update: F_new = inner(H_F, B_F, F), H_F = G_L^T G_L, B_F = G_L^T X_L, G_L = L G_new
        dF_old, dHF, dBF = nnls_adjoint(s["HF"], s["BF"], s["tF"], dF)
        GL = s["GL"]
        dGL = GL @ (dHF + dHF.T) + XL @ dBF.T
        dXL += GL @ dBF
        dG = dG + L.T @ dGL
        # G update: G_new^T = inner(H_G, B_G, G^T), H_G = F_R F_R^T, B_G = F_R X_R^T, F_R = F R
        dGt_old, dHG, dBG = nnls_adjoint(s["HG"], s["BG"], s["tG"], dG.T)
        FR = s["FR"]
        dFR = (dHG + dHG.T) @ FR + dBG @ XR
        dXR += dBG.T @ FR
        dF = dF_old + dFR @ R.T
        dG = dGt_old.T
    return dXL, dXR, dG, dF


def loss_and_gradient(X, L, R, G0, F0, T: int, K: int):
    """loss = ||X - G_T F_T||_F^2 with X_L = L X, X_R = X R (L, R fixed) and its
    gradient with respect to (X, G0, F0)."""
    X, L, R = (np.asarray(a, dtype=np.float64) for a in (X, L, R))
    XL, XR = L @ X, X @ R
    G, F, tape = compressed_forward(L, R, XL, XR, G0, F0, T, K)
    E = X - G @ F
    loss = float(np.sum(E * E))
    dXL, dXR, dG0, dF0 = compressed_backward(L, R, XL, XR, tape, -2.0 * E @ F.T, -2.0 * G.T @ E)
    dX = 2.0 * E + L.T @ dXL + dXR @ R.T
    return loss, dX, dG0, dF0


def projection_signs(X, L, R, G0, F0, T: int, K: int):
    """Signs of every z_k of the forward (which projections are active): the
    map is smooth wherever these do not change."""
    X, L, R = (np.asarray(a, dtype=np.float64) for a in (X, L, R))
    _, _, tape = compressed_forward(L, R, L @ X, X @ R, G0, F0, T, K)
    out = []
    for s in tape:
        for t in (s["tG"], s["tF"]):
            out.extend((z > 0.0) for z in t.get("z", []))
    return out
