"""Row-sharded compressed NeNMF: X split by row blocks across ranks, one GPU each.

The schedule of Alg. 2 and Alg. 1 when every rank holds rows r0 .. r1 - 1 of
X (n_r x m) and the collectives are sum all-reduces:

compression (Alg. 2, two chains, then the compression step of Alg. 1)
  * every pass over X is one local dual product: the N product X_r A with a
    replicated m x nu operand (rows of the result are local), the T product
    X_r^T B_r with this rank's rows of an n x nu operand (a partial sum);
  * the T product (m x nu) is all-reduced, then orthonormalised on every rank
    alike;
  * a row-sharded basis (n x nu) is orthonormalised by CholeskyQR2: each pass
    all-reduces the nu x nu Gram of the local rows and applies R^{-1} locally;
  * the closing pass gives X_R = X R (local rows) and X_L^T = X^T L^T
    (all-reduced once).

outer loop (Alg. 1)
  * F (p x m) is replicated: F_R = F R is formed on every rank;
  * the G update is local: the rows of G and X_R are this rank's; its stop
    test (Sec. 2) sums ||P grad||^2 over all rows, so the inner loop runs in
    blocks of up to 16 iterations that record each iteration's local share
    and iterate, one all-reduce of the block's shares decides, and the first
    passing iteration's iterate is taken, as the sequential rule takes it;
  * G_L = L G (nu x p) is all-reduced;
  * the F update is replicated (every rank solves the same problem).

eps of the relative stop rule: the G part of the initial projected gradient
is all-reduced, the F part is replicated. Adaptive restart is not offered
here. The arithmetic runs on a backend (CudaBackend: the library's kernels
through the C ABI on this rank's GPU); the collectives on a Collective
(torch.distributed, NCCL for CUDA tensors). No run here has more than one
GPU: this schedule is tested on CPU ranks (gloo) with a float64 backend and
on one GPU with CudaBackend; it is unmeasured on multi-GPU hardware.
"""

from __future__ import annotations

import math

STOP_BLOCK = 16


def row_blocks(n: int, world: int):
    """[(r0, r1)] of each rank: rows split as evenly as possible, in rank order."""
    if world < 1 or n < world:
        raise ValueError("need 1 <= world <= n")
    return [(r * n // world, (r + 1) * n // world) for r in range(world)]


class Collective:
    """Sum all-reduce over a torch.distributed process group (identity for one rank)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.group = group
        self.world = self.dist.get_world_size(group) if self.dist else 1
        self.rank = self.dist.get_rank(group) if self.dist else 0

    def all_reduce(self, x):
        """x summed over the ranks (a torch tensor, summed in place, or a numpy array)."""
        if self.world == 1:
            return x
        import numpy as np
        import torch
        if isinstance(x, np.ndarray):
            t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).copy())
            self.dist.all_reduce(t, group=self.group)
            return t.numpy()
        self.dist.all_reduce(x, group=self.group)
        return x


class CudaBackend:
    """Per-rank arithmetic on this rank's GPU through the library (float32 data)."""

    def __init__(self, prec: int = 0):
        from . import dual_product, gram, nnls_block, orth_apply
        self._dual, self._gram, self._apply, self._nnls = dual_product, gram, orth_apply, nnls_block
        self.prec = prec

    def dual(self, X, A, B):
        return self._dual(X.contiguous(), None if A is None else A.contiguous(),
                          None if B is None else B.contiguous(), prec=self.prec)

    def gram(self, Y):
        return self._gram(Y.contiguous())

    def apply(self, Y, S):
        return self._apply(Y.contiguous(), S.contiguous())

    def mm(self, A, B):
        # a small product A B as the N product of one pass over A (float32)
        return self._dual(A.contiguous(), B.contiguous(), None, prec=0)[0]

    def t(self, A):
        return A.t().contiguous()

    def copy(self, A):
        return A.clone()

    def nnls_block(self, H, B, Y, Fp, k0, kb, K):
        return self._nnls(H.contiguous(), B.contiguous(), Y, Fp, k0, kb, K)

    def host(self, x):
        return x.double().cpu().numpy()

    def pick(self, keep, i):
        return keep[i].clone()


def _orth_sharded(be, comm, Y):
    """CholeskyQR2 of a row-sharded tall matrix: two passes, each with its Gram all-reduced."""
    for _ in range(2):
        Y = be.apply(Y, comm.all_reduce(be.gram(Y)))
    return Y


def _orth_local(be, Y):
    for _ in range(2):
        Y = be.apply(Y, be.gram(Y))
    return Y


def compress(be, comm, X_r, nu: int, q: int, omega_L, omega_R_r):
    """Alg. 2 and the compression step of Alg. 1 on this rank's rows X_r (n_r x m).

    omega_L: m x nu (the same on every rank); omega_R_r: this rank's columns of
    Omega_R, transposed (n_r x nu). Returns (Lt_r, R, XLt, XR_r): this rank's
    rows of L^T (n_r x nu), R (m x nu), X_L^T (m x nu, all-reduced) and this
    rank's rows of X_R (n_r x nu).
    """
    YN, YT = be.dual(X_r, omega_L, omega_R_r)          # X Omega_L, X^T Omega_R^T (partial)
    QL = _orth_sharded(be, comm, YN)                   # Q_L^(0), local rows
    QRt = _orth_local(be, comm.all_reduce(YT))         # (Q_R^(0))^T, m x nu
    for _ in range(q):
        YN, YT = be.dual(X_r, QRt, QL)                 # X Q_R^T -> Q~_R^T; X^T Q_L -> Q~_L
        QtL = _orth_local(be, comm.all_reduce(YT))
        QtRt = _orth_sharded(be, comm, YN)
        YN, YT = be.dual(X_r, QtL, QtRt)               # X Q~_L -> Q_L; X^T Q~_R^T -> Q_R^T
        QL = _orth_sharded(be, comm, YN)
        QRt = _orth_local(be, comm.all_reduce(YT))
    XR_r, XLt = be.dual(X_r, QRt, QL)                  # X R (local rows), X^T L^T (partial)
    return QL, QRt, comm.all_reduce(XLt), XR_r


def nnls(be, comm, H, B, Y0, max_inner: int, min_inner: int = 1, eps: float | None = None):
    """The inner loop of Sec. 2 on the columns of Y0 (p x N_r); with comm, the
    stop test sums ||P grad||^2 over the ranks' columns. Returns (F, iterations)."""
    Y, Fp = be.copy(Y0), be.copy(Y0)
    k0, last = 0, None
    while k0 < max_inner:
        kb = min(STOP_BLOCK, max_inner - k0)
        keep, pg2, lc = be.nnls_block(H, B, Y, Fp, k0, kb, max_inner)
        if float(be.host(lc)[0]) <= 0.0:
            return be.copy(Y0), 0
        if eps is not None:
            tot = be.host(pg2 if comm is None else comm.all_reduce(pg2))
            for i in range(kb):
                if k0 + i + 1 >= min_inner and math.sqrt(max(float(tot[i]), 0.0)) <= eps:
                    return be.pick(keep, i), k0 + i + 1
        last = be.pick(keep, kb - 1)
        k0 += kb
    return last, max_inner


def _pg2_at(be, H, B, Y):
    """||P grad||^2 at Y of 1/2 tr(Y^T H Y) - tr(B^T Y) over these columns (no step taken)."""
    _, pg2, _ = be.nnls_block(H, B, be.copy(Y), be.copy(Y), 0, 0, 1)
    return pg2


def solve(be, comm, Lt_r, R, XLt, XR_r, G_r, F, max_outer: int, max_inner: int, min_inner: int = 1,
          tol: float = 0.0, record: bool = False):
    """Alg. 1 on the compressed data with this rank's rows of G, X_R and L^T.

    Returns (G_r, F, info): info["eps"], info["inner"] (per outer iteration the
    G and F inner counts), info["history"] ((G_r, F) after each outer
    iteration when `record`).
    """
    # products keep their right operand narrow (<= nu or p columns):
    #   H_G = F_R F_R^T, B_G = (X_R F_R^T)^T; H_F = G_L^T G_L, B_F = (X_L^T G_L)^T
    L_r = be.t(Lt_r)

    def g_side(F):
        FR = be.mm(F, R)                                        # p x nu, replicated
        return be.mm(FR, be.t(FR)), be.t(be.mm(XR_r, be.t(FR)))

    def f_side(G_r):
        GL = comm.all_reduce(be.mm(L_r, G_r))                   # nu x p, all-reduced
        return be.mm(be.t(GL), GL), be.t(be.mm(XLt, GL))

    eps = None
    if tol and tol > 0:
        Hg, Bg = g_side(F)
        pgG = be.host(comm.all_reduce(_pg2_at(be, Hg, Bg, be.t(G_r))))[0]
        Hf, Bf = f_side(G_r)
        pgF = be.host(_pg2_at(be, Hf, Bf, F))[0]
        eps = float(tol) * math.sqrt(float(pgG) + float(pgF))
    info = {"eps": eps, "inner": [], "history": []}
    for _ in range(max_outer):
        Hg, Bg = g_side(F)
        Gt, kG = nnls(be, comm, Hg, Bg, be.t(G_r), max_inner, min_inner, eps)
        G_r = be.t(Gt)
        Hf, Bf = f_side(G_r)
        F, kF = nnls(be, None, Hf, Bf, F, max_inner, min_inner, eps)
        info["inner"].append((kG, kF))
        if record:
            info["history"].append((be.copy(G_r), be.copy(F)))
    return G_r, F, info
