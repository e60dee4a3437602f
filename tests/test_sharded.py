"""Row-sharded compressed NeNMF (paper_1812_04315_gb300.sharded) on CPU ranks.

Two gloo ranks (and, in one case, three with an uneven row split; spawned
processes, as torch.distributed.run launches them) split X by rows and run
the sharded schedule with a float64 numpy backend;
rank 0 gathers G and compares everything with the single-process oracle
(Alg. 2 by Householder QR, Alg. 1 by oracle.nenmf) on the same sketches:
bases, compressed data, the G and F trajectory and the inner-iteration
counts. Sharded CholeskyQR2 and Householder QR give the same Q to rounding
(diag(R) > 0 both), so the float64 runs agree to ~1e-12; a misplaced
all-reduce, a rank's block dropped or double counted, the stop test decided
on one rank's share, or a block's kept iterate taken at the wrong index all
fail. The same schedule on one GPU with the library's kernels is
tests/test_gpu_sharded.py; multi-GPU runs are not available here.
"""

import os
import socket

import numpy as np
import pytest
from scipy.linalg import solve_triangular

import synth
from oracle import nenmf, subspace
from paper_1812_04315_gb300 import sharded


class NumpyBackend:
    """float64 arithmetic on this rank's blocks (test-side stand-in for the GPU kernels)."""

    def dual(self, X, A, B):
        return (None if A is None else X @ A, None if B is None else X.T @ B)

    def gram(self, Y):
        return Y.T @ Y

    def apply(self, Y, S):
        U = np.linalg.cholesky(S).T                      # S = U^T U, U upper with a positive diagonal
        return solve_triangular(U, Y.T, trans="T", lower=False).T   # Y U^{-1}

    def mm(self, A, B):
        return A @ B

    def t(self, A):
        return np.ascontiguousarray(A.T)

    def copy(self, A):
        return np.array(A, copy=True)

    def nnls_block(self, H, B, Y, Fp, k0, kb, K):
        Lc = float(np.linalg.eigvalsh(H)[-1])
        beta = nenmf.extrapolation_weights(K)
        pg = lambda F: float(np.sum(nenmf.projected_gradient(F, H @ F - B) ** 2))
        if kb == 0 or Lc <= 0.0:
            return [], np.full(max(kb, 1), pg(Y)), np.array([Lc])
        keep, pg2 = [], []
        for i in range(kb):
            f = np.maximum(0.0, Y - (H @ Y - B) / Lc)
            pg2.append(pg(f))
            keep.append(f)
            Y[...] = f + beta[k0 + i] * (f - Fp)
            Fp[...] = f
        return keep, np.array(pg2), np.array([Lc])

    def host(self, x):
        return np.asarray(x, dtype=np.float64)

    def pick(self, keep, i):
        return np.array(keep[i], copy=True)


def _inputs(n, m, p, nu, seed):
    X, _, _ = synth.lowrank_data(n, m, p, seed=seed, snr_db=30.0)
    G0, F0 = synth.initial_factors(n, m, p, seed=seed + 1)
    rng = np.random.default_rng(seed + 2)
    return X, G0, F0, rng.standard_normal((m, nu)), rng.standard_normal((nu, n))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n, m, p, nu, qq, T, K, min_inner, tol, seed = case
        X, G0, F0, OmL, OmR = _inputs(n, m, p, nu, seed)
        r0, r1 = sharded.row_blocks(n, world)[rank]
        be, comm = NumpyBackend(), sharded.Collective()
        Lt_r, R, XLt, XR_r = sharded.compress(be, comm, X[r0:r1], nu, qq, OmL, OmR[:, r0:r1].T.copy())
        G_r, F, info = sharded.solve(be, comm, Lt_r, R, XLt, XR_r, G0[r0:r1].copy(), F0.copy(), T, K,
                                     min_inner, tol, record=True)
        # gather the row blocks (and every outer iteration's G) on every rank
        def gather(a):
            parts = [None] * world
            dist.all_gather_object(parts, a)
            return np.vstack(parts)
        out = {"Lt": gather(Lt_r), "R": R, "XLt": XLt, "XR": gather(XR_r), "G": gather(G_r), "F": F,
               "eps": info["eps"], "inner": info["inner"],
               "Ghist": [gather(g) for g, _ in info["history"]], "Fhist": [f for _, f in info["history"]]}
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def _run_ranks(case, world=2):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = dict(q.get(timeout=300) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    return got


CASES = [
    # n, m, p, nu, q, T, K, min_inner, tol, seed
    (121, 90, 4, 9, 2, 5, 10, 1, 0.0, 3),      # fixed inner counts, odd row split
    (160, 130, 5, 10, 1, 6, 40, 1, 1e-4, 7),   # stop test across blocks of 16
    (96, 150, 3, 7, 0, 4, 25, 3, 1e-3, 11),    # q = 0, min_inner, early stops
]


def _check_against_oracle(case, got, world):
    n, m, p, nu, qq, T, K, min_inner, tol, seed = case
    X, G0, F0, OmL, OmR = _inputs(n, m, p, nu, seed)
    L, R, XL, XR = subspace.compress(X, nu, qq, OmL, OmR)
    G, F, info = nenmf.nenmf_compressed(L, R, XL, XR, G0, F0, T, K, min_inner, tol, record=True)
    for rank in range(world):
        o = got[rank]
        np.testing.assert_allclose(o["Lt"], L.T, atol=1e-10)
        np.testing.assert_allclose(o["R"], R, atol=1e-10)
        np.testing.assert_allclose(o["XLt"], XL.T, atol=1e-9 * np.abs(XL).max())
        np.testing.assert_allclose(o["XR"], XR, atol=1e-9 * np.abs(XR).max())
        assert [tuple(x) for x in o["inner"]] == [tuple(x) for x in info["inner"]]
        if tol > 0:
            assert abs(o["eps"] - info["eps"]) <= 1e-10 * info["eps"]
        for (g, f), gs, fs in zip(info["history"], o["Ghist"], o["Fhist"]):
            np.testing.assert_allclose(gs, g, atol=1e-9 * np.abs(g).max())
            np.testing.assert_allclose(fs, f, atol=1e-9 * np.abs(f).max())
    # every rank holds the same replicated F
    for rank in range(1, world):
        np.testing.assert_array_equal(got[0]["F"], got[rank]["F"])


@pytest.mark.parametrize("case", CASES)
def test_two_ranks_match_the_oracle(case):
    _check_against_oracle(case, _run_ranks(case, 2), 2)


def test_three_ranks_uneven_rows_match_the_oracle():
    # 100 rows over three ranks (33, 33, 34), the stop test across blocks
    case = (100, 140, 4, 9, 1, 5, 30, 1, 1e-4, 19)
    _check_against_oracle(case, _run_ranks(case, 3), 3)


def test_row_blocks():
    assert sharded.row_blocks(10, 3) == [(0, 3), (3, 6), (6, 10)]
    assert sharded.row_blocks(5, 1) == [(0, 5)]
    with pytest.raises(ValueError):
        sharded.row_blocks(2, 3)
