"""GPU parity of nenmf_solve_batched (many compressed problems, Alg. 1) against the FP64 oracle.

Every problem of a batch gets its own float32 L, R, X_L, X_R (the oracle's
Alg. 2 on the problem's X) and initial factors. Per problem the batched
result is compared with the oracle's compressed NeNMF on the same float32
inputs: final RRE (eq. 4) within 1e-5 (the float32 tolerance); after one
outer iteration the factors within 1e-4 relative (float32 rounding through
<= 10 Nesterov steps); with the stop test on, eps and the inner-iteration
counts (a count may move by one where a test sits at the threshold).
"""

import numpy as np
import pytest

from _parity import assert_entrywise
import synth
from oracle import metrics, nenmf, subspace

pytestmark = pytest.mark.gpu

# uneven shapes: (n, m, p, nu, q)
SHAPES = [(120, 90, 3, 8, 1), (333, 200, 6, 10, 2), (64, 500, 5, 9, 1), (257, 129, 12, 20, 2),
          (40, 41, 1, 4, 1), (300, 310, 16, 26, 1), (1, 37, 1, 1, 1)]


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _problem_inputs(n, m, p, nu, q, seed):
    X, _, _ = synth.lowrank_data(n, m, p, seed=seed, snr_db=20.0, dtype=np.float32)
    G0, F0 = synth.initial_factors(n, m, p, seed=seed + 1)
    OmL, OmR = synth.gaussian_sketches(n, m, nu, seed=seed + 2)
    L, R, XL, XR = (a.astype(np.float32) for a in subspace.compress(X.astype(np.float64), nu, q, OmL, OmR))
    return dict(X=X, G0=G0.astype(np.float32), F0=F0.astype(np.float32), L=L, R=R, XL=XL, XR=XR, p=p)


@pytest.fixture(scope="module")
def batch():
    return [_problem_inputs(*s, seed=17 * i + 3) for i, s in enumerate(SHAPES)]


def _run(nmf, batch, T, inner, tol=0.0, cluster=0, min_inner=1, restart=False):
    probs, Gs, Fs = [], [], []
    for b in batch:
        probs.append(nmf.compressed_problem(_t(b["L"]), _t(b["R"]), _t(b["XL"]), _t(b["XR"]), b["p"]))
        Gs.append(_t(b["G0"]))
        Fs.append(_t(b["F0"]))
    st = nmf.solve_batched(probs, Gs, Fs, T, inner, min_inner=min_inner, tol=tol, cluster=cluster, restart=restart)
    return Gs, Fs, nmf.read_batch_stats(st, len(batch))


def _oracle(b, T, inner, tol=0.0, min_inner=1, restart=False):
    return nenmf.nenmf_compressed(b["L"], b["R"], b["XL"], b["XR"], b["G0"], b["F0"], T, inner,
                                  min_inner=min_inner, tol=tol, restart=restart)


@pytest.mark.parametrize("T,inner,tol", [(8, 10, 0.0), (8, 10, 1e-3), (5, 40, 1e-6), (4, 20, 0.0), (6, 1, 0.0)])
def test_batched_matches_oracle(nmf, batch, T, inner, tol):
    Gs, Fs, stats = _run(nmf, batch, T, inner, tol)
    for b, G, F, st in zip(batch, Gs, Fs, stats):
        assert st.status == 0 and st.outer_done == T
        Go, Fo, info = _oracle(b, T, inner, tol)
        Xd = b["X"].astype(np.float64)
        r_gpu = metrics.rre(Xd, _np(G), _np(F))
        r_ora = metrics.rre(Xd, Go, Fo)
        assert abs(r_gpu - r_ora) <= 1e-5, (b["X"].shape, r_gpu, r_ora)
        assert (_np(G) >= 0).all() and (_np(F) >= 0).all()
        if tol > 0:
            assert st.eps == pytest.approx(info["eps"], rel=1e-4)
            ora = sum(a + c for a, c in info["inner"])
            assert abs(st.total_inner[0] + st.total_inner[1] - ora) <= 2
        else:
            assert st.total_inner[0] == T * inner and st.total_inner[1] == T * inner


@pytest.mark.parametrize("T,inner,tol", [(6, 10, 0.0), (4, 40, 1e-6)])
def test_batched_adaptive_restart_matches_oracle(nmf, batch, T, inner, tol):
    Gs, Fs, stats = _run(nmf, batch, T, inner, tol, restart=True)
    for b, G, F, st in zip(batch, Gs, Fs, stats):
        assert st.status == 0
        Go, Fo, _ = _oracle(b, T, inner, tol, restart=True)
        Xd = b["X"].astype(np.float64)
        assert abs(metrics.rre(Xd, _np(G), _np(F)) - metrics.rre(Xd, Go, Fo)) <= 1e-5


def test_batched_first_outer_iteration_factors(nmf, batch):
    Gs, Fs, _ = _run(nmf, batch, 1, 10)
    for b, G, F in zip(batch, Gs, Fs):
        Go, Fo, _ = _oracle(b, 1, 10)
        # per entry, as for nenmf_solve (tests/test_gpu_solve.py): float32 rounding of the
        # O(p)-term gradients through <= 10 non-expansive steps, at the factor's scale
        assert_entrywise(_np(G), Go, 1e-4, "G after one outer iteration")
        assert_entrywise(_np(F), Fo, 1e-4, "F after one outer iteration")


@pytest.mark.parametrize("cluster", [1, 2, 4, 8, (2, 128), (8, 128)])
def test_cluster_sizes_agree(nmf, batch, cluster):
    # a different cluster size (or CTA size) splits the sums differently: float32 rounding only
    Gs, Fs, stats = _run(nmf, batch, 6, 10, cluster=cluster)
    for b, G, F, st in zip(batch, Gs, Fs, stats):
        assert st.status == 0
        Go, Fo, _ = _oracle(b, 6, 10)
        Xd = b["X"].astype(np.float64)
        assert abs(metrics.rre(Xd, _np(G), _np(F)) - metrics.rre(Xd, Go, Fo)) <= 1e-5


def test_batched_is_deterministic(nmf, batch):
    G1, F1, _ = _run(nmf, batch, 5, 10, tol=1e-4)
    G2, F2, _ = _run(nmf, batch, 5, 10, tol=1e-4)
    for a, b in zip(G1 + F1, G2 + F2):
        assert bool((a == b).all())


def test_batched_matches_single_problem_solver(nmf, batch):
    T, inner = 6, 10
    Gs, Fs, _ = _run(nmf, batch, T, inner, tol=1e-5)
    for b, G, F in zip(batch, Gs, Fs):
        G1, F1 = _t(b["G0"]), _t(b["F0"])
        pr = nmf.compressed_problem(_t(b["L"]), _t(b["R"]), _t(b["XL"]), _t(b["XR"]), b["p"])
        nmf.solve(pr, G1, F1, T, inner, tol=1e-5)
        Xd = b["X"].astype(np.float64)
        assert abs(metrics.rre(Xd, _np(G), _np(F)) - metrics.rre(Xd, _np(G1), _np(F1))) <= 1e-5


def test_empty_batch_and_zero_outer(nmf, batch):
    nmf.solve_batched([], [], [], 5, 10)
    Gs, Fs, stats = _run(nmf, batch[:3], 0, 10)
    for b, G, F, st in zip(batch[:3], Gs, Fs, stats):
        np.testing.assert_array_equal(_np(G), b["G0"])
        np.testing.assert_array_equal(_np(F), b["F0"])
        assert st.outer_done == 0


def test_zero_factor_keeps_the_other(nmf, batch):
    # F = 0 makes H_G = 0 (L_c = 0): the G update keeps G, as in the oracle
    b = dict(batch[1])
    b["F0"] = np.zeros_like(b["F0"])
    Gs, Fs, stats = _run(nmf, [b], 1, 10)
    Go, Fo, _ = _oracle(b, 1, 10)
    np.testing.assert_allclose(_np(Gs[0]), Go, rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(_np(Fs[0]), Fo, rtol=1e-4, atol=1e-6)
    assert stats[0].status == 0


def test_full_size_batch(nmf):
    # The batched workload at full size: 256 problems, n ~ U[1000, 8000],
    # m ~ U[500, 4000], p ~ U{4..16}, nu = p + 10, q = 2, 20 dB, bfloat16
    # compression, 50 outer iterations (inner <= 10, tol 1e-6). X is drawn on
    # the device; sampled problems keep theirs for the checks.
    import torch
    shapes = synth.batched_shapes(256, seed=0)
    sizes = [s["n"] * s["m"] for s in shapes]
    sample = {int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 128}
    probs, Gs, Fs, G0s, F0s, kept = [], [], [], [], [], {}
    for i, sh in enumerate(shapes):
        X, _, _ = synth.lowrank_data_device(sh["n"], sh["m"], sh["p"], seed=1000 + i, snr_db=20.0)
        L, R, XL, XR = nmf.compress(X, sh["nu"], 2, prec=1, seed=5000 + i)
        G0, F0 = synth.initial_factors(sh["n"], sh["m"], sh["p"], seed=9000 + i)
        probs.append(nmf.compressed_problem(L, R, XL, XR, sh["p"]))
        G0s.append(G0.astype(np.float32))
        F0s.append(F0.astype(np.float32))
        Gs.append(_t(G0))
        Fs.append(_t(F0))
        if i in sample:
            kept[i] = (X, L, R, XL, XR)
        else:
            del X
    T, inner, tol = 50, 10, 1e-6
    stats = nmf.read_batch_stats(nmf.solve_batched(probs, Gs, Fs, T, inner, tol=tol), len(probs))
    torch.cuda.synchronize()
    for st, G, F in zip(stats, Gs, Fs):
        assert st.status == 0 and st.outer_done == T
        assert bool(torch.isfinite(G).all()) and bool((G >= 0).all()) and bool((F >= 0).all())
    for i, (X, L, R, XL, XR) in kept.items():
        G1, F1 = _t(G0s[i]), _t(F0s[i])
        nmf.solve(probs[i], G1, F1, T, inner, tol=tol)
        r_b, r_s = nmf.rre(X, Gs[i], Fs[i]), nmf.rre(X, G1, F1)
        assert abs(r_b - r_s) <= 1e-5, (i, r_b, r_s)
        assert r_b < 0.5 * nmf.rre(X, _t(G0s[i]), _t(F0s[i]))
    # the smallest problem against the oracle on the same float32 compressed inputs
    i = int(np.argmin(sizes))
    X, L, R, XL, XR = kept[i]
    Go, Fo, _ = nenmf.nenmf_compressed(_np(L), _np(R), _np(XL), _np(XR), G0s[i], F0s[i], T, inner, tol=tol)
    Xd = _np(X)
    assert abs(metrics.rre(Xd, _np(Gs[i]), _np(Fs[i])) - metrics.rre(Xd, Go, Fo)) <= 1e-5


def test_autotune_picks_a_measured_cluster_size(nmf, batch):
    # the autotuner times every valid (cluster size, threads per CTA) on copies
    # of the factors: it returns the fastest of its own measurements and leaves G, F alone
    probs, Gs, Fs = [], [], []
    for b in batch:
        probs.append(nmf.compressed_problem(_t(b["L"]), _t(b["R"]), _t(b["XL"]), _t(b["XR"]), b["p"]))
        Gs.append(_t(b["G0"]))
        Fs.append(_t(b["F0"]))
    best, times = nmf.batch_autotune(probs, Gs, Fs, 20, 10, tol=1e-6, trial_outer=2)
    assert best[0] in (1, 2, 4, 8) and best[1] in (128, 256) and best in times
    assert times[best] == min(times.values()) and all(t > 0.0 for t in times.values())
    assert len(times) >= 2  # both CTA sizes were measured
    assert nmf.batch_plan([probs[0]], 20, 10, cluster=best)[0] == best
    for b, G, F in zip(batch, Gs, Fs):
        np.testing.assert_array_equal(_np(G), b["G0"].astype(np.float64))
        np.testing.assert_array_equal(_np(F), b["F0"].astype(np.float64))
    # the tuned size is an ordinary configuration: same result as asking for it
    G1, F1, _ = _run(nmf, batch, 3, 10, cluster=best)
    G2, F2, _ = _run(nmf, batch, 3, 10, cluster=best)
    for a, c in zip(G1 + F1, G2 + F2):
        assert bool((a == c).all())


def test_graph_replay_equals_eager(nmf):
    # nmf_compress_batched + nenmf_solve_batched captured once in a CUDA graph
    # and replayed twice: bitwise the eager result (every kernel of both calls
    # is deterministic and the descriptors travel as kernel parameters).
    import torch
    shapes = [(400, 300, 5, 12), (257, 520, 8, 18), (130, 90, 3, 8), (600, 333, 12, 22)]
    Xs, nus, outs, probs, G0s, F0s, Gs, Fs = [], [], [], [], [], [], [], []
    for i, (n, m, p, nu) in enumerate(shapes):
        X, _, _ = synth.lowrank_data(n, m, p, seed=60 + i, snr_db=20.0, dtype=np.float32)
        Xs.append(_t(X))
        nus.append(nu)
        out = tuple(torch.empty(z, dtype=torch.float32, device="cuda") for z in [(nu, n), (m, nu), (nu, m), (n, nu)])
        outs.append(out)
        probs.append(nmf.compressed_problem(*out, p))
        G0, F0 = synth.initial_factors(n, m, p, seed=70 + i)
        G0s.append(_t(G0))
        F0s.append(_t(F0))
        Gs.append(_t(G0))
        Fs.append(_t(F0))
    T, inner, tol, q = 6, 10, 1e-5, 2
    seeds = [80 + i for i in range(len(shapes))]
    ws_c = nmf.workspace(nmf.compress_batched_workspace_size([(s[0], s[1], s[3]) for s in shapes], q, 1))
    ws_s = nmf.workspace(nmf.batch_workspace_size(probs, T, inner, tol=tol))
    stats = torch.zeros(len(probs) * 256, dtype=torch.uint8, device="cuda")

    def step():
        nmf.compress_batched(Xs, nus, q, prec=1, seeds=seeds, outs=outs, ws=ws_c)
        torch._foreach_copy_(Gs, G0s)
        torch._foreach_copy_(Fs, F0s)
        nmf.solve_batched(probs, Gs, Fs, T, inner, tol=tol, stats=stats, ws=ws_s)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = [t.clone() for t in Gs + Fs] + [t.clone() for o in outs for t in o]
    for st in nmf.read_batch_stats(stats, len(probs)):
        assert st.status == 0 and st.outer_done == T
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for _ in range(2):
        for t in Gs + Fs:
            t.fill_(-1.0)          # replay must recompute everything it returns
        for o in outs:
            for t in o:
                t.fill_(float("nan"))
        graph.replay()
        torch.cuda.synchronize()
        for st in nmf.read_batch_stats(stats, len(probs)):
            assert st.status == 0 and st.outer_done == T
        for a, b in zip(eager, [t for t in Gs + Fs] + [t for o in outs for t in o]):
            assert bool(torch.equal(a, b))
