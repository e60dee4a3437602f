"""Failure detection on the device, made without faulting or hanging the GPU.

* Host-made faults: a NaN in X, an Inf in the compressed data, a NaN in the
  initial factor. Each call must finish and report NMF_ERR_NONFINITE in its
  status word instead of returning numbers (max(0, NaN) would otherwise
  turn a NaN step into 0 without a trace).
* Bounded waits that run out: nmf_inject_fault makes CTA 0 of the solve
  kernels withhold its stop-test words, or CTA 0 of the tensor-core X pass
  arm a pipeline stage and issue no copy, with every wait limited to 20 ms.
  The call must end with NMF_ERR_DEVICE_TIMEOUT; every kernel returns (no
  wait is unbounded), so the context stays usable and the next call, with
  the fault cleared, gives the normal result bit for bit.
"""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

NONFINITE, TIMEOUT = 5, 6


def _t(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _compressed_inputs(nmf, n=1000, m=900, p=6, nu=12, q=2):
    X, _, _ = synth.lowrank_data(n, m, p, seed=3, snr_db=30.0, dtype=np.float32)
    G0, F0 = (a.astype(np.float32) for a in synth.initial_factors(n, m, p, seed=4))
    L, R, XL, XR = nmf.compress(_t(X), nu, q, prec=nmf.PREC_BF16, seed=5)
    return X, G0, F0, (L, R, XL, XR)


def test_nan_in_x_is_reported_by_the_compression(nmf):
    X, _, _ = synth.lowrank_data(500, 400, 5, seed=1, snr_db=30.0, dtype=np.float32)
    X[123, 45] = np.nan
    for prec in (nmf.PREC_FP32, nmf.PREC_BF16):
        ws = nmf.workspace(nmf.compress_workspace_size(500, 400, 10, prec))
        nmf.compress(_t(X), 10, 2, prec=prec, seed=2, ws=ws)
        assert nmf.workspace_status(ws) == NONFINITE


@pytest.mark.parametrize("where", ["XR", "XL", "G0"])
def test_nonfinite_solve_input_is_reported(nmf, where):
    X, G0, F0, (L, R, XL, XR) = _compressed_inputs(nmf)
    if where == "XR":
        XR[17, 3] = float("inf")
    elif where == "XL":
        XL[2, 400] = float("nan")
    else:
        G0 = G0.copy()
        G0[5, 1] = np.nan
    G, F = _t(G0), _t(F0)
    for per_update in (False, True):
        nmf.set_kernel_path(per_update_solve=per_update)
        try:
            for tol in (0.0, 1e-6):
                st = nmf.read_stats(nmf.solve(nmf.compressed_problem(L, R, XL, XR, 6), G.clone(), F.clone(), 5, 10,
                                              tol=tol))
                assert st.status == NONFINITE, (where, per_update, tol, st.status)
        finally:
            nmf.set_kernel_path()


def _solve_reference(nmf, comp, G0, F0, tol):
    G, F = _t(G0), _t(F0)
    st = nmf.read_stats(nmf.solve(nmf.compressed_problem(*comp, 6), G, F, 4, 10, tol=tol))
    return st, G, F


@pytest.mark.parametrize("per_update", [False, True])
def test_withheld_stop_test_word_times_out(nmf, per_update):
    # both solve paths: the persistent launch and one launch per update
    import torch
    X, G0, F0, comp = _compressed_inputs(nmf)
    nmf.set_kernel_path(per_update_solve=per_update)
    try:
        st_ref, G_ref, F_ref = _solve_reference(nmf, comp, G0, F0, 0.5)
        assert st_ref.status == 0
        # tol 0.5: every CTA's own partial is far below eps^2 at the first
        # test, so each one needs the global sum and waits for CTA 0's word
        nmf.inject_fault(nmf.FAULT_STOP_TEST, 20_000_000)
        try:
            st, _, _ = _solve_reference(nmf, comp, G0, F0, 0.5)
        finally:
            nmf.inject_fault(nmf.FAULT_NONE, 0)
        assert st.status == TIMEOUT
        st2, G2, F2 = _solve_reference(nmf, comp, G0, F0, 0.5)
        torch.cuda.synchronize()
    finally:
        nmf.set_kernel_path()
    assert st2.status == 0
    assert bool(torch.equal(G2, G_ref)) and bool(torch.equal(F2, F_ref))


def test_withheld_x_pass_copy_times_out(nmf):
    import torch
    X, _, _ = synth.lowrank_data(1000, 900, 6, seed=3, snr_db=30.0, dtype=np.float32)
    Xg = _t(X)
    ws = nmf.workspace(nmf.compress_workspace_size(1000, 900, 12, nmf.PREC_BF16))
    ref = [t.clone() for t in nmf.compress(Xg, 12, 2, prec=nmf.PREC_BF16, seed=5, ws=ws)]
    assert nmf.workspace_status(ws) == 0
    nmf.inject_fault(nmf.FAULT_XPASS_COPY, 20_000_000)
    try:
        nmf.compress(Xg, 12, 2, prec=nmf.PREC_BF16, seed=5, ws=ws)
        status = nmf.workspace_status(ws)
    finally:
        nmf.inject_fault(nmf.FAULT_NONE, 0)
    assert status == TIMEOUT
    again = nmf.compress(Xg, 12, 2, prec=nmf.PREC_BF16, seed=5, ws=ws)
    assert nmf.workspace_status(ws) == 0
    for a, b in zip(ref, again):
        assert bool(torch.equal(a, b))


def test_inject_fault_rejects_unknown_values(nmf):
    with pytest.raises(nmf.NmfError):
        nmf.inject_fault(7, 0)
    with pytest.raises(nmf.NmfError):
        nmf.inject_fault(nmf.FAULT_NONE, -1)
