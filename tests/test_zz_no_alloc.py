"""nmf_rre_static: the RRE entry point that allocates nothing.

Callers that cannot allocate device memory (a fit-monitoring hook inside a
framework that owns every device allocation, a loop that must not call
cudaMalloc because it can synchronise the device) use it with only X, G, F and
the output; its scratch is a fixed array inside the library. Checked through
the C ABI against nmf_rre (the entry point with a caller workspace) on two
calls in a row, with different sizes so that contents left by the first call
would show in the second. This file is collected last, so a run that stops
at the first failure has run all others.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _static_fn(nmf):
    fn = nmf.lib().nmf_rre_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    return fn


def test_rre_static_matches_workspace_version_twice(nmf):
    import torch
    fn = _static_fn(nmf)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (n, m, p) in enumerate([(700, 1300, 7), (333, 257, 12)]):
        rng = np.random.default_rng(40 + call)
        X = torch.tensor(rng.random((n, m)), dtype=torch.float32, device="cuda")
        G = torch.tensor(rng.random((n, p)), dtype=torch.float32, device="cuda")
        F = torch.tensor(rng.random((p, m)) / p, dtype=torch.float32, device="cuda")
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        assert fn(stream, n, m, p, X.data_ptr(), G.data_ptr(), F.data_ptr(), out.data_ptr()) == 0
        got = out.cpu().numpy()
        ref = nmf.rre_terms(X, G, F).cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def test_rre_static_rejects_sizes_beyond_its_scratch(nmf):
    import torch
    fn = _static_fn(nmf)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dummy = torch.empty(4, dtype=torch.float64, device="cuda")
    ptr = dummy.data_ptr()
    # ceil(m / 256) * min(ceil(n / 64), 65535) blocks > 65536: refused before
    # any launch (NMF_ERR_WORKSPACE); the pointers are never dereferenced.
    assert fn(stream, 64 * 65537, 512, 4, ptr, ptr, ptr, ptr) == 2
    assert fn(stream, 64, 256 * 65537, 4, ptr, ptr, ptr, ptr) == 2
