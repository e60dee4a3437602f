"""Host-side checks of the C ABI that need no GPU: the library loads, every
function declared in include/*.h is exported, size queries and argument
validation answer before any device work is enqueued."""

import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b((?:nmf|nenmf)_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_1812_04315_gb300 as pkg
    if not os.path.exists(pkg.LIB_PATH):
        from paper_1812_04315_gb300 import build
        build.build()
    return pkg.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared_functions()
    assert {"nmf_compress", "nenmf_solve", "nmf_rre", "nmf_gaussian_sketch"} <= set(names)
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    import paper_1812_04315_gb300 as pkg
    assert set(pkg.exported_symbols()) <= set(names)


def test_version_and_status_strings(L):
    assert L.nmf_version() == 100
    for code in range(8):
        assert L.nmf_status_string(code)


def test_workspace_queries(L):
    assert L.nmf_compress_workspace_size(1000, 800, 20, 1) > 1000 * 800 * 2
    assert L.nmf_compress_workspace_size(0, 800, 20, 1) == 0
    assert L.nmf_compress_workspace_size(10, 10, 65, 0) == 0
    assert L.nmf_rre_workspace_size(100, 100, 5) > 0
    # one partial (two doubles) per block; the grid's y extent stops at 65535
    # row blocks of 64 rows, beyond which blocks walk several row blocks
    assert L.nmf_rre_workspace_size(64 * 65535, 256, 4) == 65535 * 16 + 16
    assert L.nmf_rre_workspace_size(64 * 65535 + 1, 256, 4) == 65535 * 16 + 16
    # the row-sharded steps: sizes out of range are refused with 0
    assert L.nmf_gram_workspace_size(1000, 20) > 0 and L.nmf_gram_workspace_size(0, 20) == 0
    assert L.nmf_gram_workspace_size(10, 65) == 0
    assert L.nmf_orth_apply_workspace_size(10, 64) > 0 and L.nmf_orth_apply_workspace_size(10, 0) == 0
    assert L.nenmf_nnls_block_workspace_size(100, 32, 16, 40) > 0
    assert L.nenmf_nnls_block_workspace_size(100, 33, 16, 40) == 0
    assert L.nenmf_nnls_block_workspace_size(100, 4, -1, 40) == 0
    assert L.nmf_rre_workspace_size(64 * 70000, 512, 4) == 2 * 65535 * 16 + 32
    import paper_1812_04315_gb300 as pkg
    pr = pkg._problem(pkg.COMPRESSED, 100, 90, 4, 8, 0)
    pr.L = pr.R = pr.XL = pr.XR = 256
    assert pkg.solve_workspace_size(pr) > 0
    pr.nu = 2  # nu < p
    assert pkg.solve_workspace_size(pr) == 0


def test_argument_errors_are_host_side(L):
    # Invalid sizes and null pointers are rejected before any CUDA call.
    v = ctypes.c_void_p
    assert L.nmf_compress(None, 0, 10, 4, 1, 1, v(256), None, None, 0, v(256), v(256), v(256), v(256), v(256), 1 << 30) == 1
    assert L.nmf_compress(None, 10, 10, 4, 1, 1, None, None, None, 0, v(256), v(256), v(256), v(256), v(256), 1 << 30) == 1
    assert L.nmf_compress(None, 10, 10, 11, 1, 1, v(256), None, None, 0, v(256), v(256), v(256), v(256), v(256), 1 << 30) == 1
    # one sketch given without the other
    assert L.nmf_compress(None, 10, 10, 4, 1, 1, v(256), v(256), None, 0, v(256), v(256), v(256), v(256), v(256), 1 << 30) == 1
    # misaligned / too small workspace
    assert L.nmf_compress(None, 10, 10, 4, 1, 0, v(256), None, None, 0, v(256), v(256), v(256), v(256), v(100), 1 << 30) == 2
    assert L.nmf_compress(None, 10, 10, 4, 1, 0, v(256), None, None, 0, v(256), v(256), v(256), v(256), v(256), 16) == 2
    assert L.nenmf_solve(None, None, None, None, None, None, None, 0) == 1
    assert L.nmf_rre(None, 10, 10, 0, v(256), v(256), v(256), v(256), v(256), 1 << 20) == 1
    assert L.nmf_dual_product(None, 10, 10, 4, 0, v(256), None, None, None, None, v(256), 1 << 30) == 1


def test_batched_argument_errors_are_host_side(L):
    import paper_1812_04315_gb300 as pkg
    pr = pkg._problem(pkg.COMPRESSED, 100, 90, 4, 8, 0)
    pr.L = pr.R = pr.XL = pr.XR = 256
    arr, pa, cfg = pkg._batch_args([pr], 5, 10, 1, 0.0, pkg.TOL_REL, 0)
    ptrs = (ctypes.c_void_p * 1)(256)
    args = lambda arr_, n=1: (None, n, ctypes.cast(arr_, ctypes.c_void_p), ctypes.cast(ptrs, ctypes.c_void_p),
                              ctypes.cast(ptrs, ctypes.c_void_p), ctypes.byref(pa), ctypes.byref(cfg), None,
                              ctypes.c_void_p(256), 1 << 30)
    assert L.nenmf_solve_batched(*args(arr, -1)) == 1
    plain = pkg._problem(pkg.PLAIN, 100, 90, 4, 0, 0)
    plain.X = 256
    arr2, _, _ = pkg._batch_args([plain], 5, 10, 1, 0.0, pkg.TOL_REL, 0)
    assert L.nenmf_solve_batched(*args(arr2)) == 7          # plain mode: unsupported in a batch
    bad = pkg._problem(pkg.COMPRESSED, 100, 90, 9, 8, 0)    # nu < p
    bad.L = bad.R = bad.XL = bad.XR = 256
    arr3, _, _ = pkg._batch_args([bad], 5, 10, 1, 0.0, pkg.TOL_REL, 0)
    assert L.nenmf_solve_batched(*args(arr3)) == 1
    pa.record_G = 256                                        # snapshots are single-problem only
    assert L.nenmf_solve_batched(*args(arr)) == 1
    pa.record_G = None
    cfg.cluster = 3
    assert L.nenmf_solve_batched(*args(arr)) == 1


def test_variant_argument_errors_are_host_side(L):
    v = ctypes.c_void_p
    # unknown variant, swapped reading with q = 0
    assert L.nmf_compress_variant(None, 10, 10, 4, 1, 0, 7, v(256), None, None, 0, v(256), v(256), v(256), v(256),
                                  v(256), 1 << 30) == 1
    assert L.nmf_compress_variant(None, 10, 10, 4, 0, 0, 1, v(256), None, None, 0, v(256), v(256), v(256), v(256),
                                  v(256), 1 << 30) == 1


def test_f64_twin_argument_errors_are_host_side(L):
    import paper_1812_04315_gb300 as pkg
    v = ctypes.c_void_p
    assert L.nmf_compress_f64_workspace_size(500, 400, 10) > 500 * 400
    assert L.nmf_compress_f64_workspace_size(10, 10, 11) == 0
    # nu > min(n, m), q out of range, null output, one sketch only, bad workspace
    assert L.nmf_compress_f64(None, 10, 10, 11, 1, v(256), None, None, 0, v(256), v(256), v(256), v(256), v(256), 1 << 30) == 1
    assert L.nmf_compress_f64(None, 10, 10, 4, 65, v(256), None, None, 0, v(256), v(256), v(256), v(256), v(256), 1 << 30) == 1
    assert L.nmf_compress_f64(None, 10, 10, 4, 1, v(256), None, None, 0, None, v(256), v(256), v(256), v(256), 1 << 30) == 1
    assert L.nmf_compress_f64(None, 10, 10, 4, 1, v(256), v(256), None, 0, v(256), v(256), v(256), v(256), v(256), 1 << 30) == 1
    assert L.nmf_compress_f64(None, 10, 10, 4, 1, v(256), None, None, 0, v(256), v(256), v(256), v(256), v(100), 1 << 30) == 2
    assert L.nmf_compress_f64(None, 10, 10, 4, 1, v(256), None, None, 0, v(256), v(256), v(256), v(256), v(256), 16) == 2
    pr = pkg.ProblemF64()
    pr.mode, pr.n, pr.m, pr.p, pr.nu, pr.X = pkg.PLAIN, 50, 40, 5, 0, 256
    assert L.nenmf_solve_f64_workspace_size(ctypes.byref(pr)) > 0
    pa = pkg.Params()
    pa.max_outer, pa.max_inner, pa.min_inner, pa.tol = 1, 10, 1, 0.0
    big = 1 << 30
    pa.record_G = 256
    assert L.nenmf_solve_f64(None, ctypes.byref(pr), v(256), v(256), ctypes.byref(pa), None, v(256), big) == 7
    pa.record_G = None
    pa.max_inner = 0
    assert L.nenmf_solve_f64(None, ctypes.byref(pr), v(256), v(256), ctypes.byref(pa), None, v(256), big) == 1
    pa.max_inner = 10
    pr.p = 33  # above the float64 twin's limit
    assert L.nenmf_solve_f64_workspace_size(ctypes.byref(pr)) == 0
    assert L.nenmf_solve_f64(None, ctypes.byref(pr), v(256), v(256), ctypes.byref(pa), None, v(256), big) == 1
    pr.p, pr.mode, pr.nu = 5, pkg.COMPRESSED, 4  # nu < p
    assert L.nenmf_solve_f64(None, ctypes.byref(pr), v(256), v(256), ctypes.byref(pa), None, v(256), big) == 1
    pr.nu = 8
    pr.L = pr.R = pr.XL = pr.XR = 256
    assert L.nenmf_solve_f64(None, ctypes.byref(pr), v(256), v(256), ctypes.byref(pa), None, v(100), big) == 2


def test_f64_backward_argument_errors_are_host_side(L):
    import paper_1812_04315_gb300 as pkg
    v = ctypes.c_void_p
    pr = pkg.ProblemF64()
    pr.mode, pr.n, pr.m, pr.p, pr.nu = pkg.COMPRESSED, 50, 40, 4, 8
    pr.L = pr.R = pr.XL = pr.XR = 256
    pa = pkg.Params()
    pa.max_outer, pa.max_inner, pa.min_inner, pa.tol = 3, 5, 1, 0.0
    assert L.nenmf_backward_f64_workspace_size(ctypes.byref(pr), ctypes.byref(pa)) > 0
    args = [v(256)] * 8
    big = 1 << 30
    pa.tol = 1e-6  # the stop test is not differentiated
    assert L.nenmf_backward_f64(None, ctypes.byref(pr), ctypes.byref(pa), *args, None, v(256), big) == 1
    pa.tol, pa.restart = 0.0, 1
    assert L.nenmf_backward_f64(None, ctypes.byref(pr), ctypes.byref(pa), *args, None, v(256), big) == 1
    pa.restart = 0
    assert L.nenmf_backward_f64(None, ctypes.byref(pr), ctypes.byref(pa), *args, None, v(100), big) == 2
    pr.mode = pkg.PLAIN
    pr.X = 256
    assert L.nenmf_backward_f64(None, ctypes.byref(pr), ctypes.byref(pa), *args, None, v(256), big) == 7


def test_project_argument_errors_are_host_side(L):
    v = ctypes.c_void_p
    assert L.nmf_project_workspace_size(100, 80, 8, 1) > 0
    assert L.nmf_project_workspace_size(100, 80, 81, 1) == 0
    assert L.nmf_project(None, 100, 80, 8, 0, v(256), None, v(256), v(256), v(256), v(256), 1 << 30) == 1
    assert L.nmf_project(None, 100, 80, 8, 2, v(256), v(256), v(256), v(256), v(256), v(256), 1 << 30) == 1
    assert L.nmf_project(None, 100, 80, 8, 0, v(256), v(256), v(256), v(256), v(256), v(100), 1 << 30) == 2


def test_autotune_argument_errors_are_host_side(L):
    import paper_1812_04315_gb300 as pkg
    v = ctypes.c_void_p
    pr = pkg._problem(pkg.COMPRESSED, 100, 90, 4, 8, 0)
    pr.L = pr.R = pr.XL = pr.XR = 256
    arr = (pkg.Problem * 1)(pr)
    pa = pkg.Params()
    pa.max_outer, pa.max_inner, pa.min_inner, pa.tol = 10, 10, 1, 0.0
    best = pkg.BatchConfig()
    ptrs = (ctypes.c_void_p * 1)(256)
    a = ctypes.cast(arr, ctypes.c_void_p)
    p = ctypes.cast(ptrs, ctypes.c_void_p)
    assert L.nenmf_batch_autotune_workspace_size(1, a, ctypes.byref(pa), 0) == 0
    assert L.nenmf_batch_autotune(None, 1, a, p, p, ctypes.byref(pa), 0, ctypes.byref(best), None, v(256), 1 << 30) == 1
    assert L.nenmf_batch_autotune(None, 1, a, p, p, ctypes.byref(pa), 2, None, None, v(256), 1 << 30) == 1
    assert L.nenmf_batch_autotune(None, 0, a, p, p, ctypes.byref(pa), 2, ctypes.byref(best), None, v(256), 1 << 30) == 1
    assert L.nenmf_batch_autotune(None, 1, a, p, p, ctypes.byref(pa), 2, ctypes.byref(best), None, v(100), 1 << 30) == 2
