"""Python binding of libnmf (compressed NeNMF on GB300): argument marshalling only.

Every function takes and returns torch CUDA tensors (float32, contiguous) and
enqueues work on torch's current stream through the C ABI of include/nmf.h;
all arithmetic runs in the library's CUDA kernels. The library must have been
built (`paper_1812_04315_gb300.build.build()`); there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnmf.so")

PREC_FP32 = 0
PREC_BF16 = 1
PLAIN = 0
COMPRESSED = 1
TOL_REL = 0
TOL_ABS = 1
MAX_RANK = 32
MAX_SKETCH = 64

STATUS = {0: "ok", 1: "invalid argument", 2: "workspace", 3: "CUDA error", 4: "not SPD",
          5: "non-finite", 6: "device timeout", 7: "unsupported"}


class NmfError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)} (status {code})")
        self.code = code


class Problem(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("n", ctypes.c_int), ("m", ctypes.c_int), ("p", ctypes.c_int),
                ("nu", ctypes.c_int), ("prec", ctypes.c_int), ("X", ctypes.c_void_p), ("L", ctypes.c_void_p),
                ("R", ctypes.c_void_p), ("XL", ctypes.c_void_p), ("XR", ctypes.c_void_p)]


class ProblemF64(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("n", ctypes.c_int), ("m", ctypes.c_int), ("p", ctypes.c_int),
                ("nu", ctypes.c_int), ("X", ctypes.c_void_p), ("L", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("XL", ctypes.c_void_p), ("XR", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("max_outer", ctypes.c_int), ("max_inner", ctypes.c_int), ("min_inner", ctypes.c_int),
                ("tol_mode", ctypes.c_int), ("tol", ctypes.c_double), ("record_G", ctypes.c_void_p),
                ("record_F", ctypes.c_void_p), ("record_time_ns", ctypes.c_void_p), ("restart", ctypes.c_int)]


class CompressItem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("m", ctypes.c_int), ("nu", ctypes.c_int), ("q", ctypes.c_int),
                ("X", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("L", ctypes.c_void_p), ("R", ctypes.c_void_p),
                ("XL", ctypes.c_void_p), ("XR", ctypes.c_void_p)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("cluster", ctypes.c_int), ("threads", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_done", ctypes.c_int), ("last_inner", ctypes.c_int * 2),
                ("total_inner", ctypes.c_longlong * 2), ("eps", ctypes.c_double), ("pg_norm", ctypes.c_double * 2),
                ("lipschitz", ctypes.c_double * 2)]


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libnmf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1812_04315_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, sz, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_uint64
    sigs = {
        "nmf_status_string": (ctypes.c_char_p, [i]),
        "nmf_version": (i, []),
        "nmf_workspace_status": (i, [vp, vp, ctypes.POINTER(i)]),
        "nmf_gaussian_sketch": (i, [vp, i, i, u64, ctypes.c_uint32, vp]),
        "nmf_compress_workspace_size": (sz, [i, i, i, i]),
        "nmf_compress": (i, [vp, i, i, i, i, i, vp, vp, vp, u64, vp, vp, vp, vp, vp, sz]),
        "nmf_compress_variant": (i, [vp, i, i, i, i, i, i, vp, vp, vp, u64, vp, vp, vp, vp, vp, sz]),
        "nmf_compress_batched_workspace_size": (sz, [i, vp, i]),
        "nmf_compress_batched": (i, [vp, i, vp, i, i, vp, sz]),
        "nenmf_solve_workspace_size": (sz, [ctypes.POINTER(Problem)]),
        "nmf_project_workspace_size": (sz, [i, i, i, i]),
        "nenmf_batch_autotune_workspace_size": (sz, [i, vp, ctypes.POINTER(Params), i]),
        "nenmf_batch_autotune": (i, [vp, i, vp, vp, vp, ctypes.POINTER(Params), i, ctypes.POINTER(BatchConfig),
                                     ctypes.POINTER(ctypes.c_float), vp, sz]),
        "nmf_project": (i, [vp, i, i, i, i, vp, vp, vp, vp, vp, vp, sz]),
        "nmf_compress_f64_workspace_size": (sz, [i, i, i]),
        "nmf_compress_f64": (i, [vp, i, i, i, i, vp, vp, vp, u64, vp, vp, vp, vp, vp, sz]),
        "nenmf_solve_f64_workspace_size": (sz, [ctypes.POINTER(ProblemF64)]),
        "nenmf_solve_f64": (i, [vp, ctypes.POINTER(ProblemF64), vp, vp, ctypes.POINTER(Params), vp, vp, sz]),
        "nenmf_backward_f64_workspace_size": (sz, [ctypes.POINTER(ProblemF64), ctypes.POINTER(Params)]),
        "nenmf_backward_f64": (i, [vp, ctypes.POINTER(ProblemF64), ctypes.POINTER(Params), vp, vp, vp, vp, vp, vp, vp,
                                   vp, vp, vp, sz]),
        "nenmf_solve": (i, [vp, ctypes.POINTER(Problem), vp, vp, ctypes.POINTER(Params), vp, vp, sz]),
        "nmf_rre_workspace_size": (sz, [i, i, i]),
        "nmf_rre": (i, [vp, i, i, i, vp, vp, vp, vp, vp, sz]),
        "nmf_dual_product_workspace_size": (sz, [i, i, i, i]),
        "nmf_dual_product": (i, [vp, i, i, i, i, vp, vp, vp, vp, vp, vp, sz]),
        "nmf_set_kernel_path": (None, [i]),
        "nmf_kernel_launches": (ctypes.c_longlong, []),
        "nmf_rre_static": (i, [vp, i, i, i, vp, vp, vp, vp]),
        "nmf_inject_fault": (i, [i, ctypes.c_longlong]),
        "nenmf_solve_batched_workspace_size": (sz, [i, vp, ctypes.POINTER(Params), ctypes.POINTER(BatchConfig)]),
        "nenmf_batch_plan_info": (i, [i, vp, ctypes.POINTER(Params), ctypes.POINTER(BatchConfig),
                                      ctypes.POINTER(BatchConfig), ctypes.POINTER(i)]),
        "nenmf_solve_batched": (i, [vp, i, vp, vp, vp, ctypes.POINTER(Params), ctypes.POINTER(BatchConfig), vp,
                                    vp, sz]),
        "nenmf_backward_workspace_size": (sz, [ctypes.POINTER(Problem), ctypes.POINTER(Params)]),
        "nenmf_backward": (i, [vp, ctypes.POINTER(Problem), ctypes.POINTER(Params)] + [vp] * 11 + [vp, sz]),
        "nmf_gram_workspace_size": (sz, [i, i]),
        "nmf_gram": (i, [vp, i, i, vp, vp, vp, sz]),
        "nmf_orth_apply_workspace_size": (sz, [i, i]),
        "nmf_orth_apply": (i, [vp, i, i, vp, vp, vp, vp, sz]),
        "nenmf_nnls_block_workspace_size": (sz, [i, i, i, i]),
        "nenmf_nnls_block": (i, [vp, i, i, vp, vp, vp, vp, i, i, i, vp, vp, vp, vp, sz]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names declared by the binding (all must resolve in the library)."""
    return ["nmf_status_string", "nmf_version", "nmf_workspace_status", "nmf_gaussian_sketch",
            "nmf_compress_workspace_size", "nmf_compress", "nenmf_solve_workspace_size", "nenmf_solve",
            "nmf_rre_workspace_size", "nmf_rre", "nmf_dual_product_workspace_size", "nmf_dual_product",
            "nmf_set_kernel_path", "nmf_kernel_launches", "nmf_rre_static",
            "nenmf_solve_batched_workspace_size", "nenmf_batch_plan_info", "nenmf_solve_batched",
            "nenmf_backward_workspace_size", "nenmf_backward", "nmf_compress_variant",
            "nmf_compress_batched_workspace_size", "nmf_compress_batched", "nmf_compress_f64_workspace_size",
            "nmf_compress_f64", "nenmf_solve_f64_workspace_size", "nenmf_solve_f64",
            "nenmf_backward_f64_workspace_size", "nenmf_backward_f64", "nmf_project_workspace_size", "nmf_project",
            "nenmf_batch_autotune_workspace_size", "nenmf_batch_autotune", "nmf_inject_fault",
            "nmf_gram_workspace_size", "nmf_gram", "nmf_orth_apply_workspace_size", "nmf_orth_apply",
            "nenmf_nnls_block_workspace_size", "nenmf_nnls_block"]


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check_f32(name, t, shape):
    torch = _torch()
    if t.device.type != "cuda" or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


def _check_f64(name, t, shape):
    torch = _torch()
    if t.device.type != "cuda" or t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


def _ok(code, where):
    if code != 0:
        raise NmfError(code, where)


def workspace(nbytes: int):
    """Device workspace of nbytes (256-byte aligned through the caching allocator)."""
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device="cuda")


def workspace_status(ws) -> int:
    v = ctypes.c_int(0)
    _ok(lib().nmf_workspace_status(_stream(), _ptr(ws), ctypes.byref(v)), "nmf_workspace_status")
    return v.value


def kernel_launches() -> int:
    return int(lib().nmf_kernel_launches())


PATH_XPASS_CUDA_CORES = 1
PATH_SOLVE_PER_UPDATE = 2


def set_kernel_path(force_cuda_cores: bool = False, per_update_solve: bool = False):
    """nmf_set_kernel_path: alternative kernels for cross-checks (defaults: the fastest path)."""
    lib().nmf_set_kernel_path((PATH_XPASS_CUDA_CORES if force_cuda_cores else 0) |
                              (PATH_SOLVE_PER_UPDATE if per_update_solve else 0))


FAULT_NONE = 0
FAULT_STOP_TEST = 1
FAULT_XPASS_COPY = 2


def inject_fault(fault: int, wait_limit_ns: int = 0):
    """nmf_inject_fault: failure-path testing only (see include/nmf.h)."""
    _ok(lib().nmf_inject_fault(fault, wait_limit_ns), "nmf_inject_fault")


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------

def gaussian_sketch(rows: int, cols: int, seed: int, stream_id: int, out=None):
    torch = _torch()
    if out is None:
        out = torch.empty((rows, cols), dtype=torch.float32, device="cuda")
    _check_f32("out", out, (rows, cols))
    _ok(lib().nmf_gaussian_sketch(_stream(), rows, cols, seed, stream_id, _ptr(out)), "nmf_gaussian_sketch")
    return out


def compress_workspace_size(n, m, nu, prec=PREC_BF16) -> int:
    return int(lib().nmf_compress_workspace_size(n, m, nu, prec))


VARIANTS = {"subspace": 0, "swapped": 1, "single": 2, "power": 3, "gaussian": 4}


def compress(X, nu: int, q: int, prec: int = PREC_BF16, omega_L=None, omega_R=None, seed: int = 0, ws=None,
             out=None, variant: str = "subspace"):
    """Alg. 2 (or a named variant) + the compression step of Alg. 1: returns (L nu x n, R m x nu, X_L nu x m,
    X_R n x nu)."""
    torch = _torch()
    n, m = X.shape
    _check_f32("X", X, (n, m))
    if omega_L is not None:
        _check_f32("omega_L", omega_L, (m, nu))
        _check_f32("omega_R", omega_R, (nu, n))
    if out is None:
        out = (torch.empty((nu, n), dtype=torch.float32, device="cuda"),
               torch.empty((m, nu), dtype=torch.float32, device="cuda"),
               torch.empty((nu, m), dtype=torch.float32, device="cuda"),
               torch.empty((n, nu), dtype=torch.float32, device="cuda"))
    L, R, XL, XR = out
    if ws is None:
        ws = workspace(compress_workspace_size(n, m, nu, prec))
    if variant == "subspace":
        _ok(lib().nmf_compress(_stream(), n, m, nu, q, prec, _ptr(X), _ptr(omega_L), _ptr(omega_R), seed, _ptr(L),
                               _ptr(R), _ptr(XL), _ptr(XR), _ptr(ws), ws.numel()), "nmf_compress")
    else:
        _ok(lib().nmf_compress_variant(_stream(), n, m, nu, q, prec, VARIANTS[variant], _ptr(X), _ptr(omega_L),
                                       _ptr(omega_R), seed, _ptr(L), _ptr(R), _ptr(XL), _ptr(XR), _ptr(ws),
                                       ws.numel()), "nmf_compress_variant")
    return L, R, XL, XR


def compress_batched_workspace_size(shapes, q: int, prec: int = PREC_BF16) -> int:
    """Workspace bytes of nmf_compress_batched for [(n, m, nu), ...]."""
    items = (CompressItem * max(1, len(shapes)))()
    for i, (n, m, nu) in enumerate(shapes):
        items[i].n, items[i].m, items[i].nu, items[i].q = n, m, nu, q
    return int(lib().nmf_compress_batched_workspace_size(len(shapes), ctypes.cast(items, ctypes.c_void_p), prec))


def compress_batched(Xs, nus, q: int, prec: int = PREC_BF16, seeds=None, outs=None, variant: str = "subspace",
                     ws=None):
    """nmf_compress_batched over the matrices Xs (one nu per matrix); returns [(L, R, X_L, X_R), ...]."""
    torch = _torch()
    count = len(Xs)
    seeds = list(range(count)) if seeds is None else list(seeds)
    if outs is None:
        outs = []
        for X, nu in zip(Xs, nus):
            n, m = X.shape
            outs.append((torch.empty((nu, n), dtype=torch.float32, device=X.device),
                         torch.empty((m, nu), dtype=torch.float32, device=X.device),
                         torch.empty((nu, m), dtype=torch.float32, device=X.device),
                         torch.empty((n, nu), dtype=torch.float32, device=X.device)))
    items = (CompressItem * max(1, count))()
    for i, (X, nu, sd, o) in enumerate(zip(Xs, nus, seeds, outs)):
        n, m = X.shape
        _check_f32("X", X, (n, m))
        items[i].n, items[i].m, items[i].nu, items[i].q = n, m, nu, q
        items[i].X, items[i].seed = X.data_ptr(), sd
        items[i].L, items[i].R, items[i].XL, items[i].XR = (t.data_ptr() for t in o)
    if ws is None:
        ws = workspace(compress_batched_workspace_size([(X.shape[0], X.shape[1], nu) for X, nu in zip(Xs, nus)], q,
                                                       prec))
    _ok(lib().nmf_compress_batched(_stream(), count, ctypes.cast(items, ctypes.c_void_p), prec, VARIANTS[variant],
                                   _ptr(ws), ws.numel()), "nmf_compress_batched")
    return outs


def _problem(mode, n, m, p, nu=0, prec=PREC_FP32, X=None, L=None, R=None, XL=None, XR=None):
    pr = Problem()
    # The struct holds raw device pointers: keep the tensors alive with it.
    pr._tensors = (X, L, R, XL, XR)
    pr.mode, pr.n, pr.m, pr.p, pr.nu, pr.prec = mode, n, m, p, nu, prec
    pr.X = X.data_ptr() if X is not None else None
    pr.L = L.data_ptr() if L is not None else None
    pr.R = R.data_ptr() if R is not None else None
    pr.XL = XL.data_ptr() if XL is not None else None
    pr.XR = XR.data_ptr() if XR is not None else None
    return pr


def plain_problem(X, p: int, prec: int = PREC_FP32):
    n, m = X.shape
    _check_f32("X", X, (n, m))
    return _problem(PLAIN, n, m, p, 0, prec, X=X)


def compressed_problem(L, R, XL, XR, p: int):
    nu, n = L.shape
    m = R.shape[0]
    for name, t, shp in (("L", L, (nu, n)), ("R", R, (m, nu)), ("XL", XL, (nu, m)), ("XR", XR, (n, nu))):
        _check_f32(name, t, shp)
    return _problem(COMPRESSED, n, m, p, nu, PREC_FP32, L=L, R=R, XL=XL, XR=XR)


def solve_workspace_size(problem: Problem) -> int:
    return int(lib().nenmf_solve_workspace_size(ctypes.byref(problem)))


@dataclass
class SolveRecord:
    G: object = None      # [T, n, p]
    F: object = None      # [T, p, m]
    times: object = None  # int64 [T + 1] (ns, %globaltimer)


def solve(problem: Problem, G, F, max_outer: int, max_inner: int, min_inner: int = 1, tol: float = 0.0,
          tol_mode: int = TOL_REL, record: SolveRecord | None = None, stats=None, ws=None, restart: bool = False):
    """Runs nenmf_solve in place on G (n x p) and F (p x m); returns the device stats buffer."""
    torch = _torch()
    n, m, p = problem.n, problem.m, problem.p
    _check_f32("G", G, (n, p))
    _check_f32("F", F, (p, m))
    pa = Params()
    pa.max_outer, pa.max_inner, pa.min_inner, pa.tol_mode, pa.tol = max_outer, max_inner, min_inner, tol_mode, tol
    pa.restart = int(bool(restart))
    if record is not None:
        pa.record_G = record.G.data_ptr() if record.G is not None else None
        pa.record_F = record.F.data_ptr() if record.F is not None else None
        pa.record_time_ns = record.times.data_ptr() if record.times is not None else None
    if stats is None:
        stats = torch.zeros(ctypes.sizeof(Stats), dtype=torch.uint8, device="cuda")
    if ws is None:
        ws = workspace(solve_workspace_size(problem))
    _ok(lib().nenmf_solve(_stream(), ctypes.byref(problem), _ptr(G), _ptr(F), ctypes.byref(pa), _ptr(stats),
                          _ptr(ws), ws.numel()), "nenmf_solve")
    return stats


def _batch_args(problems, max_outer, max_inner, min_inner, tol, tol_mode, cluster, restart=False):
    arr = (Problem * max(1, len(problems)))(*problems)
    pa = Params()
    pa.max_outer, pa.max_inner, pa.min_inner, pa.tol_mode, pa.tol = max_outer, max_inner, min_inner, tol_mode, tol
    pa.restart = int(bool(restart))
    cfg = BatchConfig()
    # a configuration is a cluster size or a (cluster size, threads per CTA) pair; 0: the planner's choice
    cfg.cluster, cfg.threads = (cluster, 0) if isinstance(cluster, int) else (int(cluster[0]), int(cluster[1]))
    return arr, pa, cfg


def batch_plan(problems, max_outer: int, max_inner: int, min_inner: int = 1, tol: float = 0.0,
               tol_mode: int = TOL_REL, cluster: int = 0):
    """((CTAs per problem, threads per CTA), clusters launched) that nenmf_solve_batched would use."""
    arr, pa, cfg = _batch_args(problems, max_outer, max_inner, min_inner, tol, tol_mode, cluster)
    out = BatchConfig()
    ncl = ctypes.c_int(0)
    _ok(lib().nenmf_batch_plan_info(len(problems), ctypes.cast(arr, ctypes.c_void_p), ctypes.byref(pa),
                                    ctypes.byref(cfg), ctypes.byref(out), ctypes.byref(ncl)), "nenmf_batch_plan_info")
    return (out.cluster, out.threads), ncl.value


def batch_workspace_size(problems, max_outer: int, max_inner: int, min_inner: int = 1, tol: float = 0.0,
                         tol_mode: int = TOL_REL, cluster: int = 0) -> int:
    arr, pa, cfg = _batch_args(problems, max_outer, max_inner, min_inner, tol, tol_mode, cluster)
    return int(lib().nenmf_solve_batched_workspace_size(len(problems), ctypes.cast(arr, ctypes.c_void_p),
                                                        ctypes.byref(pa), ctypes.byref(cfg)))


def solve_batched(problems, Gs, Fs, max_outer: int, max_inner: int, min_inner: int = 1, tol: float = 0.0,
                  tol_mode: int = TOL_REL, cluster: int = 0, stats=None, ws=None, restart: bool = False):
    """Runs nenmf_solve_batched in place on every (G_i, F_i); returns the device stats buffer (count entries)."""
    torch = _torch()
    count = len(problems)
    if len(Gs) != count or len(Fs) != count:
        raise ValueError("one G and one F per problem")
    for pr, G, F in zip(problems, Gs, Fs):
        _check_f32("G", G, (pr.n, pr.p))
        _check_f32("F", F, (pr.p, pr.m))
    arr, pa, cfg = _batch_args(problems, max_outer, max_inner, min_inner, tol, tol_mode, cluster, restart)
    gp = (ctypes.c_void_p * max(1, count))(*[G.data_ptr() for G in Gs])
    fp = (ctypes.c_void_p * max(1, count))(*[F.data_ptr() for F in Fs])
    if stats is None:
        stats = torch.zeros(max(1, count) * ctypes.sizeof(Stats), dtype=torch.uint8, device="cuda")
    if ws is None:
        ws = workspace(batch_workspace_size(problems, max_outer, max_inner, min_inner, tol, tol_mode, cluster))
    _ok(lib().nenmf_solve_batched(_stream(), count, ctypes.cast(arr, ctypes.c_void_p), ctypes.cast(gp, ctypes.c_void_p),
                                  ctypes.cast(fp, ctypes.c_void_p), ctypes.byref(pa), ctypes.byref(cfg), _ptr(stats),
                                  _ptr(ws), ws.numel()), "nenmf_solve_batched")
    return stats


def backward(problem: Problem, G0, F0, record: SolveRecord, dG_T, dF_T, max_outer: int, max_inner: int,
             want_dX: bool = False, ws=None):
    """nenmf_backward: cotangents (dXL, dXR, dG0, dF0, dX or None) of the compressed solve's
    inputs, given those of its outputs and the forward's snapshots (fixed inner iterations)."""
    torch = _torch()
    n, m, p, nu = problem.n, problem.m, problem.p, problem.nu
    for name, t, shp in (("G0", G0, (n, p)), ("F0", F0, (p, m)), ("dG_T", dG_T, (n, p)), ("dF_T", dF_T, (p, m))):
        _check_f32(name, t, shp)
    if max_outer > 0:
        _check_f32("record.G", record.G, (max_outer, n, p))
        _check_f32("record.F", record.F, (max_outer, p, m))
    pa = Params()
    pa.max_outer, pa.max_inner, pa.min_inner, pa.tol_mode, pa.tol = max_outer, max_inner, 1, TOL_REL, 0.0
    dev = G0.device
    dXL = torch.empty((nu, m), dtype=torch.float32, device=dev)
    dXR = torch.empty((n, nu), dtype=torch.float32, device=dev)
    dG0 = torch.empty((n, p), dtype=torch.float32, device=dev)
    dF0 = torch.empty((p, m), dtype=torch.float32, device=dev)
    dX = torch.empty((n, m), dtype=torch.float32, device=dev) if want_dX else None
    if ws is None:
        ws = workspace(lib().nenmf_backward_workspace_size(ctypes.byref(problem), ctypes.byref(pa)))
    rg = _ptr(record.G) if max_outer > 0 else None
    rf = _ptr(record.F) if max_outer > 0 else None
    _ok(lib().nenmf_backward(_stream(), ctypes.byref(problem), ctypes.byref(pa), _ptr(G0), _ptr(F0), rg, rf,
                             _ptr(dG_T), _ptr(dF_T), _ptr(dXL), _ptr(dXR), _ptr(dG0), _ptr(dF0), _ptr(dX),
                             _ptr(ws), ws.numel()), "nenmf_backward")
    return dXL, dXR, dG0, dF0, dX


def batch_autotune(problems, Gs, Fs, max_outer: int, max_inner: int, min_inner: int = 1, tol: float = 0.0,
                   tol_mode: int = TOL_REL, restart: bool = False, trial_outer: int = 2, ws=None):
    """nenmf_batch_autotune: (fastest (cluster size, threads per CTA), {(cluster, threads): trial ms})
    for these problems; Gs, Fs are left unchanged. Synchronous."""
    count = len(problems)
    for pr, G, F in zip(problems, Gs, Fs):
        _check_f32("G", G, (pr.n, pr.p))
        _check_f32("F", F, (pr.p, pr.m))
    arr, pa, _ = _batch_args(problems, max_outer, max_inner, min_inner, tol, tol_mode, 0, restart)
    gp = (ctypes.c_void_p * count)(*[G.data_ptr() for G in Gs])
    fp = (ctypes.c_void_p * count)(*[F.data_ptr() for F in Fs])
    if ws is None:
        ws = workspace(lib().nenmf_batch_autotune_workspace_size(count, ctypes.cast(arr, ctypes.c_void_p),
                                                                 ctypes.byref(pa), trial_outer))
    best = BatchConfig()
    ms = (ctypes.c_float * 8)()
    _ok(lib().nenmf_batch_autotune(_stream(), count, ctypes.cast(arr, ctypes.c_void_p), ctypes.cast(gp, ctypes.c_void_p),
                                   ctypes.cast(fp, ctypes.c_void_p), ctypes.byref(pa), trial_outer, ctypes.byref(best),
                                   ms, _ptr(ws), ws.numel()), "nenmf_batch_autotune")
    cands = [(c, t) for c in (1, 2, 4, 8) for t in (256, 128)]
    return (best.cluster, best.threads), {ct: float(ms[k]) for k, ct in enumerate(cands) if ms[k] >= 0.0}


def read_batch_stats(stats, count: int):
    raw = bytes(stats.cpu().numpy().tobytes())
    k = ctypes.sizeof(Stats)
    return [Stats.from_buffer_copy(raw[i * k:(i + 1) * k]) for i in range(count)]


def read_stats(stats) -> Stats:
    raw = bytes(stats.cpu().numpy().tobytes())
    return Stats.from_buffer_copy(raw)


def rre_workspace_size(n, m, p) -> int:
    return int(lib().nmf_rre_workspace_size(n, m, p))


def rre_terms(X, G, F, out=None, ws=None):
    """Device tensor [||X - G F||^2, ||X||^2] (float64)."""
    torch = _torch()
    n, m = X.shape
    p = G.shape[1]
    _check_f32("X", X, (n, m))
    _check_f32("G", G, (n, p))
    _check_f32("F", F, (p, m))
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device="cuda")
    if ws is None:
        ws = workspace(rre_workspace_size(n, m, p))
    _ok(lib().nmf_rre(_stream(), n, m, p, _ptr(X), _ptr(G), _ptr(F), _ptr(out), _ptr(ws), ws.numel()), "nmf_rre")
    return out


def rre(X, G, F) -> float:
    t = rre_terms(X, G, F).cpu()
    return float((t[0] / t[1]).sqrt())


def dual_product(X, A=None, B=None, prec: int = PREC_FP32, ws=None):
    """(X A, X^T B) from one pass over X; either operand may be None."""
    torch = _torch()
    n, m = X.shape
    k = (A if A is not None else B).shape[1]
    _check_f32("X", X, (n, m))
    if A is not None:
        _check_f32("A", A, (m, k))
    if B is not None:
        _check_f32("B", B, (n, k))
    YN = torch.empty((n, k), dtype=torch.float32, device="cuda") if A is not None else None
    YT = torch.empty((m, k), dtype=torch.float32, device="cuda") if B is not None else None
    if ws is None:
        ws = workspace(lib().nmf_dual_product_workspace_size(n, m, k, prec))
    _ok(lib().nmf_dual_product(_stream(), n, m, k, prec, _ptr(X), _ptr(A), _ptr(B), _ptr(YN), _ptr(YT), _ptr(ws),
                               ws.numel()), "nmf_dual_product")
    return YN, YT


def project(X, L, R, prec: int = PREC_FP32, ws=None):
    """nmf_project: (X_L = L X, X_R = X R) for given bases L (nu x n), R (m x nu)."""
    torch = _torch()
    n, m = X.shape
    nu = L.shape[0]
    _check_f32("X", X, (n, m))
    _check_f32("L", L, (nu, n))
    _check_f32("R", R, (m, nu))
    XL = torch.empty((nu, m), dtype=torch.float32, device=X.device)
    XR = torch.empty((n, nu), dtype=torch.float32, device=X.device)
    if ws is None:
        ws = workspace(lib().nmf_project_workspace_size(n, m, nu, prec))
    _ok(lib().nmf_project(_stream(), n, m, nu, prec, _ptr(X), _ptr(L), _ptr(R), _ptr(XL), _ptr(XR), _ptr(ws),
                          ws.numel()), "nmf_project")
    return XL, XR


_autograd_cls = None


def _compressed_nenmf_function():
    """torch.autograd.Function of (X, G0, F0) -> (G_T, F_T): T outer iterations of
    compressed NeNMF (Alg. 1) with exactly K inner iterations each, for fixed bases
    L, R (X reaches the map through X_L = L X, X_R = X R). forward: nmf_project,
    then nenmf_solve with per-outer snapshots; backward: nenmf_backward, which
    recomputes each outer iteration's inner steps from its snapshot."""
    global _autograd_cls
    if _autograd_cls is not None:
        return _autograd_cls
    torch = _torch()

    class CompressedNeNMF(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X, G0, F0, L, R, T, K):
            n, m = X.shape
            p = G0.shape[1]
            X, G0, F0, L, R = (t.detach().contiguous() for t in (X, G0, F0, L, R))
            XL, XR = project(X, L, R)
            prob = compressed_problem(L, R, XL, XR, p)
            G, F = G0.clone(), F0.clone()
            rec = SolveRecord(G=torch.empty((max(T, 1), n, p), dtype=torch.float32, device=X.device),
                              F=torch.empty((max(T, 1), p, m), dtype=torch.float32, device=X.device))
            if T > 0:
                solve(prob, G, F, T, K, tol=0.0, record=rec)
            ctx.save_for_backward(G0, F0, L, R, XL, XR, rec.G, rec.F)
            ctx.T, ctx.K, ctx.p = T, K, p
            return G, F

        @staticmethod
        def backward(ctx, dG, dF):
            G0, F0, L, R, XL, XR, rG, rF = ctx.saved_tensors
            zeros = lambda t: torch.zeros_like(t)
            dG = zeros(G0) if dG is None else dG.contiguous()
            dF = zeros(F0) if dF is None else dF.contiguous()
            prob = compressed_problem(L, R, XL, XR, ctx.p)
            _, _, dG0, dF0, dX = backward(prob, G0, F0, SolveRecord(G=rG, F=rF), dG, dF, ctx.T, ctx.K, want_dX=True)
            return dX, dG0, dF0, None, None, None, None

    _autograd_cls = CompressedNeNMF
    return _autograd_cls


def compressed_nenmf(X, G0, F0, L, R, T: int, K: int):
    """Differentiable compressed NeNMF: (G_T, F_T) = CompressedNeNMF.apply(X, G0, F0, L, R, T, K);
    gradients flow to X, G0 and F0 (float32 CUDA tensors), not to the bases."""
    return _compressed_nenmf_function().apply(X, G0, F0, L, R, T, K)


# ---------------------------------------------------------------------------
# float64 twins
# ---------------------------------------------------------------------------

def compress_f64(X, nu: int, q: int, omega_L=None, omega_R=None, seed: int = 0, ws=None):
    """nmf_compress_f64: (L nu x n, R m x nu, X_L nu x m, X_R n x nu) in float64."""
    torch = _torch()
    n, m = X.shape
    _check_f64("X", X, (n, m))
    if omega_L is not None:
        _check_f64("omega_L", omega_L, (m, nu))
        _check_f64("omega_R", omega_R, (nu, n))
    L = torch.empty((nu, n), dtype=torch.float64, device="cuda")
    R = torch.empty((m, nu), dtype=torch.float64, device="cuda")
    XL = torch.empty((nu, m), dtype=torch.float64, device="cuda")
    XR = torch.empty((n, nu), dtype=torch.float64, device="cuda")
    if ws is None:
        ws = workspace(int(lib().nmf_compress_f64_workspace_size(n, m, nu)))
    _ok(lib().nmf_compress_f64(_stream(), n, m, nu, q, _ptr(X), _ptr(omega_L), _ptr(omega_R), seed, _ptr(L), _ptr(R),
                               _ptr(XL), _ptr(XR), _ptr(ws), ws.numel()), "nmf_compress_f64")
    return L, R, XL, XR


def plain_problem_f64(X, p: int) -> ProblemF64:
    n, m = X.shape
    _check_f64("X", X, (n, m))
    pr = ProblemF64()
    pr.mode, pr.n, pr.m, pr.p, pr.nu, pr.X = PLAIN, n, m, p, 0, X.data_ptr()
    pr._keep = (X,)
    return pr


def compressed_problem_f64(L, R, XL, XR, p: int) -> ProblemF64:
    nu, n = L.shape
    m = R.shape[0]
    for name, t, shp in (("L", L, (nu, n)), ("R", R, (m, nu)), ("XL", XL, (nu, m)), ("XR", XR, (n, nu))):
        _check_f64(name, t, shp)
    pr = ProblemF64()
    pr.mode, pr.n, pr.m, pr.p, pr.nu = COMPRESSED, n, m, p, nu
    pr.L, pr.R, pr.XL, pr.XR = L.data_ptr(), R.data_ptr(), XL.data_ptr(), XR.data_ptr()
    pr._keep = (L, R, XL, XR)
    return pr


def solve_f64(problem: ProblemF64, G, F, max_outer: int, max_inner: int, min_inner: int = 1, tol: float = 0.0,
              tol_mode: int = TOL_REL, restart: bool = False, stats=None, ws=None):
    """nenmf_solve_f64 in place on G (n x p) and F (p x m), float64; returns the device stats buffer."""
    torch = _torch()
    _check_f64("G", G, (problem.n, problem.p))
    _check_f64("F", F, (problem.p, problem.m))
    pa = Params()
    pa.max_outer, pa.max_inner, pa.min_inner, pa.tol_mode, pa.tol = max_outer, max_inner, min_inner, tol_mode, tol
    pa.restart = int(bool(restart))
    if stats is None:
        stats = torch.zeros(ctypes.sizeof(Stats), dtype=torch.uint8, device="cuda")
    if ws is None:
        ws = workspace(int(lib().nenmf_solve_f64_workspace_size(ctypes.byref(problem))))
    _ok(lib().nenmf_solve_f64(_stream(), ctypes.byref(problem), _ptr(G), _ptr(F), ctypes.byref(pa), _ptr(stats),
                              _ptr(ws), ws.numel()), "nenmf_solve_f64")
    return stats


def backward_f64(problem: ProblemF64, G0, F0, dG_T, dF_T, max_outer: int, max_inner: int, want_dX: bool = False,
                 ws=None):
    """nenmf_backward_f64: (dX_L, dX_R, dG0, dF0, dX or None), float64."""
    torch = _torch()
    n, m, p, nu = problem.n, problem.m, problem.p, problem.nu
    for name, t, shp in (("G0", G0, (n, p)), ("F0", F0, (p, m)), ("dG_T", dG_T, (n, p)), ("dF_T", dF_T, (p, m))):
        _check_f64(name, t, shp)
    pa = Params()
    pa.max_outer, pa.max_inner, pa.min_inner, pa.tol = max_outer, max_inner, 1, 0.0
    out = [torch.empty(shp, dtype=torch.float64, device="cuda") for shp in ((nu, m), (n, nu), (n, p), (p, m))]
    dX = torch.empty((n, m), dtype=torch.float64, device="cuda") if want_dX else None
    if ws is None:
        ws = workspace(int(lib().nenmf_backward_f64_workspace_size(ctypes.byref(problem), ctypes.byref(pa))))
    _ok(lib().nenmf_backward_f64(_stream(), ctypes.byref(problem), ctypes.byref(pa), _ptr(G0), _ptr(F0), _ptr(dG_T),
                                 _ptr(dF_T), *[_ptr(t) for t in out], _ptr(dX), _ptr(ws), ws.numel()),
        "nenmf_backward_f64")
    return (*out, dX)


# ---------------------------------------------------------------------------
# row-sharded runs: the per-GPU steps between the collectives
# ---------------------------------------------------------------------------

def gram(Y, ws=None):
    """nmf_gram: Y^T Y (float64 device tensor) of the N x nu rows Y."""
    torch = _torch()
    N, nu = Y.shape
    _check_f32("Y", Y, (N, nu))
    S = torch.empty((nu, nu), dtype=torch.float64, device="cuda")
    if ws is None:
        ws = workspace(lib().nmf_gram_workspace_size(N, nu))
    _ok(lib().nmf_gram(_stream(), N, nu, _ptr(Y), _ptr(S), _ptr(ws), ws.numel()), "nmf_gram")
    return S


def orth_apply(Y, S, out=None, ws=None):
    """nmf_orth_apply: Y R^{-1} with R^T R = S (one CholeskyQR pass over these rows)."""
    torch = _torch()
    N, nu = Y.shape
    _check_f32("Y", Y, (N, nu))
    if S.device.type != "cuda" or S.dtype != torch.float64 or tuple(S.shape) != (nu, nu) or not S.is_contiguous():
        raise ValueError("S must be a contiguous nu x nu float64 CUDA tensor")
    if out is None:
        out = torch.empty_like(Y)
    if ws is None:
        ws = workspace(lib().nmf_orth_apply_workspace_size(N, nu))
    _ok(lib().nmf_orth_apply(_stream(), N, nu, _ptr(Y), _ptr(S), _ptr(out), _ptr(ws), ws.numel()),
        "nmf_orth_apply")
    return out


def nnls_block(H, B, Y, Fprev, k0: int, kb: int, max_inner: int, ws=None):
    """nenmf_nnls_block: iterations k0 .. k0+kb-1 of the inner loop on these columns.

    Updates Y and Fprev in place; returns (keep [kb, p, N], pg2 [max(kb, 1)] float64, L_c float64),
    all device tensors."""
    torch = _torch()
    p, N = B.shape
    _check_f32("H", H, (p, p))
    _check_f32("B", B, (p, N))
    _check_f32("Y", Y, (p, N))
    _check_f32("Fprev", Fprev, (p, N))
    keep = torch.empty((max(kb, 1), p, N), dtype=torch.float32, device="cuda")
    pg2 = torch.empty(max(kb, 1), dtype=torch.float64, device="cuda")
    lc = torch.empty(1, dtype=torch.float64, device="cuda")
    if ws is None:
        ws = workspace(lib().nenmf_nnls_block_workspace_size(N, p, kb, max_inner))
    _ok(lib().nenmf_nnls_block(_stream(), N, p, _ptr(H), _ptr(B), _ptr(Y), _ptr(Fprev), k0, kb, max_inner,
                               _ptr(keep), _ptr(pg2), _ptr(lc), _ptr(ws), ws.numel()), "nenmf_nnls_block")
    return keep[:kb], pg2, lc
