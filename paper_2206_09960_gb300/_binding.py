"""ctypes binding of ``include/psi.h`` (argument marshalling only).

Every function of the C ABI is exposed under its own name; :class:`Graph` wraps a handle
for convenience.  All computation runs in ``libpsi_gb300.so``; if the library cannot be
loaded, :func:`load` raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpsi_gb300.so")

PSI_OK, PSI_ERR_INVALID_ARG, PSI_ERR_OUT_OF_RANGE_ID, PSI_ERR_SELF_LOOP, PSI_ERR_BAD_RATE = 0, 1, 2, 3, 4
PSI_ERR_OOM, PSI_ERR_CUDA, PSI_ERR_NOT_CONVERGED, PSI_ERR_TIMEOUT, PSI_ERR_NOT_SOLVED = 5, 6, 7, 8, 9
PSI_FP32, PSI_FP32_REFINE, PSI_FP64 = 0, 1, 2
PSI_TOL_PSI, PSI_TOL_S_ABS = 0, 1
PSI_BNORM_NONE, PSI_BNORM_INF = 0, 1
PSI_REJECT, PSI_DROP = 0, 1

PRECISION = {"fp32": PSI_FP32, "fp32_refine": PSI_FP32_REFINE, "fp64": PSI_FP64}
TOL_MODE = {"psi": PSI_TOL_PSI, "s_abs": PSI_TOL_S_ABS}
BNORM_MODE = {"none": PSI_BNORM_NONE, "inf": PSI_BNORM_INF}
SELF_LOOPS = {"reject": PSI_REJECT, "drop": PSI_DROP}

# every symbol include/psi.h declares
EXPORTS = ["psi_options_default", "psi_graph_create", "psi_solve", "psi_scores", "psi_topk",
           "psi_get_iterate", "psi_graph_get_stats", "psi_graph_destroy", "psi_status_string",
           "psi_last_error", "psi_kernel_launches", "psi_version", "psi_topk_noalloc", "psi_batch_create",
           "psi_batch_solve", "psi_batch_scores", "psi_batch_topk", "psi_batch_get_stats", "psi_batch_destroy",
           "psi_features", "psi_mlp_create", "psi_mlp_set_params", "psi_mlp_get_params", "psi_mlp_forward",
           "psi_mlp_grad", "psi_mlp_adam_step", "psi_mlp_destroy", "psi_solve_warm", "psi_multi_create",
           "psi_multi_solve", "psi_multi_scores", "psi_multi_topk", "psi_multi_get_stats", "psi_multi_destroy",
           "psi_pagerank", "psi_trim_memory", "psi_power_nf"]

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class psi_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class psi_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("tol_mode", ctypes.c_int32), ("bnorm_mode", ctypes.c_int32),
                ("self_loops", ctypes.c_int32), ("reorder", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("spmv_tile", ctypes.c_int32), ("stream", ctypes.c_void_p), ("allocator", ctypes.POINTER(psi_allocator)),
                ("autotune", ctypes.c_int32), ("spmv_hot", ctypes.c_int32)]


class psi_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("spmv_launches", ctypes.c_int32), ("gap_s_l1", ctypes.c_double), ("gap_scaled", ctypes.c_double),
                ("gap_psi_bound", ctypes.c_double), ("psi_sum", ctypes.c_double), ("ms", ctypes.c_double),
                ("spmv_ms", ctypes.c_double), ("spmv_timed", ctypes.c_int32), ("refine_timed", ctypes.c_int32),
                ("refine_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class psi_graph_stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m_input", ctypes.c_int64), ("m_unique", ctypes.c_int64),
                ("n_rows", ctypes.c_int64), ("n_gathered", ctypes.c_int64), ("max_followers", ctypes.c_int64),
                ("bnorm_inf", ctypes.c_double), ("rho_inf", ctypes.c_double), ("build_ms", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("spmv_tile", ctypes.c_int64), ("spmv_hot", ctypes.c_int64),
                ("tune_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PsiError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libpsi_gb300.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build

        if build_if_missing and not _build.up_to_date():
            _build.build_library()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2206_09960_gb300.build.build_library()")
        lib = ctypes.CDLL(LIB_PATH)
        i32, i64, dbl, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
        lib.psi_options_default.argtypes = [ctypes.POINTER(psi_options)]
        lib.psi_options_default.restype = None
        lib.psi_graph_create.argtypes = [i64, i64, vp, vp, vp, vp, ctypes.POINTER(psi_options), ctypes.POINTER(vp)]
        lib.psi_graph_create.restype = i32
        lib.psi_solve.argtypes = [vp, dbl, i32, vp, ctypes.POINTER(psi_solve_info)]
        lib.psi_solve.restype = i32
        lib.psi_scores.argtypes = [vp, vp]
        lib.psi_scores.restype = i32
        lib.psi_topk.argtypes = [vp, i32, vp, vp]
        lib.psi_topk.restype = i32
        lib.psi_get_iterate.argtypes = [vp, vp]
        lib.psi_get_iterate.restype = i32
        lib.psi_graph_get_stats.argtypes = [vp, ctypes.POINTER(psi_graph_stats)]
        lib.psi_graph_get_stats.restype = i32
        lib.psi_graph_destroy.argtypes = [vp]
        lib.psi_graph_destroy.restype = None
        lib.psi_status_string.argtypes = [i32]
        lib.psi_status_string.restype = ctypes.c_char_p
        lib.psi_last_error.argtypes = []
        lib.psi_last_error.restype = ctypes.c_char_p
        lib.psi_batch_create.argtypes = [i64, i64, vp, vp, i32, vp, vp, ctypes.POINTER(psi_options),
                                         ctypes.POINTER(vp)]
        lib.psi_batch_create.restype = i32
        lib.psi_batch_solve.argtypes = [vp, dbl, i32, vp]
        lib.psi_batch_solve.restype = i32
        lib.psi_batch_scores.argtypes = [vp, vp]
        lib.psi_batch_scores.restype = i32
        lib.psi_batch_topk.argtypes = [vp, i32, vp, vp]
        lib.psi_batch_topk.restype = i32
        lib.psi_batch_get_stats.argtypes = [vp, ctypes.POINTER(psi_graph_stats)]
        lib.psi_batch_get_stats.restype = i32
        lib.psi_batch_destroy.argtypes = [vp]
        lib.psi_batch_destroy.restype = None
        lib.psi_trim_memory.argtypes = []
        lib.psi_trim_memory.restype = i32
        lib.psi_pagerank.argtypes = [vp, dbl, dbl, i32, vp, vp]
        lib.psi_pagerank.restype = i32
        lib.psi_power_nf.argtypes = [vp, dbl, i32, i32, vp, vp]
        lib.psi_power_nf.restype = i32
        lib.psi_multi_create.argtypes = [i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(psi_options),
                                         ctypes.POINTER(vp)]
        lib.psi_multi_create.restype = i32
        lib.psi_multi_solve.argtypes = [vp, dbl, i32, vp]
        lib.psi_multi_solve.restype = i32
        lib.psi_multi_scores.argtypes = [vp, vp]
        lib.psi_multi_scores.restype = i32
        lib.psi_multi_topk.argtypes = [vp, i32, vp, vp]
        lib.psi_multi_topk.restype = i32
        lib.psi_multi_get_stats.argtypes = [vp, ctypes.POINTER(psi_graph_stats)]
        lib.psi_multi_get_stats.restype = i32
        lib.psi_multi_destroy.argtypes = [vp]
        lib.psi_multi_destroy.restype = None
        lib.psi_features.argtypes = [vp, vp]
        lib.psi_features.restype = i32
        lib.psi_mlp_create.argtypes = [ctypes.c_uint64, vp, ctypes.POINTER(vp)]
        lib.psi_mlp_create.restype = i32
        lib.psi_mlp_set_params.argtypes = [vp, vp, vp]
        lib.psi_mlp_set_params.restype = i32
        lib.psi_mlp_get_params.argtypes = [vp, vp, vp]
        lib.psi_mlp_get_params.restype = i32
        lib.psi_mlp_forward.argtypes = [vp, i64, vp, vp]
        lib.psi_mlp_forward.restype = i32
        lib.psi_mlp_grad.argtypes = [vp, i64, vp, vp, vp, ctypes.POINTER(dbl)]
        lib.psi_mlp_grad.restype = i32
        lib.psi_mlp_adam_step.argtypes = [vp, ctypes.c_float]
        lib.psi_mlp_adam_step.restype = i32
        lib.psi_mlp_destroy.argtypes = [vp]
        lib.psi_mlp_destroy.restype = None
        lib.psi_solve_warm.argtypes = [vp, vp, dbl, i32, ctypes.POINTER(psi_solve_info)]
        lib.psi_solve_warm.restype = i32
        lib.psi_topk_noalloc.argtypes = [vp, i64, i32, vp, vp, vp]
        lib.psi_topk_noalloc.restype = i32
        lib.psi_kernel_launches.argtypes = []
        lib.psi_kernel_launches.restype = i64
        lib.psi_version.argtypes = []
        lib.psi_version.restype = i32
        _lib = lib
        return lib


def status_name(s: int) -> str:
    return load().psi_status_string(int(s)).decode()


def last_error() -> str:
    return load().psi_last_error().decode()


def _check(status: int, allow=(PSI_OK,)):
    if status not in allow:
        raise PsiError(status, last_error())
    return status


# ---------------------------------------------------------------- same names as the C ABI

def psi_options_default() -> psi_options:
    o = psi_options()
    load().psi_options_default(ctypes.byref(o))
    return o


def psi_graph_create(n, m, follower_ptr, leader_ptr, lambda_ptr, mu_ptr, opt: psi_options | None):
    h = ctypes.c_void_p()
    st = load().psi_graph_create(int(n), int(m), follower_ptr, leader_ptr, lambda_ptr, mu_ptr,
                                 ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    _check(st)
    return h


def psi_solve(h, eps, max_iter, init_ptr=None):
    info = psi_solve_info()
    st = load().psi_solve(h, float(eps), int(max_iter), init_ptr, ctypes.byref(info))
    _check(st, (PSI_OK, PSI_ERR_NOT_CONVERGED))
    return st, info


def psi_scores(h, out_ptr):
    _check(load().psi_scores(h, out_ptr))


def psi_topk(h, k, ids_ptr, vals_ptr):
    _check(load().psi_topk(h, int(k), ids_ptr, vals_ptr))


def psi_get_iterate(h, out_ptr):
    _check(load().psi_get_iterate(h, out_ptr))


def psi_graph_get_stats(h) -> psi_graph_stats:
    s = psi_graph_stats()
    _check(load().psi_graph_get_stats(h, ctypes.byref(s)))
    return s


def psi_graph_destroy(h):
    load().psi_graph_destroy(h)


def psi_topk_noalloc(psi_ptr, n, k, ids_ptr, vals_ptr, stream_ptr=None):
    """Ranking of a caller-held device psi vector without any device allocation (queued on
    the stream; the call does not wait)."""
    _check(load().psi_topk_noalloc(psi_ptr, int(n), int(k), ids_ptr, vals_ptr, stream_ptr))


def psi_batch_create(n, m, follower_ptr, leader_ptr, S, lambda_ptr, mu_ptr, opt):
    h = ctypes.c_void_p()
    _check(load().psi_batch_create(int(n), int(m), follower_ptr, leader_ptr, int(S), lambda_ptr, mu_ptr,
                                   ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)))
    return h


def psi_batch_solve(h, eps, max_iter, S):
    infos = (psi_solve_info * int(S))()
    st = load().psi_batch_solve(h, float(eps), int(max_iter), infos)
    _check(st, (PSI_OK, PSI_ERR_NOT_CONVERGED))
    return st, infos


def psi_batch_scores(h, out_ptr):
    _check(load().psi_batch_scores(h, out_ptr))


def psi_batch_topk(h, k, ids_ptr, vals_ptr):
    _check(load().psi_batch_topk(h, int(k), ids_ptr, vals_ptr))


def psi_batch_get_stats(h) -> psi_graph_stats:
    s = psi_graph_stats()
    _check(load().psi_batch_get_stats(h, ctypes.byref(s)))
    return s


def psi_batch_destroy(h):
    load().psi_batch_destroy(h)


def psi_power_nf(h, eps, max_iter, origins_per_pass, out_ptr):
    info = psi_solve_info()
    st = load().psi_power_nf(h, float(eps), int(max_iter), int(origins_per_pass), out_ptr, ctypes.byref(info))
    _check(st, allow=(PSI_OK, PSI_ERR_NOT_CONVERGED))
    return st, info.as_dict()


def psi_pagerank(h, alpha, eps, max_iter, out_ptr):
    info = psi_solve_info()
    st = load().psi_pagerank(h, float(alpha), float(eps), int(max_iter), out_ptr, ctypes.byref(info))
    _check(st, (PSI_OK, PSI_ERR_NOT_CONVERGED))
    return st, info


def psi_multi_create(G, n_g_ptr, m_g_ptr, follower_ptr, leader_ptr, lambda_ptr, mu_ptr, opt):
    h = ctypes.c_void_p()
    _check(load().psi_multi_create(int(G), n_g_ptr, m_g_ptr, follower_ptr, leader_ptr, lambda_ptr, mu_ptr,
                                   ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)))
    return h


def psi_multi_solve(h, eps, max_iter, G):
    infos = (psi_solve_info * int(G))()
    st = load().psi_multi_solve(h, float(eps), int(max_iter), infos)
    _check(st, (PSI_OK, PSI_ERR_NOT_CONVERGED))
    return st, infos


def psi_multi_scores(h, out_ptr):
    _check(load().psi_multi_scores(h, out_ptr))


def psi_multi_topk(h, k, ids_ptr, vals_ptr):
    _check(load().psi_multi_topk(h, int(k), ids_ptr, vals_ptr))


def psi_multi_get_stats(h) -> psi_graph_stats:
    s = psi_graph_stats()
    _check(load().psi_multi_get_stats(h, ctypes.byref(s)))
    return s


def psi_multi_destroy(h):
    load().psi_multi_destroy(h)


def psi_features(h, out_ptr):
    _check(load().psi_features(h, out_ptr))


def psi_mlp_create(seed, stream_ptr=None):
    h = ctypes.c_void_p()
    _check(load().psi_mlp_create(int(seed), stream_ptr, ctypes.byref(h)))
    return h


def psi_mlp_set_params(h, params_ptr, norm_ptr):
    _check(load().psi_mlp_set_params(h, params_ptr, norm_ptr))


def psi_mlp_get_params(h, params_ptr, norm_ptr):
    _check(load().psi_mlp_get_params(h, params_ptr, norm_ptr))


def psi_mlp_forward(h, rows, x_ptr, y_ptr):
    _check(load().psi_mlp_forward(h, int(rows), x_ptr, y_ptr))


def psi_mlp_grad(h, rows, x_ptr, t_ptr, grad_ptr=None):
    loss = ctypes.c_double()
    _check(load().psi_mlp_grad(h, int(rows), x_ptr, t_ptr, grad_ptr, ctypes.byref(loss)))
    return loss.value


def psi_mlp_adam_step(h, lr):
    _check(load().psi_mlp_adam_step(h, float(lr)))


def psi_mlp_destroy(h):
    load().psi_mlp_destroy(h)


def psi_solve_warm(g, m, eps, max_iter):
    info = psi_solve_info()
    st = load().psi_solve_warm(g, m, float(eps), int(max_iter), ctypes.byref(info))
    _check(st, (PSI_OK, PSI_ERR_NOT_CONVERGED))
    return st, info


def psi_kernel_launches() -> int:
    return int(load().psi_kernel_launches())


def psi_version() -> int:
    return int(load().psi_version())
