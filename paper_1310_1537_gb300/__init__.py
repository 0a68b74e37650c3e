"""Python binding of the GB300 logistic-GLM library (libglm.so).

Argument marshalling only: every function here has the name of a C entry
point declared in include/glm.h and forwards device pointers (torch tensors'
``data_ptr()``), sizes and the current CUDA stream to it. All arithmetic of
the hot path runs in the library's CUDA kernels. There is no CPU fallback: if
libglm.so cannot be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libglm.so")

GLM_OK = 0
GLM_ERR_INVALID_ARG = 1
GLM_ERR_UNSUPPORTED = 2
GLM_ERR_OOM = 3
GLM_ERR_CUDA = 4
GLM_ERR_TIMEOUT = 5
GLM_ERR_NO_DEVICE = 6
GLM_PENDING = 7

GLM_X_F32 = 0
GLM_X_BF16 = 1
GLM_X_FP8E4M3 = 2

GLM_PATH_NONE = 0
GLM_PATH_CUDA_CORES = 1
GLM_PATH_TENSOR_CORES = 2

GLM_FLAG_NO_TENSOR_CORES = 0x1
GLM_FLAG_NO_PRIOR = 0x2

ELEM_BYTES = {GLM_X_F32: 4, GLM_X_BF16: 2, GLM_X_FP8E4M3: 1}

# Every C symbol the header declares (checked by the ABI test).
EXPORTS = (
    "glm_create", "glm_destroy", "glm_status_str", "glm_get_info", "glm_logpost_grad",
    "glm_logpost_grad_host", "glm_logpost_grad_grouped", "glm_rwm_run", "glm_quantize",
    "glm_sync", "glm_selftest_wait_timeout", "glm_logpost_grad_noalloc",
    "glm_autotune_grouped", "glm_grouped_set_shape", "glm_grouped_get_shape",
    "glm_server_create", "glm_server_add_dataset", "glm_server_submit",
    "glm_server_poll", "glm_server_wait", "glm_server_stats", "glm_server_destroy",
    "glm_server_remove_dataset",
    "glm_slice_create", "glm_slice_destroy", "glm_slice_eta", "glm_slice_coord_logpost",
    "glm_slice_run", "glm_slice_sync", "glm_ising_split", "glm_ising_merge", "glm_ising_sweeps",
    "glm_hess_create", "glm_hess_destroy", "glm_hess_eval", "glm_hess_sync",
)


class GLMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {glm_status_str(status)} (status {status})")


class glm_desc_t(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("p", C.c_int32), ("ld", C.c_int32),
                ("k_max", C.c_int32), ("xtype", C.c_int32), ("prior_sigma", C.c_double),
                ("device", C.c_int32), ("flags", C.c_uint32), ("g_max", C.c_int32)]


class glm_info_t(C.Structure):
    _fields_ = [("sm_count", C.c_int32), ("grid", C.c_int32), ("tile_rows", C.c_int32),
                ("stages", C.c_int32), ("smem_bytes", C.c_int32), ("tc_enabled", C.c_int32),
                ("tc_min_k", C.c_int32), ("workspace_bytes", C.c_int64)]


class glm_server_desc_t(C.Structure):
    _fields_ = [("device", C.c_int32), ("streams", C.c_int32), ("max_batch_k", C.c_int32),
                ("max_pending", C.c_int32), ("hbm_budget_bytes", C.c_int64)]


class glm_request_info_t(C.Structure):
    _fields_ = [("submit_ns", C.c_int64), ("start_ns", C.c_int64), ("done_ns", C.c_int64),
                ("batch_k", C.c_int32), ("batch_requests", C.c_int32), ("k", C.c_int32),
                ("status", C.c_int32), ("path", C.c_int32), ("deferrals", C.c_int32)]


class glm_server_stats_t(C.Structure):
    _fields_ = [("requests_done", C.c_int64), ("requests_failed", C.c_int64),
                ("requests_waiting", C.c_int64), ("batches", C.c_int64),
                ("vectors_done", C.c_int64), ("hbm_budget_bytes", C.c_int64),
                ("hbm_in_flight_bytes", C.c_int64), ("hbm_resident_bytes", C.c_int64),
                ("batches_tensor_cores", C.c_int64), ("deferrals", C.c_int64),
                ("trimmed_batches", C.c_int64), ("refused_requests", C.c_int64),
                ("max_concurrent_batches", C.c_int32),
                ("last_cuda_error", C.c_int32), ("last_error_site", C.c_int32)]


class glm_slice_desc_t(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("ld", C.c_int64), ("p", C.c_int32), ("m", C.c_int32),
                ("s_max", C.c_int32), ("device", C.c_int32), ("w", C.c_float),
                ("spec", C.c_int32), ("prior_sigma", C.c_double)]


_lib = None
_lock = threading.Lock()


def load(build_if_missing: bool = True):
    """Load libglm.so (building it in-tree with nvcc when it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _build
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; run paper_1310_1537_gb300.build")
        lib = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        st = C.c_int
        sig = {
            "glm_create": ([C.POINTER(glm_desc_t), C.POINTER(vp)], st),
            "glm_destroy": ([vp], st),
            "glm_status_str": ([st], C.c_char_p),
            "glm_get_info": ([vp, C.POINTER(glm_info_t)], st),
            "glm_logpost_grad": ([vp, vp, vp, vp, vp, C.c_int32, vp, vp, vp], st),
            "glm_logpost_grad_host": ([vp, vp, vp, vp, vp, C.c_int32, vp, vp, vp], st),
            "glm_logpost_grad_grouped": ([vp, vp, vp, vp, vp, C.c_int32, vp, vp, C.c_double,
                                          vp, vp, vp], st),
            "glm_rwm_run": ([vp, vp, vp, vp, C.c_int32, C.c_int32, C.c_float, vp, vp, vp, vp,
                             C.c_int32, vp, vp, vp, vp], st),
            "glm_quantize": ([vp, vp, C.c_int32, vp, vp, vp], st),
            "glm_sync": ([vp, vp], st),
            "glm_selftest_wait_timeout": ([vp, C.c_int32, vp], st),
            "glm_logpost_grad_noalloc": ([vp, vp, vp, C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                                          C.c_double, vp, C.c_int32, vp, vp, vp], st),
            "glm_autotune_grouped": ([vp, vp, vp, vp, vp, C.c_int32, vp, vp, C.c_double, vp, vp,
                                      C.c_int32, vp], st),
            "glm_grouped_set_shape": ([vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                       C.c_int32], st),
            "glm_grouped_get_shape": ([vp] + [C.POINTER(C.c_int32)] * 5, st),
            "glm_server_create": ([C.POINTER(glm_server_desc_t), C.POINTER(vp)], st),
            "glm_server_add_dataset": ([vp, vp, vp, vp, C.c_int64, C.c_int32, C.c_int32,
                                        C.c_int32, C.c_double, C.POINTER(C.c_int32)], st),
            "glm_server_submit": ([vp, C.c_int32, vp, C.c_int32, C.POINTER(C.c_uint64)], st),
            "glm_server_remove_dataset": ([vp, C.c_int32], st),
            "glm_server_poll": ([vp, C.c_uint64, vp, vp, C.POINTER(glm_request_info_t)], st),
            "glm_server_wait": ([vp, C.c_uint64, vp, vp, C.POINTER(glm_request_info_t),
                                 C.c_int32], st),
            "glm_server_stats": ([vp, C.POINTER(glm_server_stats_t)], st),
            "glm_server_destroy": ([vp], st),
            "glm_hess_create": ([C.c_int64, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                 C.POINTER(vp)], st),
            "glm_hess_destroy": ([vp], st),
            "glm_hess_eval": ([vp, vp, vp, vp, vp, vp, vp, vp], st),
            "glm_hess_sync": ([vp, vp], st),
            "glm_ising_split": ([vp, C.c_int32, C.c_int32, C.c_int32, vp, vp, vp], st),
            "glm_ising_merge": ([vp, vp, C.c_int32, C.c_int32, C.c_int32, vp, vp], st),
            "glm_ising_sweeps": ([vp, vp, vp, vp, C.c_int32, C.c_int32, C.c_float, C.c_int32, vp,
                                  vp, vp], st),
            "glm_slice_create": ([C.POINTER(glm_slice_desc_t), C.POINTER(vp)], st),
            "glm_slice_destroy": ([vp], st),
            "glm_slice_eta": ([vp, vp, vp, vp, vp], st),
            "glm_slice_coord_logpost": ([vp, vp, vp, vp, vp, C.c_int32, vp, C.c_int32, vp, vp],
                                        st),
            "glm_slice_run": ([vp, vp, vp, vp, vp, vp, C.c_int32, C.c_int32, vp, vp, vp, vp, vp,
                               vp], st),
            "glm_slice_sync": ([vp, vp], st),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _ptr(x):
    """Device/host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _check(status: int, where: str):
    if status != GLM_OK:
        raise GLMError(status, where)


def glm_status_str(status: int) -> str:
    return load().glm_status_str(int(status)).decode()


def glm_create(n_rows: int, p: int, ld: int, k_max: int, xtype: int = GLM_X_F32,
               prior_sigma: float = 10.0, device: int = 0, flags: int = 0, g_max: int = 0) -> int:
    d = glm_desc_t(int(n_rows), int(p), int(ld), int(k_max), int(xtype), float(prior_sigma),
                   int(device), int(flags), int(g_max))
    h = C.c_void_p()
    _check(load().glm_create(C.byref(d), C.byref(h)), "glm_create")
    return h.value


def glm_destroy(h) -> None:
    _check(load().glm_destroy(h), "glm_destroy")


def glm_get_info(h) -> dict:
    info = glm_info_t()
    _check(load().glm_get_info(h, C.byref(info)), "glm_get_info")
    return {k: getattr(info, k) for k, _ in glm_info_t._fields_}


def glm_logpost_grad(h, X, x_scale, y, beta, K, f_out, g_out, stream=None) -> None:
    _check(load().glm_logpost_grad(h, _ptr(X), _ptr(x_scale), _ptr(y), _ptr(beta), int(K),
                                   _ptr(f_out), _ptr(g_out), _stream(stream)),
           "glm_logpost_grad")


def glm_logpost_grad_host(h, X, x_scale, y, beta_host, K, f_host, g_host, stream=None) -> None:
    _check(load().glm_logpost_grad_host(h, _ptr(X), _ptr(x_scale), _ptr(y), _ptr(beta_host),
                                        int(K), _ptr(f_host), _ptr(g_host), _stream(stream)),
           "glm_logpost_grad_host")


def glm_logpost_grad_grouped(h, X, x_scale, y, group_off, G, beta, mu, tau, f_out, g_out,
                             stream=None) -> None:
    _check(load().glm_logpost_grad_grouped(h, _ptr(X), _ptr(x_scale), _ptr(y), _ptr(group_off),
                                           int(G), _ptr(beta), _ptr(mu), float(tau),
                                           _ptr(f_out), _ptr(g_out), _stream(stream)),
           "glm_logpost_grad_grouped")


def glm_autotune_grouped(h, X, x_scale, y, group_off, G, beta, mu, tau, f_out, g_out, reps=5,
                         stream=None) -> None:
    _check(load().glm_autotune_grouped(h, _ptr(X), _ptr(x_scale), _ptr(y), _ptr(group_off),
                                       int(G), _ptr(beta), _ptr(mu), float(tau), _ptr(f_out),
                                       _ptr(g_out), int(reps), _stream(stream)),
           "glm_autotune_grouped")


def glm_grouped_set_shape(h, variant, warps, units, stages, ctas_per_sm) -> None:
    _check(load().glm_grouped_set_shape(h, int(variant), int(warps), int(units), int(stages),
                                        int(ctas_per_sm)), "glm_grouped_set_shape")


def glm_grouped_get_shape(h) -> tuple:
    """(variant, warps, units, stages, ctas_per_sm) of the grouped launch."""
    vals = [C.c_int32() for _ in range(5)]
    _check(load().glm_grouped_get_shape(h, *[C.byref(v) for v in vals]), "glm_grouped_get_shape")
    return tuple(v.value for v in vals)


def glm_rwm_run(h, X, x_scale, y, K, n_steps, step, z, log_u, beta_state, f_state, init_f,
                samples=None, accept=None, logpost=None, stream=None) -> None:
    _check(load().glm_rwm_run(h, _ptr(X), _ptr(x_scale), _ptr(y), int(K), int(n_steps),
                              C.c_float(step), _ptr(z), _ptr(log_u), _ptr(beta_state),
                              _ptr(f_state), int(init_f), _ptr(samples), _ptr(accept),
                              _ptr(logpost), _stream(stream)),
           "glm_rwm_run")


def glm_quantize(h, X32, ld32, Xq, x_scale=None, stream=None) -> None:
    _check(load().glm_quantize(h, _ptr(X32), int(ld32), _ptr(Xq), _ptr(x_scale),
                               _stream(stream)), "glm_quantize")


def glm_sync(h, stream=None) -> int:
    """Synchronise and return the status code (does not raise on TIMEOUT)."""
    return int(load().glm_sync(h, _stream(stream)))


def glm_selftest_wait_timeout(h, spin_limit, stream=None) -> None:
    _check(load().glm_selftest_wait_timeout(h, int(spin_limit), _stream(stream)),
           "glm_selftest_wait_timeout")


def glm_logpost_grad_noalloc(X, x_scale, y, n_rows, p, ld, xtype, prior_sigma, beta, K, f_out,
                             g_out, stream=None) -> None:
    """Handle-free evaluation that allocates no device memory (fixed scratch)."""
    _check(load().glm_logpost_grad_noalloc(_ptr(X), _ptr(x_scale), _ptr(y), int(n_rows), int(p),
                                           int(ld), int(xtype), float(prior_sigma), _ptr(beta),
                                           int(K), _ptr(f_out), _ptr(g_out), _stream(stream)),
           "glm_logpost_grad_noalloc")


def _info_dict(info) -> dict:
    return {name: getattr(info, name) for name, _ in info._fields_}


def glm_server_create(device: int = 0, streams: int = 4, max_batch_k: int = 64,
                      max_pending: int = 65536, hbm_budget_bytes: int = 0):
    """Create a serving loop (scheduler thread + stream pool); returns the server."""
    d = glm_server_desc_t(int(device), int(streams), int(max_batch_k), int(max_pending),
                          int(hbm_budget_bytes))
    s = C.c_void_p()
    _check(load().glm_server_create(C.byref(d), C.byref(s)), "glm_server_create")
    return s.value


def glm_server_add_dataset(s, X, x_scale, y, n_rows, p, ld, xtype=GLM_X_F32,
                           prior_sigma=10.0) -> int:
    ds = C.c_int32()
    _check(load().glm_server_add_dataset(s, _ptr(X), _ptr(x_scale), _ptr(y), int(n_rows), int(p),
                                         int(ld), int(xtype), float(prior_sigma), C.byref(ds)),
           "glm_server_add_dataset")
    return ds.value


def glm_server_remove_dataset(s, dataset_id) -> bool:
    """Unregister a dataset; False (nothing changed) while requests for it
    are still waiting or running."""
    st = load().glm_server_remove_dataset(s, int(dataset_id))
    if st == GLM_PENDING:
        return False
    _check(st, "glm_server_remove_dataset")
    return True


def glm_server_submit(s, dataset_id, beta_host, K) -> int:
    """Queue K host FP32 vectors (contiguous K x P); returns the request id."""
    rid = C.c_uint64()
    _check(load().glm_server_submit(s, int(dataset_id), _ptr(beta_host), int(K), C.byref(rid)),
           "glm_server_submit")
    return rid.value


def glm_server_poll(s, request_id, f_host=None, g_host=None):
    """Returns None while pending, else the request's info dict (raises on failure)."""
    info = glm_request_info_t()
    st = load().glm_server_poll(s, C.c_uint64(request_id), _ptr(f_host), _ptr(g_host),
                                C.byref(info))
    if st == GLM_PENDING:
        return None
    _check(st, "glm_server_poll")
    return _info_dict(info)


def glm_server_wait(s, request_id, f_host=None, g_host=None, timeout_ms=60000) -> dict:
    info = glm_request_info_t()
    _check(load().glm_server_wait(s, C.c_uint64(request_id), _ptr(f_host), _ptr(g_host),
                                  C.byref(info), int(timeout_ms)), "glm_server_wait")
    return _info_dict(info)


def glm_server_stats(s) -> dict:
    st = glm_server_stats_t()
    _check(load().glm_server_stats(s, C.byref(st)), "glm_server_stats")
    return _info_dict(st)


def glm_server_destroy(s) -> None:
    _check(load().glm_server_destroy(s), "glm_server_destroy")


def glm_slice_create(n_rows, p, ld, w=1.0, m=4, s_max=30, prior_sigma=10.0, device=0, spec=0):
    """Gibbs-slice sampler for column-major X (N rows, column stride ld);
    spec = shrinkage proposals per evaluation pass (0: default)."""
    d = glm_slice_desc_t(int(n_rows), int(ld), int(p), int(m), int(s_max), int(device),
                         float(w), int(spec), float(prior_sigma))
    s = C.c_void_p()
    _check(load().glm_slice_create(C.byref(d), C.byref(s)), "glm_slice_create")
    return s.value


def glm_slice_destroy(s) -> None:
    _check(load().glm_slice_destroy(s), "glm_slice_destroy")


def glm_slice_eta(s, Xt, beta, eta, stream=None) -> None:
    _check(load().glm_slice_eta(s, _ptr(Xt), _ptr(beta), _ptr(eta), _stream(stream)),
           "glm_slice_eta")


def glm_slice_coord_logpost(s, Xt, y, eta, beta, k, x, M, f_out, stream=None) -> None:
    _check(load().glm_slice_coord_logpost(s, _ptr(Xt), _ptr(y), _ptr(eta), _ptr(beta), int(k),
                                          _ptr(x), int(M), _ptr(f_out), _stream(stream)),
           "glm_slice_coord_logpost")


def glm_slice_run(s, Xt, y, eta, beta, f_state, init_f, n_sweeps, log_u0, uni, xk_out=None,
                  gk_out=None, nshrink_out=None, stream=None) -> None:
    _check(load().glm_slice_run(s, _ptr(Xt), _ptr(y), _ptr(eta), _ptr(beta), _ptr(f_state),
                                int(init_f), int(n_sweeps), _ptr(log_u0), _ptr(uni),
                                _ptr(xk_out), _ptr(gk_out), _ptr(nshrink_out), _stream(stream)),
           "glm_slice_run")


def glm_slice_sync(s, stream=None) -> int:
    return int(load().glm_slice_sync(s, _stream(stream)))


def glm_ising_split(nat, elem_bytes, rows, cols, plane0, plane1, stream=None) -> None:
    """Natural row-major array -> its two checkerboard colour planes."""
    _check(load().glm_ising_split(_ptr(nat), int(elem_bytes), int(rows), int(cols), _ptr(plane0),
                                  _ptr(plane1), _stream(stream)), "glm_ising_split")


def glm_ising_merge(plane0, plane1, elem_bytes, rows, cols, nat, stream=None) -> None:
    """Two checkerboard colour planes -> the natural row-major array."""
    _check(load().glm_ising_merge(_ptr(plane0), _ptr(plane1), int(elem_bytes), int(rows), int(cols),
                                  _ptr(nat), _stream(stream)), "glm_ising_merge")


def glm_ising_sweeps(s0, s1, b0, b1, rows, cols, w, n_sweeps, u, ones_out=None, stream=None) -> None:
    """n_sweeps checkerboard Gibbs sweeps of the Ising model on the spin planes."""
    _check(load().glm_ising_sweeps(_ptr(s0), _ptr(s1), _ptr(b0), _ptr(b1), int(rows), int(cols),
                                   float(w), int(n_sweeps), _ptr(u), _ptr(ones_out), _stream(stream)),
           "glm_ising_sweeps")


def glm_hess_create(n_rows, p, ld, prior_sigma=10.0, device=0):
    """Evaluator of f, g and the Hessian for N x P row-major FP32 X (P <= ld <= 64)."""
    h = C.c_void_p()
    _check(load().glm_hess_create(int(n_rows), int(p), int(ld), float(prior_sigma), int(device),
                                  C.byref(h)), "glm_hess_create")
    return h.value


def glm_hess_destroy(h) -> None:
    _check(load().glm_hess_destroy(h), "glm_hess_destroy")


def glm_hess_eval(h, X, y, beta, f_out, g_out, H_out, stream=None) -> None:
    _check(load().glm_hess_eval(h, _ptr(X), _ptr(y), _ptr(beta), _ptr(f_out), _ptr(g_out),
                                _ptr(H_out), _stream(stream)), "glm_hess_eval")


def glm_hess_sync(h, stream=None) -> int:
    return load().glm_hess_sync(h, _stream(stream))
