"""Thin Python binding of the FIFA-GP C ABI (include/fifa.h).

Argument marshalling only: every step runs in the CUDA library
``_lib/libfifa.so``.  PyTorch provides the device arena, the stream and the
device buffers (their ``data_ptr()`` is passed through).  Importing this module
does not load the library; the first call does, and it raises if the library
is missing -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfifa.so")

FIFA_OK, FIFA_ERR_INVALID_ARG, FIFA_ERR_UNSORTED, FIFA_ERR_NOT_SPD = 0, 1, 2, 3
FIFA_ERR_RANK_CAP, FIFA_ERR_OOM, FIFA_ERR_CUDA, FIFA_ERR_TIMEOUT, FIFA_ERR_UNSUPPORTED = 4, 5, 6, 7, 8
FIFA_KERNEL_SE, FIFA_KERNEL_MATERN52 = 0, 1
FIFA_FP64, FIFA_MIXED = 0, 1
FIFA_TRACE_FIELDS = 13
TRACE_COLUMNS = ["iter", "sigma2", "tau2", "rho", "accept", "log_alpha", "logdet", "q", "rss", "refine_res", "status",
                 "refactored", "cg_iters"]


class fifa_hyper(C.Structure):
    _fields_ = [("kernel", C.c_int), ("tau2", C.c_double), ("rho", C.c_double), ("sigma2", C.c_double),
                ("nugget", C.c_double)]


class fifa_opts(C.Structure):
    _fields_ = [("leaf_size", C.c_int), ("aca_tol", C.c_double), ("rank_cap", C.c_int), ("prec", C.c_int),
                ("refine_tol", C.c_double), ("refine_max", C.c_int), ("independent_ctas", C.c_int),
                ("wait_polls", C.c_int), ("coresident_share", C.c_int), ("overlap_proposal", C.c_int)]


class fifa_plan_info(C.Structure):
    _fields_ = [("levels", C.c_int), ("nleaf", C.c_int), ("leaf_max", C.c_int), ("aca_grouped_ctas", C.c_int),
                ("aca_solo_blocks", C.c_int), ("aca_warp_blocks", C.c_int), ("scratch_bytes", C.c_int64)]


class fifa_prior(C.Structure):
    _fields_ = [("a_tau2", C.c_double), ("b_tau2", C.c_double), ("a_sigma2", C.c_double), ("b_sigma2", C.c_double),
                ("logrho_mu", C.c_double), ("logrho_sd", C.c_double), ("prop_sd", C.c_double)]


class fifa_server_opts(C.Structure):
    _fields_ = [("opts", fifa_opts), ("hbm_budget", C.c_size_t), ("slots", C.c_int), ("wide_min_n", C.c_int64),
                ("wide_workers", C.c_int)]


class fifa_request(C.Structure):
    _fields_ = [("x_host", C.c_void_p), ("y_host", C.c_void_p), ("n", C.c_int64), ("init", fifa_hyper),
                ("prior", fifa_prior), ("seed", C.c_uint64), ("chain_id", C.c_uint64), ("iters", C.c_int),
                ("burn", C.c_int), ("ndraws", C.c_int)]


class fifa_result(C.Structure):
    _fields_ = [("status", C.c_int), ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("last", fifa_hyper), ("accept_rate", C.c_double), ("bytes", C.c_size_t)]


class fifa_server_counters(C.Structure):
    _fields_ = [("now", C.c_double), ("queued", C.c_int), ("in_flight", C.c_int), ("peak_in_flight", C.c_int),
                ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t), ("completed", C.c_uint64),
                ("iterations_done", C.c_uint64)]


class FifaError(RuntimeError):
    def __init__(self, code, where, detail=""):
        self.code = code
        super().__init__(f"{where}: {status_str(code)} ({code}){detail}")


_lib = None
_P = C.c_void_p


def lib():
    """Load libfifa.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"FIFA CUDA library not built: {LIB_PATH} missing (run __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    sig = {
        "fifa_create": (C.c_int, [C.POINTER(_P), C.POINTER(fifa_opts), _P, _P, C.c_size_t]),
        "fifa_destroy_ctx": (None, [_P]),
        "fifa_assemble": (C.c_int, [_P, _P, C.c_int64, C.POINTER(fifa_hyper), C.POINTER(_P)]),
        "fifa_shift_scale": (C.c_int, [_P, _P, C.c_double, C.POINTER(_P)]),
        "fifa_add_diagonal": (C.c_int, [_P, _P, C.c_double, _P, C.POINTER(_P)]),
        "fifa_sample_hetero": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, _P, C.c_uint64, C.c_uint64, C.c_uint64,
                                         _P, _P]),
        "fifa_predict": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int64, C.c_double, _P, _P]),
        "fifa_grid_create": (C.c_int, [_P, _P, C.c_int64, C.c_int, C.c_double, _P, C.c_int, _P, C.POINTER(_P)]),
        "fifa_grid_draw": (C.c_int, [_P, _P, _P, C.c_double, C.c_uint64, C.c_uint64, C.c_uint64,
                                     C.POINTER(C.c_int), _P]),
        "fifa_grid_get": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.POINTER(_P)]),
        "fifa_destroy_grid": (None, [_P, _P]),
        "fifa_factor": (C.c_int, [_P, _P, C.POINTER(_P)]),
        "fifa_logdet": (C.c_int, [_P, _P, C.POINTER(C.c_double)]),
        "fifa_solve": (C.c_int, [_P, _P, _P, _P, C.c_int]),
        "fifa_apply_W": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P, C.c_int]),
        "fifa_apply_precond": (C.c_int, [_P, _P, _P, _P, C.c_int]),
        "fifa_matvec": (C.c_int, [_P, _P, _P, _P, C.c_int]),
        "fifa_matvec_static": (C.c_int, [_P, _P, _P, _P, C.c_int]),
        "fifa_sample": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, C.c_double, C.c_uint64, C.c_uint64, C.c_uint64,
                                  _P, _P]),
        "fifa_chain_create": (C.c_int, [_P, _P, _P, C.c_int64, C.POINTER(fifa_hyper), C.POINTER(fifa_prior),
                                        C.c_uint64, C.c_uint64, C.POINTER(_P)]),
        "fifa_gibbs_step": (C.c_int, [_P, _P, C.c_int, _P]),
        "fifa_chain_get": (C.c_int, [_P, _P, _P, _P, C.POINTER(fifa_hyper)]),
        "fifa_chain_set_y": (C.c_int, [_P, _P, _P]),
        "fifa_chain_kernel_nodes": (C.c_int, [_P, C.POINTER(C.c_int)]),
        "fifa_chain_bytes": (C.c_int, [C.POINTER(fifa_opts), C.c_int64, C.POINTER(C.c_size_t)]),
        "fifa_server_create": (C.c_int, [C.POINTER(fifa_server_opts), C.POINTER(_P)]),
        "fifa_server_submit": (C.c_int, [_P, C.POINTER(fifa_request), C.POINTER(C.c_uint64)]),
        "fifa_server_wait": (C.c_int, [_P, C.c_uint64, _P, _P, C.POINTER(fifa_result)]),
        "fifa_server_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(C.c_int)]),
        "fifa_server_stats": (C.c_int, [_P, C.POINTER(fifa_server_counters)]),
        "fifa_server_destroy": (None, [_P]),
        "fifa_additive_create": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int, C.POINTER(fifa_hyper),
                                           C.POINTER(fifa_prior), C.c_uint64, C.POINTER(_P)]),
        "fifa_additive_sweep": (C.c_int, [_P, _P, C.c_int, _P]),
        "fifa_additive_get": (C.c_int, [_P, _P, _P, C.POINTER(C.c_double), C.POINTER(fifa_hyper)]),
        "fifa_additive_kernel_nodes": (C.c_int, [_P, C.POINTER(C.c_int)]),
        "fifa_destroy_additive": (None, [_P, _P]),
        "fifa_tensor_create": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int, C.POINTER(fifa_hyper), C.POINTER(fifa_prior),
                                         C.c_double, C.c_double, C.c_double, C.c_uint64, C.POINTER(_P)]),
        "fifa_tensor_sweep": (C.c_int, [_P, _P, C.c_int, _P]),
        "fifa_tensor_get": (C.c_int, [_P, _P, _P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(fifa_hyper)]),
        "fifa_destroy_tensor": (None, [_P, _P]),
        "fifa_hmat_dims": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "fifa_plan_describe": (C.c_int, [C.POINTER(fifa_opts), C.c_int64, C.c_int, _P, C.POINTER(fifa_plan_info), _P, _P, _P]),
        "fifa_hmat_level_rows": (C.c_int, [_P, _P, C.c_int, C.c_int64, C.c_int64, _P]),
        "fifa_hmat_export": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
        "fifa_fact_export": (C.c_int, [_P, _P, _P, _P, _P, _P]),
        "fifa_destroy_hmat": (None, [_P, _P]),
        "fifa_destroy_fact": (None, [_P, _P]),
        "fifa_destroy_chain": (None, [_P, _P]),
        "fifa_status_str": (C.c_char_p, [C.c_int]),
        "fifa_last_cuda_error": (C.c_char_p, [_P]),
        "fifa_det_exp": (C.c_int, [_P, _P, _P, C.c_int64]),
        "fifa_normals": (C.c_int, [_P, C.c_uint64, C.c_uint32, C.c_uint64, C.c_uint64, _P, C.c_int64]),
        "fifa_philox": (C.c_int, [_P, C.c_uint64, _P, _P, C.c_int64]),
        "fifa_probe_fp64_fma": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def status_str(code: int) -> str:
    return lib().fifa_status_str(int(code)).decode()


def _check(code, where, allow=(), ctx=None):
    if code != FIFA_OK and code not in allow:
        detail = ""
        if code == FIFA_ERR_CUDA and ctx is not None:
            detail = " [" + lib().fifa_last_cuda_error(ctx).decode() + "]"
        raise FifaError(code, where, detail)
    return code


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


# ---------------------------------------------------------------------------
# One function per C entry point.
# ---------------------------------------------------------------------------
def fifa_create(opts: fifa_opts, stream_ptr: int, arena_ptr: int, arena_bytes: int):
    h = C.c_void_p()
    _check(lib().fifa_create(C.byref(h), C.byref(opts), C.c_void_p(stream_ptr), C.c_void_p(arena_ptr),
                             C.c_size_t(arena_bytes)), "fifa_create")
    return h


def fifa_destroy_ctx(ctx):
    lib().fifa_destroy_ctx(ctx)


def fifa_assemble(ctx, x, n: int, hyper: fifa_hyper):
    h = C.c_void_p()
    _check(lib().fifa_assemble(ctx, _ptr(x), C.c_int64(n), C.byref(hyper), C.byref(h)), "fifa_assemble", ctx=ctx)
    return h


def fifa_shift_scale(ctx, Cm, s: float):
    h = C.c_void_p()
    _check(lib().fifa_shift_scale(ctx, Cm, C.c_double(s), C.byref(h)), "fifa_shift_scale", ctx=ctx)
    return h


def fifa_add_diagonal(ctx, Cm, s: float, diag):
    h = C.c_void_p()
    _check(lib().fifa_add_diagonal(ctx, Cm, C.c_double(s), _ptr(diag), C.byref(h)), "fifa_add_diagonal", ctx=ctx)
    return h


def fifa_sample_hetero(ctx, Cm, WC, WP, y, tau2, d, seed, stream_id, it, f, R=None):
    _check(lib().fifa_sample_hetero(ctx, Cm, WC, WP, _ptr(y), C.c_double(tau2), _ptr(d), C.c_uint64(seed),
                                    C.c_uint64(stream_id), C.c_uint64(it), _ptr(f), _ptr(R)), "fifa_sample_hetero",
           ctx=ctx)


def fifa_predict(ctx, Cm, WC, x, f, xstar, nstar, tau2, mu=None, var=None):
    _check(lib().fifa_predict(ctx, Cm, WC, _ptr(x), _ptr(f), _ptr(xstar), C.c_int64(nstar), C.c_double(tau2), _ptr(mu),
                              _ptr(var)), "fifa_predict", ctx=ctx)


def fifa_grid_create(ctx, x, n, kernel, nugget, rhos, log_prior=None):
    r = np.ascontiguousarray(rhos, dtype=np.float64)
    lp = np.ascontiguousarray(log_prior, dtype=np.float64) if log_prior is not None else None
    h = C.c_void_p()
    _check(lib().fifa_grid_create(ctx, _ptr(x), C.c_int64(n), int(kernel), C.c_double(nugget), _np_ptr(r), len(r),
                                  _np_ptr(lp), C.byref(h)), "fifa_grid_create", ctx=ctx)
    return h


def fifa_grid_draw(ctx, grid, f, tau2, seed, stream_id, it, G=None):
    """(index, probabilities (G floats, when G is given))."""
    idx = C.c_int()
    pr = np.zeros(G) if G else None
    _check(lib().fifa_grid_draw(ctx, grid, _ptr(f), C.c_double(tau2), C.c_uint64(seed), C.c_uint64(stream_id),
                                C.c_uint64(it), C.byref(idx), _np_ptr(pr)), "fifa_grid_draw", ctx=ctx)
    return idx.value, pr


def fifa_grid_get(grid, h):
    Cm, W = C.c_void_p(), C.c_void_p()
    _check(lib().fifa_grid_get(grid, int(h), C.byref(Cm), C.byref(W)), "fifa_grid_get")
    return Cm, W


def fifa_destroy_grid(ctx, grid):
    lib().fifa_destroy_grid(ctx, grid)


def fifa_factor(ctx, A):
    h = C.c_void_p()
    _check(lib().fifa_factor(ctx, A, C.byref(h)), "fifa_factor", ctx=ctx)
    return h


def fifa_logdet(ctx, F, allow=()):
    out = C.c_double()
    code = _check(lib().fifa_logdet(ctx, F, C.byref(out)), "fifa_logdet", allow, ctx=ctx)
    return out.value, code


def fifa_solve(ctx, F, b, x, nrhs: int = 1):
    _check(lib().fifa_solve(ctx, F, _ptr(b), _ptr(x), int(nrhs)), "fifa_solve", ctx=ctx)


def fifa_apply_W(ctx, F, trans: int, inverse: int, x_in, x_out, nrhs: int = 1):
    _check(lib().fifa_apply_W(ctx, F, int(trans), int(inverse), _ptr(x_in), _ptr(x_out), int(nrhs)), "fifa_apply_W", ctx=ctx)


def fifa_apply_precond(ctx, F, x_in, x_out, nrhs: int = 1):
    _check(lib().fifa_apply_precond(ctx, F, _ptr(x_in), _ptr(x_out), int(nrhs)), "fifa_apply_precond", ctx=ctx)


def fifa_matvec(ctx, A, x_in, x_out, nrhs: int = 1):
    _check(lib().fifa_matvec(ctx, A, _ptr(x_in), _ptr(x_out), int(nrhs)), "fifa_matvec", ctx=ctx)


def fifa_matvec_static(ctx, A, x_in, x_out, nrhs: int = 1, allow=()):
    return _check(lib().fifa_matvec_static(ctx, A, _ptr(x_in), _ptr(x_out), int(nrhs)), "fifa_matvec_static", allow,
                  ctx=ctx)


def fifa_sample(ctx, Cm, WC, WM, y, tau2, sigma2, seed, stream_id, it, f, mean=None):
    _check(lib().fifa_sample(ctx, Cm, WC, WM, _ptr(y), C.c_double(tau2), C.c_double(sigma2), C.c_uint64(seed),
                             C.c_uint64(stream_id), C.c_uint64(it), _ptr(f), _ptr(mean)), "fifa_sample", ctx=ctx)


def fifa_chain_create(ctx, x, y, n, init: fifa_hyper, prior: fifa_prior, seed: int, chain_id: int):
    h = C.c_void_p()
    _check(lib().fifa_chain_create(ctx, _ptr(x), _ptr(y), C.c_int64(n), C.byref(init), C.byref(prior),
                                   C.c_uint64(seed), C.c_uint64(chain_id), C.byref(h)), "fifa_chain_create", ctx=ctx)
    return h


def fifa_gibbs_step(ctx, chain, iters: int, trace: np.ndarray | None = None, allow=()):
    tp = trace.ctypes.data_as(C.c_void_p) if trace is not None else None
    return _check(lib().fifa_gibbs_step(ctx, chain, int(iters), tp), "fifa_gibbs_step", allow, ctx=ctx)


def fifa_chain_get(ctx, chain, f=None, mean=None):
    h = fifa_hyper()
    _check(lib().fifa_chain_get(ctx, chain, _ptr(f), _ptr(mean), C.byref(h)), "fifa_chain_get", ctx=ctx)
    return h


def fifa_chain_set_y(ctx, chain, y):
    """y: a torch tensor on the device or in (pinned) host memory; copied on the context's stream."""
    _check(lib().fifa_chain_set_y(ctx, chain, _ptr(y)), "fifa_chain_set_y", ctx=ctx)


def fifa_chain_kernel_nodes(chain):
    k = C.c_int()
    _check(lib().fifa_chain_kernel_nodes(chain, C.byref(k)), "fifa_chain_kernel_nodes")
    return k.value


FIFA_ADDITIVE_MAX_D = 16


def fifa_chain_bytes(opts: fifa_opts, n: int) -> int:
    b = C.c_size_t()
    _check(lib().fifa_chain_bytes(C.byref(opts), C.c_int64(n), C.byref(b)), "fifa_chain_bytes")
    return b.value


def fifa_additive_trace_fields(d: int) -> int:
    return 5 + 3 * d


def fifa_additive_create(ctx, X_cols, y, n, d, init: fifa_hyper, prior: fifa_prior, seed: int):
    """X_cols: d x n device doubles (coordinate k of point i at [k, i])."""
    h = C.c_void_p()
    _check(lib().fifa_additive_create(ctx, _ptr(X_cols), _ptr(y), C.c_int64(n), C.c_int(d), C.byref(init),
                                      C.byref(prior), C.c_uint64(seed), C.byref(h)), "fifa_additive_create", ctx=ctx)
    return h


def fifa_additive_sweep(ctx, model, sweeps: int, trace: np.ndarray | None = None, allow=()):
    tp = trace.ctypes.data_as(C.c_void_p) if trace is not None else None
    return _check(lib().fifa_additive_sweep(ctx, model, int(sweeps), tp), "fifa_additive_sweep", allow, ctx=ctx)


def fifa_additive_get(ctx, model, d: int, F=None):
    """Returns (sigma2, [fifa_hyper] * d); F (d x n device doubles) receives f_1..f_d."""
    s2 = C.c_double()
    hs = (fifa_hyper * d)()
    _check(lib().fifa_additive_get(ctx, model, _ptr(F), C.byref(s2), hs), "fifa_additive_get", ctx=ctx)
    return s2.value, list(hs)


def fifa_additive_kernel_nodes(model):
    k = C.c_int()
    _check(lib().fifa_additive_kernel_nodes(model, C.byref(k)), "fifa_additive_kernel_nodes")
    return k.value


def fifa_destroy_additive(ctx, model):
    lib().fifa_destroy_additive(ctx, model)


def fifa_tensor_trace_fields(d: int) -> int:
    return 5 + 2 * d


def fifa_tensor_create(ctx, X_cols, y, n, d, init: fifa_hyper, prior: fifa_prior, beta0: float, beta_mu: float,
                       beta_sd: float, seed: int):
    """X_cols: d x n device doubles (coordinate h of point i at [h, i])."""
    h = C.c_void_p()
    _check(lib().fifa_tensor_create(ctx, _ptr(X_cols), _ptr(y), C.c_int64(n), C.c_int(d), C.byref(init),
                                    C.byref(prior), C.c_double(beta0), C.c_double(beta_mu), C.c_double(beta_sd),
                                    C.c_uint64(seed), C.byref(h)), "fifa_tensor_create", ctx=ctx)
    return h


def fifa_tensor_sweep(ctx, model, sweeps: int, trace: np.ndarray | None = None, allow=()):
    tp = trace.ctypes.data_as(C.c_void_p) if trace is not None else None
    return _check(lib().fifa_tensor_sweep(ctx, model, int(sweeps), tp), "fifa_tensor_sweep", allow, ctx=ctx)


def fifa_tensor_get(ctx, model, d: int, F=None):
    """Returns (beta, sigma2, [fifa_hyper] * d); F (d x n device doubles) receives f_1..f_d."""
    b, s2 = C.c_double(), C.c_double()
    hs = (fifa_hyper * d)()
    _check(lib().fifa_tensor_get(ctx, model, _ptr(F), C.byref(b), C.byref(s2), hs), "fifa_tensor_get", ctx=ctx)
    return b.value, s2.value, list(hs)


def fifa_destroy_tensor(ctx, model):
    lib().fifa_destroy_tensor(ctx, model)


def fifa_server_create(opts: fifa_opts, hbm_budget: int, slots: int, wide_min_n: int = 0, wide_workers: int = 1):
    h = C.c_void_p()
    so = fifa_server_opts(opts, C.c_size_t(int(hbm_budget)), int(slots), int(wide_min_n), int(wide_workers))
    _check(lib().fifa_server_create(C.byref(so), C.byref(h)), "fifa_server_create")
    return h


def fifa_server_submit(server, x: np.ndarray, y: np.ndarray, init: fifa_hyper, prior: fifa_prior, seed: int,
                       chain_id: int, iters: int, burn: int, ndraws: int) -> int:
    """x, y: host float64 arrays (copied by the call)."""
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    r = fifa_request(x.ctypes.data, y.ctypes.data, len(x), init, prior, int(seed), int(chain_id), int(iters),
                     int(burn), int(ndraws))
    rid = C.c_uint64()
    _check(lib().fifa_server_submit(server, C.byref(r), C.byref(rid)), "fifa_server_submit")
    return rid.value


def fifa_server_wait(server, rid: int, mean: np.ndarray | None = None, draws: np.ndarray | None = None, allow=()):
    """Blocks until request rid is done; returns (status, fifa_result)."""
    res = fifa_result()
    mp = mean.ctypes.data_as(C.c_void_p) if mean is not None else None
    dp = draws.ctypes.data_as(C.c_void_p) if draws is not None else None
    st = _check(lib().fifa_server_wait(server, C.c_uint64(rid), mp, dp, C.byref(res)), "fifa_server_wait", allow)
    return st, res


def fifa_server_poll(server, rid: int) -> bool:
    done = C.c_int(0)
    _check(lib().fifa_server_poll(server, C.c_uint64(rid), C.byref(done)), "fifa_server_poll")
    return bool(done.value)


def fifa_server_stats(server) -> fifa_server_counters:
    c = fifa_server_counters()
    _check(lib().fifa_server_stats(server, C.byref(c)), "fifa_server_stats")
    return c


def fifa_server_destroy(server):
    lib().fifa_server_destroy(server)


def fifa_hmat_dims(H):
    n, L, nl, bm, cap = C.c_int64(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(lib().fifa_hmat_dims(H, C.byref(n), C.byref(L), C.byref(nl), C.byref(bm), C.byref(cap)), "fifa_hmat_dims")
    return n.value, L.value, nl.value, bm.value, cap.value


def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def fifa_plan_describe(opts, n: int, aca_cores: int, lvl_cores) -> dict:
    """Host-only plan for n points: info, tree bounds, ACA work list (k x 4) and level group sizes (3 x L)."""
    lc = np.ascontiguousarray(lvl_cores, dtype=np.int32)
    info = fifa_plan_info()
    _check(lib().fifa_plan_describe(C.byref(opts), int(n), int(aca_cores), _np_ptr(lc), C.byref(info), None, None,
                                    None), "fifa_plan_describe")
    L = info.levels
    nb = (1 << (L + 1)) + L  # levels 0..L, 2^l + 1 bounds each
    nw = info.aca_grouped_ctas + info.aca_solo_blocks + info.aca_warp_blocks
    bounds = np.zeros(nb, np.int32)
    work = np.zeros(max(1, 4 * nw), np.int32)
    groups = np.zeros(max(1, 3 * L), np.int32)
    _check(lib().fifa_plan_describe(C.byref(opts), int(n), int(aca_cores), _np_ptr(lc), C.byref(info),
                                    _np_ptr(bounds), _np_ptr(work), _np_ptr(groups)), "fifa_plan_describe")
    return dict(info=info, bounds=bounds, work=work[:4 * nw].reshape(nw, 4), groups=groups[:3 * L].reshape(3, L))


def fifa_hmat_level_rows(ctx, H, level: int, row0: int, nrows: int) -> np.ndarray:
    """(rank_cap, nrows) array: the level's basis columns on rows [row0, row0 + nrows)."""
    cap = fifa_hmat_dims(H)[4]
    out = np.zeros((cap, nrows))
    _check(lib().fifa_hmat_level_rows(ctx, H, int(level), int(row0), int(nrows), _np_ptr(out)), "fifa_hmat_level_rows")
    return out


def fifa_hmat_export(ctx, H, allow=(FIFA_ERR_RANK_CAP,), bases=True, leaves=True):
    n, L, nl, bm, cap = fifa_hmat_dims(H)
    nn = max(1, (1 << L) - 1)
    ranks = np.zeros(nn, np.int32)
    rp = np.zeros(nn * cap, np.int32)
    cp = np.zeros(nn * cap, np.int32)
    bs = np.zeros(max(1, L) * cap * n) if bases else None
    lv = np.zeros(nl * bm * bm) if leaves else None
    code = _check(lib().fifa_hmat_export(ctx, H, _np_ptr(ranks), _np_ptr(rp), _np_ptr(cp), _np_ptr(bs),
                                         _np_ptr(lv)), "fifa_hmat_export", allow)
    return dict(n=n, L=L, nleaf=nl, Bm=bm, cap=cap, ranks=ranks, row_piv=rp.reshape(nn, cap),
                col_piv=cp.reshape(nn, cap), bases=bs.reshape(max(1, L), cap, n) if bases else None,
                leaves=lv.reshape(nl, bm, bm) if leaves else None, status=code)


def fifa_fact_export(ctx, F, dims, allow=()):
    n, L, nl, bm, cap = dims
    nn = max(1, (1 << L) - 1)
    bases = np.zeros(max(1, L) * cap * n)
    leaves = np.zeros(nl * bm * bm)
    zf = np.zeros(nn * 4 * cap * cap)
    zi = np.zeros(nn * 4 * cap * cap)
    code = _check(lib().fifa_fact_export(ctx, F, _np_ptr(bases), _np_ptr(leaves), _np_ptr(zf), _np_ptr(zi)),
                  "fifa_fact_export", allow)
    return dict(bases=bases.reshape(max(1, L), cap, n), leaves=leaves.reshape(nl, bm, bm),
                Zf=zf.reshape(nn, 2 * cap, 2 * cap), Zi=zi.reshape(nn, 2 * cap, 2 * cap), status=code)


def fifa_destroy_hmat(ctx, H):
    lib().fifa_destroy_hmat(ctx, H)


def fifa_destroy_fact(ctx, F):
    lib().fifa_destroy_fact(ctx, F)


def fifa_destroy_chain(ctx, ch):
    lib().fifa_destroy_chain(ctx, ch)


def fifa_det_exp(ctx, x_in, x_out, n):
    _check(lib().fifa_det_exp(ctx, _ptr(x_in), _ptr(x_out), C.c_int64(n)), "fifa_det_exp", ctx=ctx)


def fifa_normals(ctx, seed, tag, it, stream_id, out, n):
    _check(lib().fifa_normals(ctx, C.c_uint64(seed), C.c_uint32(tag), C.c_uint64(it), C.c_uint64(stream_id),
                              _ptr(out), C.c_int64(n)), "fifa_normals", ctx=ctx)


def fifa_philox(ctx, seed, ctr, out, count):
    _check(lib().fifa_philox(ctx, C.c_uint64(seed), _ptr(ctr), _ptr(out), C.c_int64(count)), "fifa_philox", ctx=ctx)


def fifa_probe_fp64_fma(ctx, iters: int = 200000):
    """(TFLOP/s, ms) of the FP64 fused multiply-add probe (synchronizes)."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib().fifa_probe_fp64_fma(ctx, int(iters), C.byref(tf), C.byref(ms)), "fifa_probe_fp64_fma", ctx=ctx)
    return tf.value, ms.value


# ---------------------------------------------------------------------------
# Convenience: a context whose arena and stream come from PyTorch.
# ---------------------------------------------------------------------------
class Context:
    def __init__(self, leaf_size=64, aca_tol=1e-12, rank_cap=32, prec=FIFA_FP64, refine_tol=1e-12, refine_max=3,
                 arena_bytes=1 << 30, device="cuda", stream=None, independent_ctas=0, wait_polls=0,
                 coresident_share=0, overlap_proposal=0):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=self.device)
        self.opts = fifa_opts(int(leaf_size), float(aca_tol), int(rank_cap), int(prec), float(refine_tol),
                              int(refine_max), int(independent_ctas), int(wait_polls), int(coresident_share),
                              int(overlap_proposal))
        self.h = fifa_create(self.opts, self.stream.cuda_stream, self.arena.data_ptr(), int(arena_bytes))

    def close(self):
        if self.h is not None:
            fifa_destroy_ctx(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
