"""ctypes binding of libdscreen (include/dscreen.h), one Python function per C entry point.

Argument marshalling only: every step of a solve runs in the CUDA library.
Arrays may be CUDA ``torch.Tensor`` objects (device memory) or NumPy arrays
(host memory); the library copies host data itself.  Dictionaries are
column-major N x K (a torch tensor of shape (N, K) with stride (1, ld), or a
Fortran-ordered NumPy array).  Non-OK statuses raise :class:`DscreenError`.
There is no fallback: if the CUDA library cannot be built or loaded, importing
a function raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "dscreen.h")

(DS_OK, DS_ERR_INVALID, DS_ERR_OOM, DS_ERR_CUDA, DS_ERR_TIMEOUT, DS_ERR_NOT_CONVERGED, DS_ERR_UNSUPPORTED,
 DS_PENDING) = range(8)
DS_ISTA, DS_FISTA, DS_CP, DS_SPARSA, DS_TWIST = 0, 1, 2, 3, 4
DS_TEST_NONE, DS_SAFE, DS_DST3, DS_DOME, DS_GSAFE, DS_DGST3 = range(6)
DS_FP64, DS_FP32, DS_BF16, DS_FP8 = range(4)
TESTS = {"none": DS_TEST_NONE, "safe": DS_SAFE, "dst3": DS_DST3, "dome": DS_DOME, "gsafe": DS_GSAFE,
         "dgst3": DS_DGST3}
ALGS = {"ista": DS_ISTA, "fista": DS_FISTA, "cp": DS_CP, "sparsa": DS_SPARSA, "twist": DS_TWIST}
HIST_COLS = ("active", "nnz", "R", "radius", "gap", "mu")


class ds_options(ctypes.Structure):
    _fields_ = [("alg", ctypes.c_int), ("test", ctypes.c_int), ("dynamic", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("tol_gap_rel", ctypes.c_double), ("L", ctypes.c_double),
                ("lambda_rel", ctypes.c_int), ("lowp_switch", ctypes.c_double),
                ("batch_multi_rhs", ctypes.c_int), ("warm_start", ctypes.c_int), ("cp_tau", ctypes.c_double),
                ("cp_sigma", ctypes.c_double), ("cp_gamma", ctypes.c_double), ("step_backtracking", ctypes.c_int),
                ("bt_L0", ctypes.c_double), ("twist_xi1", ctypes.c_double), ("gap_every", ctypes.c_int),
                ("team_size", ctypes.c_int)]


class ds_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("n_active", ctypes.c_int64),
                ("nnz", ctypes.c_int64), ("gap", ctypes.c_double), ("primal", ctypes.c_double),
                ("dual", ctypes.c_double), ("lambda_", ctypes.c_double), ("lambda_max", ctypes.c_double),
                ("ms", ctypes.c_double), ("cols_corr", ctypes.c_int64), ("cols_synth", ctypes.c_int64),
                ("cols_lowp", ctypes.c_int64)]

    def as_dict(self):
        return {"iters": self.iters, "status": self.status, "n_active": self.n_active, "nnz": self.nnz,
                "gap": self.gap, "primal": self.primal, "dual": self.dual, "lambda": self.lambda_,
                "lambda_max": self.lambda_max, "ms": self.ms, "cols_corr": self.cols_corr,
                "cols_synth": self.cols_synth, "cols_lowp": self.cols_lowp}


class DscreenError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {lib().ds_status_str(status).decode()} ({status})")


def declared_functions():
    """Names of the entry points declared in include/dscreen.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ds_[a-z_]+)\s*\(", txt)))


def lib():
    """Load (building first if needed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
            L.ds_status_str.restype = ctypes.c_char_p
            L.ds_status_str.argtypes = [ctypes.c_int]
            L.ds_options_default.argtypes = [ctypes.POINTER(ds_options)]
            L.ds_create.argtypes = [ctypes.c_int, vp, ctypes.POINTER(vp)]
            L.ds_destroy.argtypes = [vp]
            L.ds_dict_create.argtypes = [vp, vp, i64, i64, i64, ctypes.c_int, vp, vp, i64, ctypes.c_int,
                                         ctypes.POINTER(vp)]
            L.ds_dict_destroy.argtypes = [vp]
            L.ds_dict_lipschitz.argtypes = [vp, ctypes.POINTER(dp)]
            L.ds_lambda_max.argtypes = [vp, vp, vp, ctypes.POINTER(dp)]
            L.ds_solve.argtypes = [vp, vp, vp, dp, ctypes.POINTER(ds_options), vp, vp, ctypes.POINTER(ds_result)]
            L.ds_solve_path.argtypes = [vp, vp, vp, ctypes.c_int, vp, ctypes.POINTER(ds_options), vp, vp,
                                        ctypes.POINTER(ds_result)]
            L.ds_set_history.argtypes = [vp, vp, ctypes.c_int]
            L.ds_set_screen_log.argtypes = [vp, vp, i64]
            L.ds_selftest_wait_timeout.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(dp)]
            L.ds_ctx_kernel_launches.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
            L.ds_batch_create.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, ctypes.POINTER(ds_options), vp,
                                          ctypes.POINTER(vp)]
            L.ds_batch_run.argtypes = [vp, vp]
            L.ds_batch_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int)]
            L.ds_batch_layout.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int)] * 4
            L.ds_batch_autotune.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
            L.ds_batch_schedule.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int)] * 3 + [ctypes.POINTER(ctypes.c_double)]
            L.ds_batch_destroy.argtypes = [vp]
            L.ds_solve_batch.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, ctypes.POINTER(ds_options), vp, vp]
            L.ds_server_create.argtypes = [vp, ctypes.c_size_t, i64, i64, ctypes.c_int, ctypes.POINTER(vp)]
            L.ds_server_submit.argtypes = [vp, vp, vp, dp, ctypes.POINTER(ds_options), vp,
                                           ctypes.POINTER(ctypes.c_uint64)]
            L.ds_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ds_result)]
            L.ds_server_stats.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int64)] * 4 + [ctypes.POINTER(ctypes.c_size_t)]
            L.ds_server_destroy.argtypes = [vp]
            L.ds_solve_lasso_noalloc.argtypes = [ctypes.c_int, vp, vp, i64, i64, i64, vp, dp,
                                                 ctypes.POINTER(ds_options), vp, ctypes.POINTER(ds_result)]
            for name in declared_functions():
                if name != "ds_status_str":
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(st, where):
    if st != DS_OK:
        raise DscreenError(st, where)


# ----------------------------------------------------------------- marshalling

def _ptr(a):
    """(address, is_torch) of a torch tensor or NumPy array; None -> (None, False)."""
    if a is None:
        return None, False
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), True
    return a.ctypes.data, False


def _dtype_code(a):
    name = str(a.dtype)
    if name.endswith("float32"):
        return DS_FP32
    if name.endswith("float64"):
        return DS_FP64
    raise TypeError(f"dictionary dtype must be float32 or float64, got {a.dtype}")


class _DictHandle(ctypes.c_void_p):
    """A registered dictionary: the C handle, plus its N, K and element size for the
    buffer checks of the calls that take it."""


def _check_buffer(a, n, esize, name, where):
    """A vector argument must be contiguous, hold the dictionary's element type and
    at least n elements: the library writes and reads exactly that many through the
    raw pointer, so a short buffer would be an out-of-bounds access."""
    if a is None:
        return
    if hasattr(a, "data_ptr"):
        count, size, contiguous = a.numel(), a.element_size(), a.is_contiguous()
    else:
        count, size, contiguous = a.size, a.itemsize, a.flags.c_contiguous
    if size != esize:
        raise TypeError(f"{where}: {name} has {size}-byte elements, the dictionary {esize}-byte ones")
    if not contiguous:
        raise ValueError(f"{where}: {name} must be contiguous (row-major)")
    if count < n:
        raise ValueError(f"{where}: {name} has {count} elements, {n} needed")


def _check_vectors(dct, where, y=None, x_out=None, x0=None, n_lambda=1):
    N, K, esize = getattr(dct, "N", None), getattr(dct, "K", None), getattr(dct, "esize", None)
    if N is None:
        return
    _check_buffer(y, N, esize, "y", where)
    _check_buffer(x_out, K * n_lambda, esize, "x_out", where)
    _check_buffer(x0, K, esize, "x0", where)


def _dict_layout(D):
    N, K = D.shape
    if hasattr(D, "stride"):
        s0, s1 = D.stride()
        if s0 != 1 and K > 1:
            raise ValueError("torch dictionary must be column-major: stride (1, ld)")
        return N, K, (s1 if K > 1 else N)
    if not D.flags.f_contiguous:
        raise ValueError("NumPy dictionary must be Fortran-ordered (column-major)")
    return N, K, N


# -------------------------------------------------------------------- entry points

def ds_status_str(status: int) -> str:
    return lib().ds_status_str(int(status)).decode()


def ds_options_default(**kw) -> ds_options:
    o = ds_options()
    _check(lib().ds_options_default(ctypes.byref(o)), "ds_options_default")
    for k, v in kw.items():
        if k == "test" and isinstance(v, str):
            v = TESTS[v]
        if k == "alg" and isinstance(v, str):
            v = ALGS[v]
        setattr(o, k, v)
    return o


def ds_create(device: int = 0, stream=None):
    h = ctypes.c_void_p()
    s = None
    if stream is not None:
        s = getattr(stream, "cuda_stream", stream)
    _check(lib().ds_create(int(device), s, ctypes.byref(h)), "ds_create")
    return h


def ds_destroy(ctx):
    _check(lib().ds_destroy(ctx), "ds_destroy")


def ds_dict_create(ctx, D, group_offsets=None, weights=None, work_prec=None):
    N, K, ld = _dict_layout(D)
    dt = _dtype_code(D)
    goff = None if group_offsets is None else np.ascontiguousarray(group_offsets, dtype=np.int64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    if w is not None and (goff is None or w.size != goff.size - 1):
        raise ValueError("ds_dict_create: weights need group_offsets and one value per group")
    h = _DictHandle()
    h.N, h.K, h.esize = N, K, 4 if dt == DS_FP32 else 8
    p, _ = _ptr(D)
    st = lib().ds_dict_create(ctx, p, N, K, ld, dt, None if goff is None else goff.ctypes.data,
                              None if w is None else w.ctypes.data, 0 if goff is None else goff.size - 1,
                              dt if work_prec is None else int(work_prec), ctypes.byref(h))
    _check(st, "ds_dict_create")
    return h


def ds_dict_destroy(dct):
    _check(lib().ds_dict_destroy(dct), "ds_dict_destroy")


def ds_dict_lipschitz(dct) -> float:
    L = ctypes.c_double()
    _check(lib().ds_dict_lipschitz(dct, ctypes.byref(L)), "ds_dict_lipschitz")
    return L.value


def ds_lambda_max(ctx, dct, y) -> float:
    _check_vectors(dct, "ds_lambda_max", y=y)
    v = ctypes.c_double()
    _check(lib().ds_lambda_max(ctx, dct, _ptr(y)[0], ctypes.byref(v)), "ds_lambda_max")
    return v.value


def ds_solve(ctx, dct, y, lam, opt, x_out, x0=None):
    _check_vectors(dct, "ds_solve", y=y, x_out=x_out, x0=x0)
    r = ds_result()
    st = lib().ds_solve(ctx, dct, _ptr(y)[0], float(lam), ctypes.byref(opt), _ptr(x0)[0], _ptr(x_out)[0],
                        ctypes.byref(r))
    _check(st, "ds_solve")
    return r.as_dict()


def ds_solve_path(ctx, dct, y, lambdas, opt, X_out, x0=None):
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    _check_vectors(dct, "ds_solve_path", y=y, x_out=X_out, x0=x0, n_lambda=lam.size)
    res = (ds_result * lam.size)()
    st = lib().ds_solve_path(ctx, dct, _ptr(y)[0], int(lam.size), lam.ctypes.data, ctypes.byref(opt),
                             _ptr(x0)[0], _ptr(X_out)[0], res)
    _check(st, "ds_solve_path")
    return [r.as_dict() for r in res]


def ds_ctx_kernel_launches(ctx) -> int:
    n = ctypes.c_int64()
    _check(lib().ds_ctx_kernel_launches(ctx, ctypes.byref(n)), "ds_ctx_kernel_launches")
    return n.value


class _BatchArgs:
    """ctypes arrays describing a batch (kept alive as long as the plan)."""

    def __init__(self, dicts, Ys, lambdas, Xs):
        n = len(dicts)
        if not (len(Ys) == len(lambdas) == len(Xs) == n):
            raise ValueError("batch: dicts, Ys, lambdas and Xs must have one entry per instance")
        for i in range(n):
            nrhs = int(Ys[i].shape[0]) if len(Ys[i].shape) == 2 else 1
            d = dicts[i]
            if getattr(d, "N", None) is not None:
                _check_buffer(Ys[i], d.N * nrhs, d.esize, f"Ys[{i}]", "batch")
                _check_buffer(Xs[i], d.K * nrhs, d.esize, f"Xs[{i}]", "batch")
            if np.size(lambdas[i]) < nrhs:
                raise ValueError(f"batch: lambdas[{i}] has {np.size(lambdas[i])} values, {nrhs} needed")
        self.n = n
        self.dicts = (ctypes.c_void_p * n)(*[d.value for d in dicts])
        self.Y = (ctypes.c_void_p * n)(*[_ptr(y)[0] for y in Ys])
        self.nrhs = (ctypes.c_int * n)(*[int(y.shape[0]) if len(y.shape) == 2 else 1 for y in Ys])
        self.lam_arrays = [np.ascontiguousarray(l, dtype=np.float64) for l in lambdas]
        self.lam = (ctypes.c_void_p * n)(*[a.ctypes.data for a in self.lam_arrays])
        self.X = (ctypes.c_void_p * n)(*[_ptr(x)[0] for x in Xs])
        self.total = sum(self.nrhs)


class ds_batch_handle:
    def __init__(self, h, args, opt):
        self.h, self.args, self.opt = h, args, opt


def ds_batch_create(ctx, dicts, Ys, lambdas, opt, Xs):
    """Ys[i]: device (n_rhs_i, N_i) tensor (row r = right-hand side r); Xs[i]: (n_rhs_i, K_i)."""
    a = _BatchArgs(dicts, Ys, lambdas, Xs)
    h = ctypes.c_void_p()
    _check(lib().ds_batch_create(ctx, a.n, a.dicts, a.Y, a.nrhs, a.lam, ctypes.byref(opt), a.X, ctypes.byref(h)),
           "ds_batch_create")
    return ds_batch_handle(h, a, opt)


def ds_batch_run(batch):
    res = (ds_result * batch.args.total)()
    _check(lib().ds_batch_run(batch.h, res), "ds_batch_run")
    return [r.as_dict() for r in res]


def ds_batch_info(batch):
    g, t, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().ds_batch_info(batch.h, ctypes.byref(g), ctypes.byref(t), ctypes.byref(s)), "ds_batch_info")
    return {"uses_graph": bool(g.value), "teams": t.value, "team_size": s.value}


def ds_batch_layout(batch):
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().ds_batch_layout(batch.h, *[ctypes.byref(x) for x in v]), "ds_batch_layout")
    return {"multi_rhs_blocks": v[0].value, "multi_rhs_teams": v[1].value, "multi_rhs_team_size": v[2].value,
            "single_problems": v[3].value}


def ds_batch_autotune(batch, max_candidates=8):
    ms = (ctypes.c_float * max_candidates)()
    c, n = ctypes.c_int(), ctypes.c_int()
    _check(lib().ds_batch_autotune(batch.h, max_candidates, ctypes.byref(c), ctypes.byref(n), ms), "ds_batch_autotune")
    return {"chosen": c.value, "ms": [ms[k] for k in range(n.value)], "schedule": ds_batch_schedule(batch)}


def ds_batch_schedule(batch):
    v = [ctypes.c_int() for _ in range(3)]
    sw = ctypes.c_double()
    _check(lib().ds_batch_schedule(batch.h, *[ctypes.byref(x) for x in v], ctypes.byref(sw)), "ds_batch_schedule")
    return {"tensor_bulk": v[0].value, "block_rhs": v[1].value, "sort_lambda": v[2].value, "lowp_switch": sw.value}


def ds_batch_destroy(batch):
    _check(lib().ds_batch_destroy(batch.h), "ds_batch_destroy")


def ds_solve_batch(ctx, dicts, Ys, lambdas, opt, Xs):
    a = _BatchArgs(dicts, Ys, lambdas, Xs)
    res = (ds_result * a.total)()
    _check(lib().ds_solve_batch(ctx, a.n, a.dicts, a.Y, a.nrhs, a.lam, ctypes.byref(opt), a.X, res),
           "ds_solve_batch")
    return [r.as_dict() for r in res]


def ds_server_create(ctx, hbm_budget_bytes, max_N, max_K, team_size=0):
    h = ctypes.c_void_p()
    _check(lib().ds_server_create(ctx, int(hbm_budget_bytes), int(max_N), int(max_K), int(team_size),
                                  ctypes.byref(h)), "ds_server_create")
    return h


def ds_server_submit(server, dct, y, lam, opt, x_out):
    """y, x_out: host float32 NumPy arrays; keep x_out alive until ds_server_poll returns a result."""
    _check_vectors(dct, "ds_server_submit", y=y, x_out=x_out)
    t = ctypes.c_uint64()
    _check(lib().ds_server_submit(server, dct, _ptr(y)[0], float(lam), ctypes.byref(opt), _ptr(x_out)[0],
                                  ctypes.byref(t)), "ds_server_submit")
    return t.value


def ds_server_poll(server, ticket):
    """The result dict when the request has completed, None while it is pending."""
    r = ds_result()
    st = lib().ds_server_poll(server, ctypes.c_uint64(ticket), ctypes.byref(r))
    if st == DS_PENDING:
        return None
    _check(st, "ds_server_poll")
    return r.as_dict()


def ds_server_stats(server):
    v = [ctypes.c_int64() for _ in range(4)]
    m = ctypes.c_size_t()
    _check(lib().ds_server_stats(server, *[ctypes.byref(x) for x in v], ctypes.byref(m)), "ds_server_stats")
    return {"completed": v[0].value, "in_flight": v[1].value, "pending": v[2].value, "launches": v[3].value,
            "pool_in_use": m.value}


def ds_server_destroy(server):
    _check(lib().ds_server_destroy(server), "ds_server_destroy")


def ds_solve_lasso_noalloc(device, stream, D, y, lam, opt, x_out):
    """Allocation-free Lasso solve on caller-owned device buffers (opt.L > 0 required)."""
    N, K, ld = _dict_layout(D)
    if _dtype_code(D) != DS_FP32:
        raise TypeError("ds_solve_lasso_noalloc: D must be float32")
    _check_buffer(y, N, 4, "y", "ds_solve_lasso_noalloc")
    _check_buffer(x_out, K, 4, "x_out", "ds_solve_lasso_noalloc")
    r = ds_result()
    s = None if stream is None else getattr(stream, "cuda_stream", stream)
    st = lib().ds_solve_lasso_noalloc(int(device), s, _ptr(D)[0], N, K, ld, _ptr(y)[0], float(lam),
                                      ctypes.byref(opt), _ptr(x_out)[0], ctypes.byref(r))
    _check(st, "ds_solve_lasso_noalloc")
    return r.as_dict()


def ds_selftest_wait_timeout(device: int = 0):
    """Run the bounded-wait self-test: returns (status, waited_ms); status is DS_ERR_TIMEOUT when the
    barrier wait that can never complete gave up as designed."""
    st_out = ctypes.c_int(-1)
    ms = ctypes.c_double(0.0)
    _check(lib().ds_selftest_wait_timeout(int(device), ctypes.byref(st_out), ctypes.byref(ms)),
           "ds_selftest_wait_timeout")
    return st_out.value, ms.value


def ds_set_history(ctx, hist=None):
    if hist is None:
        _check(lib().ds_set_history(ctx, None, 0), "ds_set_history")
    else:
        # the library writes max_rows x 6 doubles, row t-1 = iteration t
        if len(hist.shape) != 2 or hist.shape[1] != len(HIST_COLS):
            raise ValueError(f"ds_set_history: hist must have shape (rows, {len(HIST_COLS)})")
        _check_buffer(hist, hist.shape[0] * len(HIST_COLS), 8, "hist", "ds_set_history")
        _check(lib().ds_set_history(ctx, _ptr(hist)[0], int(hist.shape[0])), "ds_set_history")


def ds_set_screen_log(ctx, scr_iter=None):
    """Record per-atom screening iterations of the following solves into scr_iter, an int32
    device tensor of shape (rows, K) (row j = lambda j of a path), or stop recording (None)."""
    if scr_iter is None:
        _check(lib().ds_set_screen_log(ctx, None, 0), "ds_set_screen_log")
        return
    if str(scr_iter.dtype) not in ("torch.int32", "int32"):
        raise TypeError("ds_set_screen_log: scr_iter must hold int32 values")
    _check_buffer(scr_iter, 1, 4, "scr_iter", "ds_set_screen_log")
    n = scr_iter.numel() if hasattr(scr_iter, "numel") else scr_iter.size
    _check(lib().ds_set_screen_log(ctx, _ptr(scr_iter)[0], int(n)), "ds_set_screen_log")
