"""FP64 CPU oracle for dynamic screening (arXiv 1412.4080).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by ``bench.py``'s CPU-baseline leg and reference arm (``--impl reference``).
The product path (the CUDA library under ``paper_1412_4080_gb300/`` and its
binding) never imports it.

The arithmetic lives in ``dscreen_oracle.c`` (plain C loops, double
precision, single thread); this module compiles it with gcc on first use and
marshals NumPy arrays to it with ctypes.  Nothing here computes any step of
the method.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dscreen_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALGS = {"ista": 0, "fista": 1, "cp": 2, "sparsa": 3, "twist": 4}
TESTS = {"none": 0, "safe": 1, "dst3": 2, "dome": 3, "gsafe": 4, "dgst3": 5}
HIST_COLS = ("active", "nnz", "R", "radius", "gap", "mu")


class _Options(ctypes.Structure):
    _fields_ = [("alg", ctypes.c_int), ("test", ctypes.c_int), ("dynamic", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("tol_gap_rel", ctypes.c_double), ("L", ctypes.c_double),
                ("cp_tau", ctypes.c_double), ("cp_sigma", ctypes.c_double), ("cp_gamma", ctypes.c_double),
                ("step_backtracking", ctypes.c_int), ("bt_L0", ctypes.c_double), ("twist_xi1", ctypes.c_double),
                ("gap_every", ctypes.c_int)]


class _Result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("n_active", ctypes.c_int), ("nnz", ctypes.c_int),
                ("status", ctypes.c_int), ("gap", ctypes.c_double), ("primal", ctypes.c_double),
                ("dual", ctypes.c_double), ("lambda_max", ctypes.c_double), ("L", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (portable flags: x86 and Arm).  -O3 in ISO C mode keeps
    floating-point contraction off, so its results are those of -O2 bit for bit (only faster); no
    -march=native, since the same build must run on the x86 host and the Arm GPU machine."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O3", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i64 = ctypes.c_int64
        lib.or_lambda_max.argtypes = [dp, i64, i64, i64, dp, i64p, dp, i64, dp, i64p, dp]
        lib.or_lambda_max.restype = ctypes.c_int
        lib.or_spectral_norm_sq.argtypes = [dp, i64, i64, i64, ctypes.c_double, ctypes.c_int]
        lib.or_spectral_norm_sq.restype = ctypes.c_double
        lib.or_group_spec_norm.argtypes = [dp, i64, i64, i64, i64]
        lib.or_group_spec_norm.restype = ctypes.c_double
        lib.or_dual_scaling.argtypes = [dp, dp, i64, ctypes.c_double, ctypes.c_double]
        lib.or_dual_scaling.restype = ctypes.c_double
        lib.or_dome_max.argtypes = [ctypes.c_double] * 4
        lib.or_dome_max.restype = ctypes.c_double
        lib.or_solve.argtypes = [dp, i64, i64, i64, dp, ctypes.c_double, i64p, dp, i64,
                                 ctypes.POINTER(_Options), dp, dp, ctypes.POINTER(ctypes.c_int), dp, dp,
                                 ctypes.POINTER(_Result)]
        lib.or_solve.restype = ctypes.c_int
        lib.or_solve_log.argtypes = [dp, i64, i64, i64, dp, ctypes.c_double, i64p, dp, i64,
                                     ctypes.POINTER(_Options), dp, dp, ctypes.POINTER(ctypes.c_int), dp, dp, dp,
                                     ctypes.c_int, ctypes.POINTER(_Result)]
        lib.or_solve_log.restype = ctypes.c_int
        lib.or_sequential_screen.argtypes = [dp, i64, i64, i64, dp, ctypes.c_double, i64p, dp, i64, ctypes.c_int,
                                             dp, ctypes.POINTER(ctypes.c_int), dp, dp, dp, dp]
        lib.or_sequential_screen.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dict(D):
    D = np.asfortranarray(np.asarray(D, dtype=np.float64))
    N, K = D.shape
    return D, N, K, N


def _groups(groups, weights):
    if groups is None:
        return None, None, 0
    goff = np.ascontiguousarray(np.asarray(groups, dtype=np.int64))
    nG = goff.size - 1
    w = np.ones(nG) if weights is None else np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    return goff, w, nG


def lambda_max(D, y, groups=None, weights=None):
    """Return (lambda_*, index of the maximising atom / group, D^T y)."""
    lib = _load()
    D, N, K, ld = _dict(D)
    y = np.ascontiguousarray(y, dtype=np.float64)
    goff, w, nG = _groups(groups, weights)
    b = np.zeros(K)
    lm = ctypes.c_double()
    star = ctypes.c_int64()
    rc = lib.or_lambda_max(_dptr(D), N, K, ld, _dptr(y),
                           None if goff is None else goff.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           _dptr(w), nG, ctypes.byref(lm), ctypes.byref(star), _dptr(b))
    if rc != 0:
        raise ValueError("oracle lambda_max rejected its input")
    return lm.value, star.value, b


def spectral_norm_sq(D, tol=1e-12, max_iter=100000):
    lib = _load()
    D, N, K, ld = _dict(D)
    return lib.or_spectral_norm_sq(_dptr(D), N, K, ld, tol, max_iter)


def group_spec_norm(D, c0, c1):
    lib = _load()
    D, N, K, ld = _dict(D)
    return lib.or_group_spec_norm(_dptr(D), N, ld, int(c0), int(c1))


def dual_scaling(theta, y, lam, m):
    lib = _load()
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return lib.or_dual_scaling(_dptr(theta), _dptr(y), theta.size, float(lam), float(m))


def dome_max(dc0, t, psi, R):
    return _load().or_dome_max(float(dc0), float(t), float(psi), float(R))


def solve(D, y, lam, groups=None, weights=None, alg="fista", test="dst3", dynamic=True,
          tol=1e-6, max_iter=1000, L=None, x0=None, cp_tau=0.0, cp_sigma=0.0, cp_gamma=0.0, margins=0,
          backtracking=False, bt_L0=0.0, twist_xi1=0.0, gap_every=1):
    """Solve eq. (1) with Algorithm 3 and the ISTA, FISTA, Chambolle-Pock ("cp"), SpaRSA or TwIST
    update of Table 1 (ISTA / FISTA with backtracking of L when backtracking=True).
    Returns a dict with x, scr_iter, hist, theta (theta_t of the last iteration) and scalars; with
    margins=T > 0 also "margins": (min(iters, T) + 1) x G test margins, row 0 the static test, row t
    the test of iteration t (NaN where a group was not tested)."""
    lib = _load()
    D, N, K, ld = _dict(D)
    y = np.ascontiguousarray(y, dtype=np.float64)
    goff, w, nG = _groups(groups, weights)
    opt = _Options(ALGS[alg], TESTS[test], 1 if dynamic else 0, int(max_iter), float(tol),
                   float(L) if L is not None else 0.0, float(cp_tau), float(cp_sigma), float(cp_gamma),
                   1 if backtracking else 0, float(bt_L0), float(twist_xi1), int(gap_every))
    x = np.zeros(K)
    scr = np.zeros(K, dtype=np.int32)
    hist = np.zeros((max(int(max_iter), 1), len(HIST_COLS)))
    theta = np.zeros(N)
    res = _Result()
    x0a = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    G = K if goff is None else nG
    rows = int(margins) + 1 if margins else 0
    mlog = np.empty((rows, G)) if margins else None
    rc = lib.or_solve_log(_dptr(D), N, K, ld, _dptr(y), float(lam),
                          None if goff is None else goff.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                          _dptr(w), nG, ctypes.byref(opt), _dptr(x0a), _dptr(x),
                          scr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(hist), _dptr(theta),
                          _dptr(mlog), rows, ctypes.byref(res))
    if rc != 0:
        raise ValueError("oracle solve rejected its input")
    it = res.iters
    out = {"x": x, "scr_iter": scr, "hist": hist[:it], "theta": theta, "iters": it, "gap": res.gap,
           "primal": res.primal, "dual": res.dual, "lambda_max": res.lambda_max, "L": res.L,
           "n_active": res.n_active, "nnz": res.nnz, "status": res.status}
    if margins:
        out["margins"] = mlog[: min(it, rows - 1) + 1]
    return out


def sequential_screen(D, y, lam, theta, groups=None, weights=None, test="safe"):
    """The safe test at lambda from the dual point theta scaled over the whole dictionary
    (Lemma 8), e.g. theta = D x_k - y of a solution at a previous lambda_k.
    Returns a dict: screened (K bools), margins (G), R, radius, mu."""
    lib = _load()
    D, N, K, ld = _dict(D)
    y = np.ascontiguousarray(y, dtype=np.float64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    goff, w, nG = _groups(groups, weights)
    G = K if goff is None else nG
    scr = np.zeros(K, dtype=np.int32)
    marg = np.empty(G)
    R, rad, mu = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    rc = lib.or_sequential_screen(_dptr(D), N, K, ld, _dptr(y), float(lam),
                                  None if goff is None else goff.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  _dptr(w), nG, TESTS[test], _dptr(th),
                                  scr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(marg),
                                  ctypes.byref(R), ctypes.byref(rad), ctypes.byref(mu))
    if rc != 0:
        raise ValueError("oracle sequential_screen rejected its input")
    return {"screened": scr.astype(bool), "margins": marg, "R": R.value, "radius": rad.value, "mu": mu.value}
