"""The allocation-free Lasso entry point against the regular one.

ds_solve_lasso_noalloc serves callers that cannot allocate device memory: a
framework whose caching allocator owns all device memory, a service with a
fixed memory budget committed up front, or a latency-critical loop that must
not pay for cudaMalloc/cudaFree.  Its scratch is one fixed device array shared
by every call, so two calls in a row (different problems) must each match
ds_solve, through the C ABI, within the parity tolerance of the GPU tests.

This file is collected last on purpose: a failure here leaves every other test
already run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import gen
import paper_1412_4080_gb300 as ds

pytestmark = pytest.mark.gpu


def _dev_dict(D):
    return torch.from_numpy(np.ascontiguousarray(D.T)).to("cuda", torch.float32).t()


def test_noalloc_matches_ds_solve_on_two_calls_in_a_row():
    N, K = 700, 3000
    D, y1, _ = gen.lasso_problem(N, K, seed=91, p=0.02)
    g = gen.rng(92)
    y2 = gen.observe(D, gen.bernoulli_gaussian_x0(K, 0.02, g), g)
    Dt = _dev_dict(D)
    ctx = ds.ds_create(0, None)
    dct = ds.ds_dict_create(ctx, Dt)
    try:
        L = ds.ds_dict_lipschitz(dct)
        for (y, ratio, test) in ((y1, 0.5, "dst3"), (y2, 0.8, "dome")):
            yt = torch.from_numpy(y).to("cuda", torch.float32)
            o = ds.ds_options_default(test=test, tol_gap_rel=1e-6, max_iter=20000, L=L, lambda_rel=1)
            x_ref = torch.empty(K, device="cuda")
            ref = ds.ds_solve(ctx, dct, yt, ratio, o, x_ref)
            x_na = torch.full((K,), float("nan"), device="cuda")
            got = ds.ds_solve_lasso_noalloc(0, None, Dt, yt, ratio, o, x_na)
            torch.cuda.synchronize()
            a = x_ref.double().cpu().numpy()
            b = x_na.double().cpu().numpy()
            assert got["status"] == 0 and ref["status"] == 0
            assert got["iters"] == ref["iters"]
            assert np.abs(b - a).max() <= 1e-5 * np.abs(a).max()
            assert abs(got["gap"] - ref["gap"]) <= 1e-9 * 0.5 * float(y @ y)
    finally:
        ds.ds_dict_destroy(dct)
        ds.ds_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    o = ds.ds_options_default(L=10.0)
    r = ds.ds_result()
    fake = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    st = ds.lib().ds_solve_lasso_noalloc(0, None, fake, 5000, 100, 5000, fake, 1.0, ctypes.byref(o), fake,
                                         ctypes.byref(r))
    assert st == ds.DS_ERR_UNSUPPORTED
    st = ds.lib().ds_solve_lasso_noalloc(0, None, fake, 100, 20000, 100, fake, 1.0, ctypes.byref(o), fake,
                                         ctypes.byref(r))
    assert st == ds.DS_ERR_UNSUPPORTED


def _compare_with_ds_solve(D, Dt_noalloc, y, ratio, test):
    """ds_solve on a registered copy of D against the allocation-free call on
    Dt_noalloc (the same atoms, possibly inside a taller column-major buffer)."""
    K = D.shape[1]
    ctx = ds.ds_create(0, None)
    dct = ds.ds_dict_create(ctx, _dev_dict(D))
    try:
        L = ds.ds_dict_lipschitz(dct)
        yt = torch.from_numpy(y).to("cuda", torch.float32)
        o = ds.ds_options_default(test=test, tol_gap_rel=1e-6, max_iter=20000, L=L, lambda_rel=1)
        x_ref = torch.empty(K, device="cuda")
        ref = ds.ds_solve(ctx, dct, yt, ratio, o, x_ref)
        x_na = torch.full((K,), float("nan"), device="cuda")
        got = ds.ds_solve_lasso_noalloc(0, None, Dt_noalloc, yt, ratio, o, x_na)
        torch.cuda.synchronize()
    finally:
        ds.ds_dict_destroy(dct)
        ds.ds_destroy(ctx)
    a = x_ref.double().cpu().numpy()
    b = x_na.double().cpu().numpy()
    assert got["status"] == 0 and ref["status"] == 0
    assert got["iters"] == ref["iters"]
    assert np.abs(b - a).max() <= 1e-5 * np.abs(a).max()
    assert abs(got["gap"] - ref["gap"]) <= 1e-9 * 0.5 * float(y @ y)


def test_noalloc_at_its_documented_size_limits():
    # N = 4096, K = 16384: the fixed scratch must hold the whole workspace on this GPU
    D, y, _ = gen.lasso_problem(4096, 16384, seed=93, p=0.01)
    _compare_with_ds_solve(D, _dev_dict(D), y, 0.5, "dst3")
    assert torch.cuda.current_device() == 0


def test_noalloc_row_slice_of_a_taller_matrix_with_nonzero_padding():
    # D is rows 0..N-1 of an ld x K column-major buffer whose rows N..ld-1 hold
    # nonzero finite values: they are not part of the atoms
    N, K, ld = 700, 2000, 1024
    D, y, _ = gen.lasso_problem(N, K, seed=94, p=0.02)
    tall = np.ascontiguousarray(np.vstack([D, gen.rng(95).standard_normal((ld - N, K))]).T)
    Tt = torch.from_numpy(tall).to("cuda", torch.float32).t()  # (ld, K), strides (1, ld)
    _compare_with_ds_solve(D, Tt[:N], y, 0.7, "safe")
