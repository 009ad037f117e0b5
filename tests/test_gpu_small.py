"""The one-cluster solve of small FP64 Lasso problems (ISTA / FISTA at a fixed step, one
lambda, no history): the path ds_solve takes by default for them.  Against the FP64
oracle after the same number of iterations: the iteration that screened each atom
(static: -1) is the oracle's, atom for atom, and x is the oracle's within 1e-9 of its
largest entry.  With the gap rule: the oracle's stopping iteration within one, the
tolerance met.  ds_options.team_size > 0 runs the same problems on the grid kernel.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import gen
import oracle
import paper_1412_4080_gb300 as ds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    c = ds.ds_create(0, None)
    yield c
    ds.ds_destroy(c)


def _dev_dict(D):
    return torch.from_numpy(np.ascontiguousarray(D.T)).to("cuda", torch.float64).t()


def _solve(ctx, dct, y, lam, K, x0=None, **opt):
    o = ds.ds_options_default(**opt)
    log = torch.full((1, K), 12345, device="cuda", dtype=torch.int32)
    ds.ds_set_screen_log(ctx, log)
    try:
        x = torch.empty(K, device="cuda", dtype=torch.float64)
        x0t = None if x0 is None else torch.from_numpy(x0).cuda()
        r = ds.ds_solve(ctx, dct, torch.from_numpy(y).cuda(), lam, o, x, x0=x0t)
        torch.cuda.synchronize()
    finally:
        ds.ds_set_screen_log(ctx, None)
    return x.cpu().numpy(), r, log.cpu().numpy()[0]


CASES = [(alg, test, dyn) for alg in ("ista", "fista") for test in ("none", "safe", "dst3", "dome")
         for dyn in (True, False) if not (test == "none" and not dyn)]


@pytest.mark.parametrize("alg,test,dynamic", CASES)
def test_small_path_follows_the_oracle(ctx, alg, test, dynamic):
    """100 x 500 (the small workload, four CTAs of 125 atoms): screening log and x."""
    D, y, _ = gen.config1(1001)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    T = oracle.solve(D, y, lam, alg=alg, test=test, dynamic=dynamic, tol=1e-8, max_iter=100000, L=L)["iters"]
    ref = oracle.solve(D, y, lam, alg=alg, test=test, dynamic=dynamic, tol=0, max_iter=T, L=L)
    dct = ds.ds_dict_create(ctx, _dev_dict(D))
    try:
        x, r, log = _solve(ctx, dct, y, lam, 500, alg=alg, test=test, dynamic=int(dynamic), tol_gap_rel=0.0,
                           max_iter=T, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    assert r["status"] == 0 and r["iters"] == T
    np.testing.assert_array_equal(log, ref["scr_iter"])
    np.testing.assert_allclose(x, ref["x"], atol=1e-9 * np.abs(ref["x"]).max())
    assert abs(r["lambda_max"] - lm) <= 1e-12 * lm
    assert r["nnz"] == int((ref["x"] != 0).sum())


@pytest.mark.parametrize("N,K,seed", [(17, 33, 1301), (60, 97, 1302), (256, 300, 1303), (40, 2000, 1304),
                                      (100, 513, 1305)])
def test_small_path_shapes(ctx, N, K, seed):
    """Cluster sizes 2 to 8, N up to 256, ragged slices."""
    g = gen.rng(seed)
    D = gen.gaussian_dict(N, K, g)
    y = gen.observe(D, gen.sparse_x0(K, max(2, K // 50), g), g, sigma=0.01)
    lm, _, _ = oracle.lambda_max(D, y)
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    dct = ds.ds_dict_create(ctx, _dev_dict(D))
    try:
        for test, alg in (("dst3", "fista"), ("dome", "ista"), ("safe", "fista")):
            ref = oracle.solve(D, y, 0.4 * lm, alg=alg, test=test, tol=0, max_iter=300, L=L)
            x, r, log = _solve(ctx, dct, y, 0.4 * lm, K, alg=alg, test=test, tol_gap_rel=0.0, max_iter=300, L=L)
            assert r["iters"] == 300
            np.testing.assert_array_equal(log, ref["scr_iter"])
            np.testing.assert_allclose(x, ref["x"], atol=1e-9 * np.abs(ref["x"]).max())
    finally:
        ds.ds_dict_destroy(dct)


def test_small_path_gap_rule_start_point_and_lambda_max(ctx):
    D, y, _ = gen.config1(1001)
    lm, _, _ = oracle.lambda_max(D, y)
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    yy = float(y @ y)
    dct = ds.ds_dict_create(ctx, _dev_dict(D))
    try:
        # the gap rule: the oracle's stopping iteration (within one: the gap is summed in another order)
        ref = oracle.solve(D, y, 0.3 * lm, alg="fista", test="dst3", tol=1e-8, max_iter=100000, L=L)
        x, r, _ = _solve(ctx, dct, y, 0.3 * lm, 500, alg="fista", test="dst3", tol_gap_rel=1e-8, max_iter=100000, L=L)
        assert r["status"] == 0 and abs(r["iters"] - ref["iters"]) <= 1
        assert r["gap"] <= 1e-8 * 0.5 * yy and abs(r["primal"] - r["dual"] - r["gap"]) <= 1e-12 * yy
        # a starting point x0
        x0 = ref["x"] * 0.5
        ref0 = oracle.solve(D, y, 0.3 * lm, alg="ista", test="dst3", tol=0, max_iter=50, L=L, x0=x0)
        x, r, log = _solve(ctx, dct, y, 0.3 * lm, 500, x0=x0, alg="ista", test="dst3", tol_gap_rel=0.0,
                           max_iter=50, L=L)
        np.testing.assert_array_equal(log, ref0["scr_iter"])
        np.testing.assert_allclose(x, ref0["x"], atol=1e-9 * np.abs(ref0["x"]).max())
        # lambda >= lambda_*: x = 0 without iterations
        x, r, log = _solve(ctx, dct, y, 1.01 * lm, 500, test="dst3")
        assert r["iters"] == 0 and r["status"] == 0 and not x.any() and not log.any()
        # the iteration cap: not converged
        x, r, _ = _solve(ctx, dct, y, 0.1 * lm, 500, test="dst3", tol_gap_rel=1e-12, max_iter=5, L=L)
        assert r["iters"] == 5 and r["status"] == ds.DS_ERR_NOT_CONVERGED
    finally:
        ds.ds_dict_destroy(dct)


def test_small_path_equals_the_grid_kernel_and_is_faster(ctx):
    """The same solve on the grid kernel (team_size = 152): same screening log, x within the parity
    tolerance; the cluster path takes well under half its time."""
    D, y, _ = gen.config1(1001)
    lm, _, _ = oracle.lambda_max(D, y)
    dct = ds.ds_dict_create(ctx, _dev_dict(D))
    try:
        fixed = dict(alg="ista", test="dst3", tol_gap_rel=0.0, max_iter=150)
        xs, rs, ls = _solve(ctx, dct, y, 0.5 * lm, 500, **fixed)
        xg, rg, lg = _solve(ctx, dct, y, 0.5 * lm, 500, team_size=152, **fixed)
        assert rs["iters"] == rg["iters"] == 150
        np.testing.assert_array_equal(ls, lg)
        np.testing.assert_allclose(xs, xg, atol=1e-9 * np.abs(xg).max())
        assert rs["n_active"] == rg["n_active"] and rs["nnz"] == rg["nnz"]
        assert abs(rs["gap"] - rg["gap"]) <= 1e-9 * abs(rg["primal"])
        kw = dict(alg="ista", test="dst3", tol_gap_rel=1e-8, max_iter=100000)

        def median_ms(**extra):
            o = ds.ds_options_default(**kw, **extra)
            yt = torch.from_numpy(y).cuda()
            x = torch.empty(500, device="cuda", dtype=torch.float64)
            ts = []
            for _ in range(7):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ds.ds_solve(ctx, dct, yt, 0.5 * lm, o, x)
                ts.append(time.perf_counter() - t0)
            return float(np.median(ts[2:])) * 1e3

        assert median_ms() < 0.5 * median_ms(team_size=152)
    finally:
        ds.ds_dict_destroy(dct)
