"""Adaptive steps on the GPU against the FP64 oracle: ISTA / FISTA with backtracking,
SpaRSA (Barzilai-Borwein step with its acceptance test) and TwIST (two-step shrinkage
with its monotone safeguard), the Table 1 rows whose step constant changes from one
iteration to the next.  A rejected step is redone inside the persistent kernel.

FP64 dictionaries: after the same number of iterations the GPU's iterate and screening
log are the oracle's.  FP32: the oracle's minimiser within the parity tolerance
(||x - x*||_inf <= 1e-5 ||x*||_inf), the gap tolerance met, no screened atom active.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import gen
import oracle
import paper_1412_4080_gb300 as ds

pytestmark = pytest.mark.gpu

RULES = [("sparsa", False), ("twist", False), ("ista", True), ("fista", True)]


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    c = ds.ds_create(0, None)
    yield c
    ds.ds_destroy(c)


def _f32(a):
    return a.astype(np.float32).astype(np.float64)


def _dev_dict(D, dtype):
    return torch.from_numpy(np.ascontiguousarray(D.T)).to("cuda", dtype).t()


def _solve(ctx, dct, y, lam, dtype, K, log=False, **opt):
    o = ds.ds_options_default(**opt)
    yt = torch.from_numpy(y).to("cuda", dtype)
    x = torch.empty(K, device="cuda", dtype=dtype)
    lg = torch.zeros((1, K), device="cuda", dtype=torch.int32)
    if log:
        ds.ds_set_screen_log(ctx, lg)
    try:
        r = ds.ds_solve(ctx, dct, yt, lam, o, x)
        torch.cuda.synchronize()
    finally:
        if log:
            ds.ds_set_screen_log(ctx, None)
    return x.double().cpu().numpy(), r, lg.cpu().numpy()[0]


@pytest.mark.parametrize("alg,bt", RULES)
@pytest.mark.parametrize("test", ["dst3", "dome"])
def test_fp64_adaptive_steps_follow_the_oracle(ctx, alg, bt, test):
    """100 x 500 FP64 (the small workload): the same iterate and the same screening log as
    the oracle after T iterations, T the oracle's count to gap 1e-10."""
    D, y, _ = gen.config1(1001)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    T = oracle.solve(D, y, lam, alg=alg, backtracking=bt, test=test, tol=1e-10, max_iter=100000, L=L)["iters"]
    ref = oracle.solve(D, y, lam, alg=alg, backtracking=bt, test=test, tol=0, max_iter=T, L=L)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float64))
    try:
        x, r, log = _solve(ctx, dct, y, lam, torch.float64, 500, log=True, alg=alg, step_backtracking=int(bt),
                           test=test, tol_gap_rel=0.0, max_iter=T, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    assert r["iters"] == T
    np.testing.assert_allclose(x, ref["x"], atol=1e-9 * np.abs(ref["x"]).max())
    np.testing.assert_array_equal(log, ref["scr_iter"])


@pytest.mark.parametrize("alg,bt", RULES)
def test_fp64_adaptive_steps_on_pnoise_follow_the_oracle(ctx, alg, bt):
    """An ill-conditioned Pnoise dictionary (Sec. 4.2), where SpaRSA rejects and redoes
    steps and TwIST falls back to the shrinkage step: same iterate and screening log."""
    D, y, _ = gen.lasso_problem(120, 600, seed=2101, p=0.02, kind="pnoise")
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    T = 150
    ref = oracle.solve(D, y, lam, alg=alg, backtracking=bt, test="dst3", tol=0, max_iter=T, L=L)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float64))
    try:
        x, r, log = _solve(ctx, dct, y, lam, torch.float64, 600, log=True, alg=alg, step_backtracking=int(bt),
                           test="dst3", tol_gap_rel=0.0, max_iter=T, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    assert r["iters"] == T
    np.testing.assert_allclose(x, ref["x"], atol=1e-8 * np.abs(ref["x"]).max())
    np.testing.assert_array_equal(log, ref["scr_iter"])


@pytest.mark.parametrize("alg,bt", RULES)
@pytest.mark.parametrize("kind,ratio", [("gaussian", 0.3), ("pnoise", 0.5)])
def test_fp32_adaptive_steps_reach_the_minimiser(ctx, alg, bt, kind, ratio):
    D, y, _ = gen.lasso_problem(1100, 3000, seed=2102, p=0.02, kind=kind)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = ratio * lm
    x_star = oracle.solve(D, y, lam, alg="sparsa", test="dst3", tol=1e-13, max_iter=200000)["x"]
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        x, r, log = _solve(ctx, dct, y, lam, torch.float32, 3000, log=True, alg=alg, step_backtracking=int(bt),
                           test="dst3", tol_gap_rel=0.0, max_iter=4000)
        xg, rg, _ = _solve(ctx, dct, y, lam, torch.float32, 3000, alg=alg, step_backtracking=int(bt),
                           test="dst3", tol_gap_rel=1e-6, max_iter=200000)
    finally:
        ds.ds_dict_destroy(dct)
    scale = np.abs(x_star).max()
    assert np.abs(x - x_star).max() <= 1e-5 * scale, np.abs(x - x_star).max() / scale
    assert np.all(np.abs(x_star[log != 0]) <= 1e-9 * scale)
    assert rg["status"] == 0 and rg["gap"] <= 1e-6 * 0.5 * float(y @ y)


@pytest.mark.parametrize("alg", ["sparsa", "twist"])
def test_fp32_adaptive_group_lasso(ctx, alg):
    D, y, _, goff, w = gen.config3(2103, N=600, K=1800, gsize=5, n_active=6)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.5 * lm
    x_star = oracle.solve(D, y, lam, goff, w, alg="sparsa", test="dgst3", tol=1e-13, max_iter=200000)["x"]
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32), goff, w)
    try:
        x, r, log = _solve(ctx, dct, y, lam, torch.float32, 1800, log=True, alg=alg, test="dgst3",
                           tol_gap_rel=0.0, max_iter=3000)
    finally:
        ds.ds_dict_destroy(dct)
    scale = np.abs(x_star).max()
    assert np.abs(x - x_star).max() <= 1e-5 * scale
    assert np.all(np.abs(x_star[log != 0]) <= 1e-9 * scale)


def test_gap_every_and_batched_sparsa(ctx):
    """gap_every: the solve stops on a multiple of it; SpaRSA problems in a batch (teams of
    CTAs) reach the same solutions as ds_solve."""
    D, y, _ = gen.lasso_problem(500, 2000, seed=2104, p=0.02)
    D, y = _f32(D), _f32(y)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        _, a, _ = _solve(ctx, dct, y, 0.3, torch.float32, 2000, test="dst3", tol_gap_rel=1e-6, max_iter=100000,
                         lambda_rel=1)
        _, b, _ = _solve(ctx, dct, y, 0.3, torch.float32, 2000, test="dst3", tol_gap_rel=1e-6, max_iter=100000,
                         lambda_rel=1, gap_every=10)
        # the same iterates, the rule evaluated at multiples of 10 only (FISTA's gap is not monotone, so the
        # first multiple of 10 past a's stop need not meet the tolerance)
        assert b["iters"] % 10 == 0 and b["iters"] >= a["iters"] and b["status"] == 0
        assert b["gap"] <= 1e-6 * 0.5 * float(y @ y)
        g = gen.rng(2105)
        Y = np.stack([y] + [gen.observe(D, gen.bernoulli_gaussian_x0(2000, 0.02, g), g) for _ in range(3)])
        Yt = torch.from_numpy(Y.astype(np.float32)).cuda()
        X = torch.zeros((4, 2000), device="cuda")
        lams = np.array([0.3, 0.5, 0.7, 0.4])
        opt = ds.ds_options_default(alg="sparsa", test="dst3", tol_gap_rel=1e-7, max_iter=100000, lambda_rel=1)
        res = ds.ds_solve_batch(ctx, [dct], [Yt], [lams], opt, [X])
        for r_ in range(4):
            xs, rs, _ = _solve(ctx, dct, Y[r_].astype(np.float64), lams[r_], torch.float32, 2000, alg="sparsa",
                               test="dst3", tol_gap_rel=1e-7, max_iter=100000, lambda_rel=1)
            assert res[r_]["status"] == 0
            xb = X[r_].double().cpu().numpy()
            assert np.abs(xb - xs).max() <= 1e-4 * np.abs(xs).max()
    finally:
        ds.ds_dict_destroy(dct)
