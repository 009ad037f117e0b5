"""Screened sets atom by atom: the CUDA path (through the C ABI) against the FP64 oracle.

Definition 1 and Lemmas 2-7 fix which atoms a test may remove.  The library's
screening log (ds_set_screen_log) gives, per atom, the iteration whose test
screened it (-1: the static test of Algorithm 1, 0: never); the oracle returns
the same (scr_iter) and, per iteration, every tested atom's margin.

* FP64 dictionaries: the two logs are equal atom for atom, at the same fixed
  iteration count, for every test, static and dynamic.
* FP32 dictionaries: the kernel runs its tests in FP32 with the threshold
  rounded down and the radius rounded up, on an FP32 trajectory.  An atom may be
  screened at a different iteration (or not at all) only where the oracle's margin
  at the first iteration on which the two differ is within the error bound
      |rad_gpu,t - rad_oracle,t| + eps_t,
      eps_t = 1e-6 (1 + rad_t)  (sphere tests),  2e-6 (1 + rad_t)  (dome),
  the radii taken from both histories (the FP32 trajectory's drift and the rigorous
  bound on max |z| the kernel adds, asserted below 1e-3 relative) and eps_t covering
  the FP32 rounding of the threshold, the
  radius and, for the dome, its stored constants.  No atom screened by the GPU is
  nonzero in the oracle's solution.
"""
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


def _f32(a):
    return a.astype(np.float32).astype(np.float64)


def _dev_dict(D, dtype):
    return torch.from_numpy(np.ascontiguousarray(D.T)).to("cuda", dtype).t()


def _gpu_logged(ctx, dct, y, lams, dtype, K, rows=None, path=False, **opt):
    """Solve (or solve a path) with the history and the screening log recorded.
    Returns x (n_lambda x K), results, the history of the first lambda and the
    screening log (n_lambda x K)."""
    lams = np.atleast_1d(np.asarray(lams, dtype=np.float64))
    n = lams.size
    o = ds.ds_options_default(**opt)
    hist = torch.zeros((rows or o.max_iter + 2, 6), device="cuda", dtype=torch.float64)
    log = torch.full((n, K), 12345, device="cuda", dtype=torch.int32)
    ds.ds_set_history(ctx, hist)
    ds.ds_set_screen_log(ctx, log)
    try:
        yt = torch.from_numpy(y).to("cuda", dtype)
        X = torch.empty((n, K), device="cuda", dtype=dtype)
        if path:
            res = ds.ds_solve_path(ctx, dct, yt, lams, o, X)
        else:
            res = [ds.ds_solve(ctx, dct, yt, float(lams[0]), o, X[0])]
        torch.cuda.synchronize()
    finally:
        ds.ds_set_screen_log(ctx, None)
        ds.ds_set_history(ctx, None)
    return X.double().cpu().numpy(), res, hist.cpu().numpy(), log.cpu().numpy()


# ------------------------------------------------------------------ FP64: exact

FP64_CASES = [
    # (alg, test, dynamic)
    ("ista", "dst3", True), ("ista", "dst3", False), ("fista", "safe", True), ("fista", "dome", True),
    ("fista", "dome", False), ("fista", "safe", False), ("cp", "dst3", True),
]


@pytest.mark.parametrize("alg,test,dynamic", FP64_CASES)
def test_fp64_screened_sets_equal_the_oracle_atom_by_atom(ctx, alg, test, dynamic):
    """100 x 500 FP64 (the small workload): the iteration that screened each atom is the
    oracle's, atom for atom, after the same number of iterations."""
    D, y, _ = gen.config1(1001)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    T = oracle.solve(D, y, lam, alg=alg, test=test, dynamic=dynamic, tol=1e-8, max_iter=100000, L=L)["iters"]
    ref = oracle.solve(D, y, lam, alg=alg, test=test, dynamic=dynamic, tol=0, max_iter=T, L=L)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float64))
    try:
        X, res, _, log = _gpu_logged(ctx, dct, y, lam, torch.float64, 500, alg=alg, test=test,
                                     dynamic=int(dynamic), tol_gap_rel=0.0, max_iter=T, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    assert res[0]["iters"] == T
    np.testing.assert_array_equal(log[0], ref["scr_iter"])
    if dynamic and test != "safe":  # (at 0.5 lambda_* SAFE screens little or nothing on this problem)
        assert (ref["scr_iter"] != 0).sum() > 40
    np.testing.assert_allclose(X[0], ref["x"], atol=1e-9 * np.abs(ref["x"]).max())


@pytest.mark.parametrize("test", ["gsafe", "dgst3"])
@pytest.mark.parametrize("dynamic", [True, False])
def test_fp64_group_screened_sets_equal_the_oracle(ctx, test, dynamic):
    """FP64 Group-Lasso, groups of 5 with unequal weights: every atom's screening
    iteration is the oracle's."""
    g = gen.rng(1201)
    N, K = 120, 600
    D = gen.gaussian_dict(N, K, g)
    goff = gen.contiguous_groups(K, 5)
    w = g.uniform(1.5, 3.0, size=goff.size - 1)
    y = gen.observe(D, gen.group_x0(goff, 3, g), g)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.6 * lm
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    T = 400
    ref = oracle.solve(D, y, lam, goff, w, alg="fista", test=test, dynamic=dynamic, tol=0, max_iter=T, L=L)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float64), goff, w)
    try:
        X, res, _, log = _gpu_logged(ctx, dct, y, lam, torch.float64, K, test=test, dynamic=int(dynamic),
                                     tol_gap_rel=0.0, max_iter=T, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    np.testing.assert_array_equal(log[0], ref["scr_iter"])
    if dynamic:
        assert (ref["scr_iter"] != 0).sum() > 10
    np.testing.assert_allclose(X[0], ref["x"], atol=1e-9 * np.abs(ref["x"]).max())


def test_fp64_fewer_atoms_than_ctas(ctx):
    """K = 97 < 152 CTAs (most CTAs own an empty slice): same screening log and iterates."""
    g = gen.rng(1202)
    N, K = 60, 97
    D = gen.gaussian_dict(N, K, g)
    y = gen.observe(D, gen.sparse_x0(K, 4, g), g, sigma=0.01)
    lm, _, _ = oracle.lambda_max(D, y)
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float64))
    try:
        for test in ("safe", "dst3", "dome"):
            ref = oracle.solve(D, y, 0.4 * lm, test=test, tol=0, max_iter=600, L=L)
            X, _, _, log = _gpu_logged(ctx, dct, y, 0.4 * lm, torch.float64, K, test=test, tol_gap_rel=0.0,
                                       max_iter=600, L=L)
            np.testing.assert_array_equal(log[0], ref["scr_iter"])
            np.testing.assert_allclose(X[0], ref["x"], atol=1e-9 * np.abs(ref["x"]).max())
    finally:
        ds.ds_dict_destroy(dct)


# ------------------------------------------------- FP32: the margin rule

def _group_of_atom(K, goff):
    if goff is None:
        return np.arange(K)
    return np.repeat(np.arange(goff.size - 1), np.diff(goff))


def _check_margin_rule(log, hist, ref, x_star, test, goff=None):
    """Every atom screened at a different iteration by the GPU and the oracle has an oracle
    margin within the error bound at the first iteration where the two differ; the
    trajectories' radii agree to 1e-3; no GPU-screened atom is nonzero in the minimiser."""
    K = log.size
    s_o = ref["scr_iter"]
    M = ref["margins"]
    T = M.shape[0] - 1
    rad_o = ref["hist"][:T, 3]
    rad_g = hist[:T, 3]
    # the radii differ by the FP32 trajectory and by the rigorous bound on max |z| that the kernel adds
    # (its radius is never below the nominal one): a sanity limit, the bound below uses the difference
    assert np.all(np.abs(rad_g - rad_o) <= 1e-3 * rad_o + 1e-12), np.max(np.abs(rad_g - rad_o) / rad_o)
    eps_rel = 2e-6 if test == "dome" else 1e-6
    gid = _group_of_atom(K, goff)
    worst = 0.0
    for i in np.flatnonzero(log != s_o):
        t1 = min(v for v in (int(log[i]), int(s_o[i])) if v != 0)
        assert 1 <= t1 <= T, (i, log[i], s_o[i])
        m = M[t1, gid[i]]
        bound = abs(rad_g[t1 - 1] - rad_o[t1 - 1]) + eps_rel * (1.0 + rad_o[t1 - 1])
        assert not np.isnan(m) and abs(m) <= bound, (i, int(log[i]), int(s_o[i]), m, bound)
        worst = max(worst, abs(m) / bound)
    scale = np.abs(x_star).max()
    assert np.all(np.abs(x_star[log != 0]) <= 1e-9 * scale), "a screened atom is active in the minimiser"
    return int((log != s_o).sum()), worst


FP32_CASES = [
    # (N, K, ratio, test, seed)
    (1100, 3000, 0.5, "safe", 1301), (1100, 3000, 0.5, "dst3", 1301), (1100, 3000, 0.5, "dome", 1301),
    (1100, 3000, 0.8, "dst3", 1302), (1100, 3000, 0.3, "dome", 1303),
    (2000, 10000, 0.5, "safe", 1002), (2000, 10000, 0.5, "dst3", 1002), (2000, 10000, 0.7, "dome", 1002),
]


@pytest.mark.parametrize("N,K,ratio,test,seed", FP32_CASES)
def test_fp32_screened_sets_follow_the_margin_rule(ctx, N, K, ratio, test, seed):
    D, y, _ = gen.lasso_problem(N, K, seed=seed) if seed != 1002 else gen.config2(1002)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = ratio * lm
    L = oracle.spectral_norm_sq(D, tol=1e-10, max_iter=5000) * (1 + 1e-6)
    T = 1000 if K <= 3000 else 400
    ref = oracle.solve(D, y, lam, alg="fista", test=test, tol=0, max_iter=T, L=L, margins=T)
    # the minimiser (Theorem 1: the screened solve reaches it exactly), to 1e-12
    x_star = oracle.solve(D, y, lam, alg="fista", test=test, tol=1e-12, max_iter=200000, L=L)["x"]
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        X, res, hist, log = _gpu_logged(ctx, dct, y, lam, torch.float32, K, test=test, tol_gap_rel=0.0,
                                        max_iter=T, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    n_diff, worst = _check_margin_rule(log[0], hist, ref, x_star, test)
    assert (log[0] != 0).sum() >= 0.5 * (ref["scr_iter"] != 0).sum()
    assert n_diff <= 0.01 * K, n_diff
    # the iterates after T iterations: the oracle's within the parity tolerance
    assert np.abs(X[0] - ref["x"]).max() <= 1e-5 * np.abs(ref["x"]).max()


@pytest.mark.parametrize("gsize,test,ratio", [(10, "gsafe", 0.7), (10, "dgst3", 0.6), (5, "dgst3", 0.6),
                                              (5, "gsafe", 0.7)])
def test_fp32_group_screened_sets_follow_the_margin_rule(ctx, gsize, test, ratio):
    D, y, _, goff, w = gen.config3(1401, N=1100, K=3000, gsize=gsize, n_active=6)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = ratio * lm
    L = oracle.spectral_norm_sq(D, tol=1e-10, max_iter=5000) * (1 + 1e-6)
    T = 1000
    ref = oracle.solve(D, y, lam, goff, w, alg="fista", test=test, tol=0, max_iter=T, L=L, margins=T)
    x_star = oracle.solve(D, y, lam, goff, w, test=test, tol=1e-12, max_iter=200000, L=L)["x"]
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32), goff, w)
    try:
        X, res, hist, log = _gpu_logged(ctx, dct, y, lam, torch.float32, 3000, test=test, tol_gap_rel=0.0,
                                        max_iter=T, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    _check_margin_rule(log[0], hist, ref, x_star, test, goff)
    assert (log[0] != 0).sum() > 0
    assert np.abs(X[0] - ref["x"]).max() <= 1e-5 * np.abs(ref["x"]).max()


def test_fp32_full_size_group_workload_follows_the_margin_rule(ctx):
    """The 2000 x 10000 Group-Lasso workload (groups of 10, w_g = sqrt(10)), DGST3 at 0.5."""
    D, y, _, goff, w = gen.config3(1003)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.5 * lm
    L = oracle.spectral_norm_sq(D, tol=1e-10, max_iter=5000) * (1 + 1e-6)
    T = 300
    ref = oracle.solve(D, y, lam, goff, w, alg="fista", test="dgst3", tol=0, max_iter=T, L=L, margins=T)
    x_star = oracle.solve(D, y, lam, goff, w, test="dgst3", tol=1e-12, max_iter=100000, L=L)["x"]
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32), goff, w)
    try:
        X, res, hist, log = _gpu_logged(ctx, dct, y, lam, torch.float32, 10000, test="dgst3", tol_gap_rel=0.0,
                                        max_iter=T, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    _check_margin_rule(log[0], hist, ref, x_star, "dgst3", goff)
    assert np.abs(X[0] - ref["x"]).max() <= 1e-5 * np.abs(ref["x"]).max()


# ------------------------------------ fewer atoms than CTAs, group sizes, FP32

@pytest.mark.parametrize("K", [64, 151])
def test_fp32_fewer_atoms_than_ctas(ctx, K):
    """A Lasso dictionary with fewer atoms than the 152 CTAs of the grid (several CTAs own an
    empty slice): the oracle's iterates and the margin rule."""
    D, y, _ = gen.lasso_problem(300, K, seed=1500 + K, p=0.05)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.3 * lm
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    T = 2000
    ref = oracle.solve(D, y, lam, test="dst3", tol=0, max_iter=T, L=L, margins=T)
    x_star = oracle.solve(D, y, lam, test="dst3", tol=1e-13, max_iter=200000, L=L)["x"]
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        X, _, hist, log = _gpu_logged(ctx, dct, y, lam, torch.float32, K, test="dst3", tol_gap_rel=0.0,
                                      max_iter=T, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    _check_margin_rule(log[0], hist, ref, x_star, "dst3")
    assert np.abs(X[0] - ref["x"]).max() <= 1e-5 * np.abs(ref["x"]).max()


@pytest.mark.parametrize("test", ["gsafe", "dgst3"])
def test_paper_group_data_groups_of_five(ctx, test):
    """The paper's Group-Lasso data (Sec. 4.2, 4.4): Pnoise atoms, groups of 5, each group
    active with probability 0.05, unit-norm y at 20 dB: the GPU reaches the oracle's
    solution and its screening is safe."""
    D, y, _, goff, w = gen.paper_group_problem(5, seed=1601, N=500, K=2000)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.7 * lm
    L = oracle.spectral_norm_sq(D, tol=1e-12, max_iter=20000) * (1 + 1e-6)
    x_star = oracle.solve(D, y, lam, goff, w, test=test, tol=1e-13, max_iter=400000, L=L)["x"]
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32), goff, w)
    try:
        X, res, _, log = _gpu_logged(ctx, dct, y, lam, torch.float32, 2000, test=test, tol_gap_rel=0.0,
                                     max_iter=20000, L=L, rows=8)
    finally:
        ds.ds_dict_destroy(dct)
    scale = np.abs(x_star).max()
    assert np.abs(X[0] - x_star).max() <= 1e-5 * scale
    assert np.all(np.abs(x_star[log[0] != 0]) <= 1e-9 * scale) and (log[0] != 0).sum() > 0


# ------------------------------------ precision variant against the oracle

@pytest.mark.parametrize("prec", ["bf16", "fp8"])
@pytest.mark.parametrize("test,ratio", [("dst3", 0.6), ("dome", 0.7), ("safe", 0.8)])
def test_lowp_lasso_matches_the_oracle(ctx, prec, test, ratio):
    """BF16 / FP8 working copies: after the bulk phase on the copy and the FP32 polish, x is
    the FP64 oracle's minimiser within the parity tolerance, and no screened atom is
    active in it."""
    D, y, _ = gen.lasso_problem(1100, 3000, seed=1701, p=0.02)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = ratio * lm
    x_star = oracle.solve(D, y, lam, test=test, tol=1e-13, max_iter=200000)["x"]
    work = ds.DS_BF16 if prec == "bf16" else ds.DS_FP8
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32), work_prec=work)
    try:
        X, res, _, log = _gpu_logged(ctx, dct, y, lam, torch.float32, 3000, test=test, tol_gap_rel=0.0,
                                     max_iter=3000, rows=8)
    finally:
        ds.ds_dict_destroy(dct)
    assert 0 < res[0]["cols_lowp"] < res[0]["cols_corr"]
    scale = np.abs(x_star).max()
    assert np.abs(X[0] - x_star).max() <= 1e-5 * scale
    assert np.all(np.abs(x_star[log[0] != 0]) <= 1e-9 * scale) and (log[0] != 0).sum() > 0


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_lowp_group_lasso_matches_the_oracle(ctx, prec):
    D, y, _, goff, w = gen.config3(1702, N=600, K=1800, gsize=10, n_active=6)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.5 * lm
    x_star = oracle.solve(D, y, lam, goff, w, test="dgst3", tol=1e-13, max_iter=200000)["x"]
    work = ds.DS_BF16 if prec == "bf16" else ds.DS_FP8
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32), goff, w, work_prec=work)
    try:
        X, res, _, log = _gpu_logged(ctx, dct, y, lam, torch.float32, 1800, test="dgst3", tol_gap_rel=0.0,
                                     max_iter=2500, rows=8)
    finally:
        ds.ds_dict_destroy(dct)
    assert res[0]["cols_lowp"] > 0
    scale = np.abs(x_star).max()
    assert np.abs(X[0] - x_star).max() <= 1e-5 * scale
    assert np.all(np.abs(x_star[log[0] != 0]) <= 1e-9 * scale)


# ------------------------------------ regularization paths (warm starts)

def test_fp32_warm_started_path_matches_the_oracle_at_each_lambda(ctx):
    """A decreasing lambda path with warm starts: every lambda's x is the oracle's
    minimiser at that lambda within the parity tolerance, and no screened atom is active."""
    D, y, _ = gen.lasso_problem(1100, 3000, seed=1801, p=0.02)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y)
    ratios = np.array([0.9, 0.8, 0.7, 0.6])
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        X, res, _, log = _gpu_logged(ctx, dct, y, ratios, torch.float32, 3000, path=True, rows=8, test="dst3",
                                     tol_gap_rel=0.0, max_iter=2000, lambda_rel=1, warm_start=1)
    finally:
        ds.ds_dict_destroy(dct)
    for j, r in enumerate(ratios):
        x_star = oracle.solve(D, y, r * lm, test="dst3", tol=1e-13, max_iter=200000)["x"]
        scale = np.abs(x_star).max()
        assert np.abs(X[j] - x_star).max() <= 1e-5 * scale, (j, np.abs(X[j] - x_star).max() / scale)
        assert np.all(np.abs(x_star[log[j] != 0]) <= 1e-9 * scale)
        assert (log[j] != 0).sum() > 0


@pytest.mark.parametrize("test", ["safe", "dst3", "dome"])
def test_fp64_warm_path_first_test_is_the_sequential_test(ctx, test):
    """FP64, decreasing lambdas with warm starts: the atoms screened by the test of
    iteration 1 at lambda_j are exactly those of the oracle's sequential test (Sec. 5) from
    the GPU's solution at lambda_{j-1} (theta = D x_{j-1} - y, scaled over every atom), and
    each lambda's whole screening log is that of the oracle started from the same x."""
    D, y, _ = gen.config1(1001)
    lm, _, _ = oracle.lambda_max(D, y)
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    ratios = np.array([0.9, 0.85, 0.8, 0.75])  # the sequential test needs small steps of lambda
    T = 300
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float64))
    try:
        X, res, _, log = _gpu_logged(ctx, dct, y, ratios, torch.float64, 500, path=True, rows=8, test=test,
                                     tol_gap_rel=0.0, max_iter=T, L=L, lambda_rel=1, warm_start=1)
    finally:
        ds.ds_dict_destroy(dct)
    for j in range(1, ratios.size):
        lam = ratios[j] * lm
        seq = oracle.sequential_screen(D, y, lam, D @ X[j - 1] - y, test=test)
        first = log[j] == 1
        differ = first != seq["screened"]
        assert np.all(np.abs(seq["margins"][differ]) <= 1e-9), seq["margins"][differ]
        assert seq["screened"].sum() > 0
        ref = oracle.solve(D, y, lam, test=test, tol=0, max_iter=T, L=L, x0=X[j - 1])
        np.testing.assert_array_equal(log[j], ref["scr_iter"])
        np.testing.assert_allclose(X[j], ref["x"], atol=1e-9 * np.abs(ref["x"]).max())
