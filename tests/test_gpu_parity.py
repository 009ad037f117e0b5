"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Each case runs the oracle and the GPU on the same seeded input and the same
step constant L.  The bar for FP32:
||x - x_oracle||_inf <= 1e-5 ||x_oracle||_inf once both have converged, and
the GPU's own duality gap <= 1e-6 * 1/2 ||y||^2 when it stops on tolerance.
FP64 dictionaries are held to 1e-9.  Sizes span several GEMV row chunks
(512 rows) and synthesis tiles with ragged tails.
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
    """The FP32 problem the GPU solves, in FP64 for the oracle."""
    return a.astype(np.float32).astype(np.float64)


def _dev_dict(D, dtype):
    # column-major (N, K) device tensor: transpose of a contiguous (K, N)
    return torch.from_numpy(np.ascontiguousarray(D.T)).to("cuda", dtype).t()


def _solve_gpu(ctx, dct, y, lam, dtype, K, **opt):
    o = ds.ds_options_default(**opt)
    yt = torch.from_numpy(y).to("cuda", dtype)
    x = torch.empty(K, device="cuda", dtype=dtype)
    r = ds.ds_solve(ctx, dct, yt, lam, o, x)
    torch.cuda.synchronize()
    return x.double().cpu().numpy(), r


def _fp64_gap(D, y, x, lam, goff=None, w=None):
    """Exact (FP64) duality gap of x with the dual point built from its residual."""
    r = y - D @ x
    c = D.T @ r
    if goff is None:
        m = np.abs(c).max()
        om = np.abs(x).sum()
    else:
        m = max(np.linalg.norm(c[goff[i]:goff[i + 1]]) / w[i] for i in range(goff.size - 1))
        om = sum(w[i] * np.linalg.norm(x[goff[i]:goff[i + 1]]) for i in range(goff.size - 1))
    s = min(1.0 / lam, 1.0 / m) if m > 0 else 1.0 / lam
    v = s * r
    P = 0.5 * r @ r + lam * om
    Dv = 0.5 * y @ y - 0.5 * lam * lam * np.sum((v - y / lam) ** 2)
    return P - Dv


CASES = [
    # (N, K, ratio)
    (300, 1500, 0.5),
    (700, 2100, 0.2),
    (1100, 3000, 0.8),
]


@pytest.mark.parametrize("N,K,ratio", CASES)
@pytest.mark.parametrize("test", ["none", "safe", "dst3", "dome"])
def test_lasso_fp32_parity(ctx, N, K, ratio, test):
    D, y, _ = gen.lasso_problem(N, K, seed=N + K, p=0.02)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = ratio * lm
    L = oracle.spectral_norm_sq(D, tol=1e-10, max_iter=5000) * (1 + 1e-6)
    ref = oracle.solve(D, y, lam, alg="fista", test=test, tol=0, max_iter=3000, L=L)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        x, r = _solve_gpu(ctx, dct, y, lam, torch.float32, K, test=test, tol_gap_rel=0.0, max_iter=3000, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    assert r["status"] == 0 and r["iters"] == 3000
    scale = np.abs(ref["x"]).max()
    assert np.abs(x - ref["x"]).max() <= 1e-5 * scale, np.abs(x - ref["x"]).max() / scale
    # screening never removed an atom of the solution: its support is recovered
    assert np.all(x[np.abs(ref["x"]) > 1e-4 * scale] != 0)
    assert abs(r["lambda_max"] - lm) <= 1e-12 * lm


@pytest.mark.parametrize("test", ["safe", "dst3", "dome"])
@pytest.mark.parametrize("alg", ["ista", "fista"])
def test_lasso_fp32_stops_on_gap(ctx, test, alg):
    N, K = 513, 2049
    D, y, _ = gen.lasso_problem(N, K, seed=7, p=0.01)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        x, r = _solve_gpu(ctx, dct, y, lam, torch.float32, K, test=test, alg=alg, tol_gap_rel=1e-6,
                          max_iter=20000)
    finally:
        ds.ds_dict_destroy(dct)
    yy = y @ y
    assert r["status"] == 0 and r["gap"] <= 1e-6 * 0.5 * yy
    assert _fp64_gap(D, y, x, lam) <= 2e-6 * 0.5 * yy
    ref = oracle.solve(D, y, lam, alg=alg, test=test, tol=1e-14, max_iter=100000)
    # ||D (x - x~)|| <= sqrt(2 gap): checked on the FP64 residuals
    assert np.linalg.norm(D @ (x - ref["x"])) <= np.sqrt(2 * 2e-6 * 0.5 * yy) * 1.01


@pytest.mark.parametrize("dynamic", [True, False])
def test_config1_fp64_ista_dst3(ctx, dynamic):
    """100 x 500 FP64, ISTA + DST3, gap 1e-8: GPU and oracle take the same iterations."""
    D, y, _ = gen.config1(1001)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    ref = oracle.solve(D, y, lam, alg="ista", test="dst3", dynamic=dynamic, tol=1e-8, max_iter=100000, L=L)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float64))
    hist = torch.zeros((ref["iters"] + 10, 6), device="cuda", dtype=torch.float64)
    ds.ds_set_history(ctx, hist)
    try:
        x, r = _solve_gpu(ctx, dct, y, lam, torch.float64, 500, alg="ista", test="dst3", dynamic=int(dynamic),
                          tol_gap_rel=1e-8, max_iter=100000, L=L)
    finally:
        ds.ds_set_history(ctx, None)
        ds.ds_dict_destroy(dct)
    assert r["status"] == 0
    assert abs(r["iters"] - ref["iters"]) <= 1
    np.testing.assert_allclose(x, ref["x"], atol=1e-9 * np.abs(ref["x"]).max())
    h = hist.cpu().numpy()[: r["iters"]]
    n = min(r["iters"], ref["iters"])
    # same screening trajectory: active-set sizes agree iteration by iteration
    np.testing.assert_array_equal(h[:n, 0], ref["hist"][:n, 0])
    np.testing.assert_allclose(h[:n, 4], ref["hist"][:n, 4], rtol=1e-6, atol=1e-12 * (y @ y))


@pytest.mark.parametrize("test", ["none", "gsafe", "dgst3"])
@pytest.mark.parametrize("ratio", [0.3, 0.7])
def test_group_lasso_fp32_parity(ctx, test, ratio):
    N, K = 600, 1800
    D, y, _, goff, w = gen.config3(31, N=N, K=K, gsize=10, n_active=6)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = ratio * lm
    L = oracle.spectral_norm_sq(D, tol=1e-10, max_iter=5000) * (1 + 1e-6)
    ref = oracle.solve(D, y, lam, goff, w, alg="fista", test=test, tol=0, max_iter=2500, L=L)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32), goff, w)
    try:
        x, r = _solve_gpu(ctx, dct, y, lam, torch.float32, K, test=test, tol_gap_rel=0.0, max_iter=2500, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    scale = np.abs(ref["x"]).max()
    assert np.abs(x - ref["x"]).max() <= 1e-5 * scale
    assert abs(r["lambda_max"] - lm) <= 1e-12 * lm


@pytest.mark.parametrize("gsize", [50, 100])
@pytest.mark.parametrize("test", ["gsafe", "dgst3"])
def test_group_lasso_large_groups(ctx, test, gsize):
    """The paper's larger groups (Sec. 4.4 sweeps 5 to 100 atoms per group): ||D_g||_2 by
    the CTA-parallel Jacobi, and the solve, match the oracle."""
    N, K = 500, 2000
    D, y, _, goff, w = gen.config3(41, N=N, K=K, gsize=gsize, n_active=2)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.5 * lm
    L = oracle.spectral_norm_sq(D, tol=1e-10, max_iter=5000) * (1 + 1e-6)
    ref = oracle.solve(D, y, lam, goff, w, alg="fista", test=test, tol=0, max_iter=1500, L=L)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32), goff, w)
    try:
        x, r = _solve_gpu(ctx, dct, y, lam, torch.float32, K, test=test, tol_gap_rel=0.0, max_iter=1500, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    scale = np.abs(ref["x"]).max()
    assert np.abs(x - ref["x"]).max() <= 1e-5 * scale
    assert abs(r["lambda_max"] - lm) <= 1e-12 * lm


def test_group_lasso_ragged_groups(ctx):
    """Groups of unequal sizes (1 to 17 atoms) and weights."""
    g = gen.rng(41)
    N, K = 257, 900
    D = gen.gaussian_dict(N, K, g)
    sizes = []
    while sum(sizes) < K:
        sizes.append(int(min(g.integers(1, 18), K - sum(sizes))))
    goff = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    w = g.uniform(0.5, 2.0, size=len(sizes))
    x0 = gen.group_x0(goff, 4, g)
    y = gen.observe(D, x0, g)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.4 * lm
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    ref = oracle.solve(D, y, lam, goff, w, test="dgst3", tol=0, max_iter=3000, L=L)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32), goff, w)
    try:
        x, r = _solve_gpu(ctx, dct, y, lam, torch.float32, K, test="dgst3", tol_gap_rel=0.0, max_iter=3000, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    assert np.abs(x - ref["x"]).max() <= 1e-5 * np.abs(ref["x"]).max()


def test_lambda_max_and_trivial_case(ctx):
    D, y, _ = gen.lasso_problem(333, 999, seed=5)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        yt = torch.from_numpy(y).to("cuda", torch.float32)
        got = ds.ds_lambda_max(ctx, dct, yt)
        assert abs(got - lm) <= 1e-12 * lm
        x, r = _solve_gpu(ctx, dct, y, got * 1.0001, torch.float32, 999)
        assert r["iters"] == 0 and not x.any() and r["gap"] == 0.0
    finally:
        ds.ds_dict_destroy(dct)


def test_step_constant_upper_bound(ctx):
    for (N, K, seed) in ((100, 500, 1), (2000, 10000, 2), (257, 257, 3)):
        g = gen.rng(seed)
        D = gen.gaussian_dict(N, K, g)
        D = _f32(D)
        dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
        L = ds.ds_dict_lipschitz(dct)
        ds.ds_dict_destroy(dct)
        true = np.linalg.norm(D, 2) ** 2
        assert true <= L <= true * (1 + 1e-4), (N, K, L / true - 1)


def test_path_and_host_buffers_match_device_single_solves(ctx):
    N, K = 400, 1600
    D, y, _ = gen.lasso_problem(N, K, seed=11)
    ratios = np.array([0.9, 0.5, 0.2])
    dct = ds.ds_dict_create(ctx, np.asfortranarray(D.astype(np.float32)))  # host dictionary
    try:
        o = ds.ds_options_default(test="dst3", tol_gap_rel=1e-7, max_iter=20000, lambda_rel=1)
        X = np.zeros((ratios.size, K), dtype=np.float32)  # host output, column j = lambda j
        res = ds.ds_solve_path(ctx, dct, y.astype(np.float32), ratios, o, X)
        lm = res[0]["lambda_max"]
        for j, rt in enumerate(ratios):
            x, r = _solve_gpu(ctx, dct, y, rt * lm, torch.float32, K, test="dst3", tol_gap_rel=1e-7,
                              max_iter=20000)
            np.testing.assert_array_equal(X[j], x.astype(np.float32))
            assert r["iters"] == res[j]["iters"]
    finally:
        ds.ds_dict_destroy(dct)


def test_warm_start_from_solution(ctx):
    N, K = 300, 1200
    D, y, _ = gen.lasso_problem(N, K, seed=13)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.4 * lm
    ref = oracle.solve(D, y, lam, test="dst3", tol=1e-14, max_iter=100000)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        o = ds.ds_options_default(test="dst3", tol_gap_rel=1e-6, max_iter=20000)
        yt = torch.from_numpy(y).to("cuda", torch.float32)
        x = torch.empty(K, device="cuda")
        cold = ds.ds_solve(ctx, dct, yt, lam, o, x)
        warm = ds.ds_solve(ctx, dct, yt, lam, o, x, x0=torch.from_numpy(ref["x"]).to("cuda", torch.float32))
        assert warm["iters"] <= 3 < cold["iters"]
    finally:
        ds.ds_dict_destroy(dct)


def test_history_nested_and_gap_nonnegative(ctx):
    D, y, _ = gen.lasso_problem(800, 4000, seed=17)
    D, y = _f32(D), _f32(y)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    hist = torch.zeros((5000, 6), device="cuda", dtype=torch.float64)
    ds.ds_set_history(ctx, hist)
    try:
        lm, _, _ = oracle.lambda_max(D, y)
        x, r = _solve_gpu(ctx, dct, y, 0.75 * lm, torch.float32, 4000, test="dome", tol_gap_rel=1e-6,
                          max_iter=5000)
    finally:
        ds.ds_set_history(ctx, None)
        ds.ds_dict_destroy(dct)
    h = hist.cpu().numpy()[: r["iters"]]
    assert np.all(np.diff(h[:, 0]) <= 0)
    assert np.all(h[:, 4] >= -1e-6 * (y @ y))
    assert h[-1, 0] < 0.5 * 4000  # dynamic screening removed most atoms


@pytest.mark.parametrize("ratio", [0.3, 0.7])
def test_config2_full_size(ctx, ratio):
    """2000 x 10000 FP32, FISTA + DST3, gap 1e-6 (the benchmark's problem):
    the GPU's answer checked by its FP64 duality gap and the KKT conditions."""
    D, y, _ = gen.config2(1002)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = ratio * lm
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        x, r = _solve_gpu(ctx, dct, y, lam, torch.float32, 10000, test="dst3", tol_gap_rel=1e-6, max_iter=20000)
    finally:
        ds.ds_dict_destroy(dct)
    yy = y @ y
    assert r["status"] == 0 and r["gap"] <= 1e-6 * 0.5 * yy
    assert _fp64_gap(D, y, x, lam) <= 2e-6 * 0.5 * yy
    c = D.T @ (y - D @ x)
    assert np.abs(c).max() <= lam * (1 + 1e-2)


def test_warm_started_path_matches_cold_lambdas(ctx):
    """A regularization path (descending lambda) started from each previous solution reaches
    the same solutions as cold starts, in fewer iterations; the first lambda (>= lambda_*)
    gives x = 0 and seeds the next one."""
    N, K = 400, 2400
    D, y, _ = gen.lasso_problem(N, K, seed=91, p=0.01)
    D, y = _f32(D), _f32(y)
    ratios = np.array([1.2, 0.8, 0.6, 0.45, 0.3, 0.2])
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        yt = torch.from_numpy(y).to("cuda", torch.float32)
        res = {}
        Xs = {}
        for warm in (0, 1):
            X = torch.empty((len(ratios), K), device="cuda")
            o = ds.ds_options_default(test="dst3", tol_gap_rel=1e-7, max_iter=50000, lambda_rel=1, warm_start=warm)
            res[warm] = ds.ds_solve_path(ctx, dct, yt, ratios, o, X)
            Xs[warm] = X.double().cpu().numpy()
    finally:
        ds.ds_dict_destroy(dct)
    yy = float(y @ y)
    for j in range(len(ratios)):
        for warm in (0, 1):
            assert res[warm][j]["status"] == 0 and res[warm][j]["gap"] <= 1e-7 * 0.5 * yy
        # both certify 1e-7: their fits differ by at most sqrt(2 gap) each
        assert np.linalg.norm(D @ (Xs[0][j] - Xs[1][j])) <= 2 * np.sqrt(2e-7 * 0.5 * yy) * 1.01
    assert res[1][0]["iters"] == 0 and not Xs[1][0].any()
    assert sum(r["iters"] for r in res[1]) < sum(r["iters"] for r in res[0])


@pytest.mark.parametrize("test", ["safe", "dst3", "dome", "none"])
def test_chambolle_pock_matches_oracle_iterates(ctx, test):
    """Chambolle-Pock (Table 1, gamma = 0): after a fixed number of iterations the GPU iterate
    equals the FP64 oracle's, with screening inside every iteration (Algorithm 3)."""
    N, K = 400, 1500
    D, y, _ = gen.lasso_problem(N, K, seed=61, p=0.01)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    L = oracle.spectral_norm_sq(D, tol=1e-10, max_iter=5000) * (1 + 1e-6)
    tau = 0.99 / np.sqrt(L)
    ref = oracle.solve(D, y, lam, alg="cp", test=test, tol=0, max_iter=300, L=L, cp_tau=tau, cp_sigma=tau)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32))
    try:
        x, r = _solve_gpu(ctx, dct, y, lam, torch.float32, K, alg="cp", test=test, tol_gap_rel=0.0, max_iter=300,
                          L=L, cp_tau=tau, cp_sigma=tau)
    finally:
        ds.ds_dict_destroy(dct)
    assert r["iters"] == 300
    assert np.abs(x - ref["x"]).max() <= 1e-5 * np.abs(ref["x"]).max()
    assert abs(r["gap"] - ref["gap"]) <= 1e-5 * 0.5 * float(y @ y)


@pytest.mark.parametrize("test", ["gsafe", "dgst3"])
def test_chambolle_pock_group_lasso_certifies_the_gap(ctx, test):
    """Chambolle-Pock on the Group-Lasso, run to the duality gap: certified, and its objective is
    within the tolerance of the FP64 oracle's optimum."""
    N, K = 500, 1500
    D, y, _, goff, w = gen.config3(62, N=N, K=K, gsize=10, n_active=4)
    D, y = _f32(D), _f32(y)
    lm, _, _ = oracle.lambda_max(D, y, goff, w)
    lam = 0.4 * lm
    ref = oracle.solve(D, y, lam, goff, w, alg="fista", test=test, tol=1e-12, max_iter=100000)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float32), goff, w)
    try:
        x, r = _solve_gpu(ctx, dct, y, lam, torch.float32, K, alg="cp", test=test, tol_gap_rel=1e-6, max_iter=100000)
    finally:
        ds.ds_dict_destroy(dct)
    yy = float(y @ y)
    assert r["status"] == 0 and r["gap"] <= 1e-6 * 0.5 * yy
    xg = [x[goff[g]:goff[g + 1]] for g in range(len(w))]
    p = 0.5 * np.sum((D @ x - y) ** 2) + lam * sum(wg * np.linalg.norm(v) for wg, v in zip(w, xg))
    assert p - ref["primal"] <= 1.05e-6 * 0.5 * yy + 1e-9 * yy


def test_chambolle_pock_fp64_config1(ctx):
    """100 x 500 FP64: Chambolle-Pock with dynamic DST3 takes the oracle's iterations."""
    D, y, _ = gen.config1(1001)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    L = oracle.spectral_norm_sq(D) * (1 + 1e-6)
    ref = oracle.solve(D, y, lam, alg="cp", test="dst3", tol=1e-8, max_iter=100000, L=L)
    dct = ds.ds_dict_create(ctx, _dev_dict(D, torch.float64))
    try:
        x, r = _solve_gpu(ctx, dct, y, lam, torch.float64, 500, alg="cp", test="dst3", tol_gap_rel=1e-8,
                          max_iter=100000, L=L)
    finally:
        ds.ds_dict_destroy(dct)
    assert r["status"] == 0
    assert abs(r["iters"] - ref["iters"]) <= 1
    np.testing.assert_allclose(x, ref["x"], atol=1e-9 * np.abs(ref["x"]).max())


def test_bench_workload_full_size_certified_in_fp64(ctx):
    """The benchmark's own workload at full size (2000 x 10000, seed 1002, the three tests x five
    lambdas, in the bench's launch configuration: one path per test): every solution is
    certified independently of the kernel's report, by an FP64 duality gap computed here from
    the returned x with the dual point of Lemma 8 built from its residual."""
    D, y, _ = gen.config2(1002)
    D32, y32 = D.astype(np.float32), y.astype(np.float32)
    D64, y64 = D32.astype(np.float64), y32.astype(np.float64)
    yy = float(y64 @ y64)
    ratios = np.array(gen.CONFIG2_RATIOS)
    dct = ds.ds_dict_create(ctx, _dev_dict(D64, torch.float32))
    try:
        yt = torch.from_numpy(y32).cuda()
        for test in ("safe", "dst3", "dome"):
            X = torch.empty((ratios.size, D.shape[1]), device="cuda")
            o = ds.ds_options_default(test=test, tol_gap_rel=1e-6, max_iter=20000, lambda_rel=1)
            res = ds.ds_solve_path(ctx, dct, yt, ratios, o, X)
            Xh = X.double().cpu().numpy()
            for j, r in enumerate(res):
                assert r["status"] == 0 and r["gap"] <= 1e-6 * 0.5 * yy, (test, j, r)
                lam = r["lambda"]
                x = Xh[j]
                res64 = y64 - D64 @ x
                primal = 0.5 * res64 @ res64 + lam * np.abs(x).sum()
                # dual point s (y - D x): the scaling closest to y / lambda within the feasible set (Lemma 8)
                lim = 1.0 / np.abs(D64.T @ res64).max()
                sc = float(np.clip(res64 @ y64 / (lam * (res64 @ res64)), -lim, lim))
                theta = sc * res64
                dual = 0.5 * yy - 0.5 * lam * lam * np.sum((theta - y64 / lam) ** 2)
                # the FP32 rounding of the returned x adds a little to the kernel's certified gap
                assert primal - dual <= 1.2e-6 * 0.5 * yy, (test, j, (primal - dual) / (0.5 * yy))
                assert abs(lam - ratios[j] * r["lambda_max"]) <= 1e-12 * lam
    finally:
        ds.ds_dict_destroy(dct)
