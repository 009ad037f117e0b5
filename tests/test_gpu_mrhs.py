"""Right-hand sides solved together (multi-RHS blocks) against single solves
and against the oracle's optimum.

A batch instance with several right-hand sides on an FP32 Lasso dictionary is
solved as blocks of up to 64 problems in lockstep, the correlation of each
iteration being one contraction over the union of their active sets.  The
block must reproduce, problem by problem:
  - the single-solve entry point at a fixed iteration count (same updates of
    Table 1, same screening tests of Lemmas 2-4 and 8), within the parity
    tolerance, for every test, FISTA and ISTA, dynamic and static screening;
  - with the gap stopping rule, a certified solution: gap <= tol * 1/2 ||y||^2
    and an objective within that gap of the oracle's FP64 optimum;
  - the degenerate cases: lambda >= lambda_* (x = 0, no iteration) and an
    iteration cap (status "not converged").
Team layouts covered: two blocks on the whole GPU (row splits of the
contraction tiles) and many small blocks with one CTA per team.
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
    c = ds.ds_create(0, None)
    yield c
    ds.ds_destroy(c)


def _dev_dict(D):
    return torch.from_numpy(np.ascontiguousarray(D.T)).to("cuda", torch.float32).t()


def _instance(seed, N, K, nrhs, p=0.02, lo=0.1, hi=0.9):
    g = gen.rng(seed)
    D = gen.gaussian_dict(N, K, g)
    Y = np.stack([gen.observe(D, gen.bernoulli_gaussian_x0(K, p, g), g) for _ in range(nrhs)])
    lam = g.uniform(lo, hi, size=nrhs)
    return D, Y, lam


def _run_batch(ctx, insts, opt):
    dicts = [ds.ds_dict_create(ctx, _dev_dict(D)) for (D, Y, lam) in insts]
    Ys = [torch.from_numpy(Y).to("cuda", torch.float32) for (D, Y, lam) in insts]
    Xs = [torch.full((Y.shape[0], D.shape[1]), float("nan"), device="cuda") for (D, Y, lam) in insts]
    lams = [lam.copy() for (D, Y, lam) in insts]
    plan = ds.ds_batch_create(ctx, dicts, Ys, lams, opt, Xs)
    layout = ds.ds_batch_layout(plan)
    res = ds.ds_batch_run(plan)
    torch.cuda.synchronize()
    ds.ds_batch_destroy(plan)
    return dicts, Ys, Xs, lams, res, layout


@pytest.mark.parametrize("test,alg,dynamic", [("none", "fista", 1), ("safe", "fista", 1), ("dst3", "fista", 1),
                                              ("dome", "fista", 1), ("dst3", "ista", 1), ("dome", "fista", 0)])
def test_multi_rhs_matches_single_solves(ctx, test, alg, dynamic):
    # 70 right-hand sides: a block of 64 and a ragged one of 6; N, K off every tile size
    insts = [_instance(301, 300, 1500, 70)]
    opt = ds.ds_options_default(test=test, alg=alg, dynamic=dynamic, tol_gap_rel=0.0, max_iter=300, lambda_rel=1)
    dicts, Ys, Xs, lams, res, layout = _run_batch(ctx, insts, opt)
    try:
        assert layout["multi_rhs_blocks"] == 2 and layout["single_problems"] == 0, layout
        D, Y, lam = insts[0]
        for r in range(Y.shape[0]):
            x1 = torch.zeros(D.shape[1], device="cuda")
            one = ds.ds_solve(ctx, dicts[0], Ys[0][r].contiguous(), lams[0][r], opt, x1)
            a = x1.double().cpu().numpy()
            b = Xs[0][r].double().cpu().numpy()
            assert res[r]["status"] == 0 and res[r]["iters"] == one["iters"] == 300, (r, res[r])
            assert np.isfinite(b).all()
            assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1e-30), (r, np.abs(a - b).max())
            assert abs(res[r]["lambda_max"] - one["lambda_max"]) <= 1e-12 * one["lambda_max"]
            assert abs(res[r]["gap"] - one["gap"]) <= 1e-6 * 0.5 * float(Y[r] @ Y[r])
            if test != "none":
                # the same screening decisions up to the rounding margin
                assert abs(res[r]["n_active"] - one["n_active"]) <= max(2, one["n_active"] // 100), (r, res[r], one)
    finally:
        for d in dicts:
            ds.ds_dict_destroy(d)


def _primal(D, y, x, lam):
    r = D @ x - y
    return 0.5 * float(r @ r) + lam * float(np.abs(x).sum())


@pytest.mark.parametrize("test", ["dst3", "dome"])
def test_multi_rhs_certified_against_oracle_optimum(ctx, test):
    insts = [_instance(302, 100, 400, 20, p=0.03)]
    tol = 1e-6
    opt = ds.ds_options_default(test=test, tol_gap_rel=tol, max_iter=50000, lambda_rel=1)
    dicts, Ys, Xs, lams, res, layout = _run_batch(ctx, insts, opt)
    try:
        D, Y, lam = insts[0]
        D32 = D.astype(np.float32).astype(np.float64)
        for r in range(Y.shape[0]):
            y = Y[r].astype(np.float32).astype(np.float64)
            yy = float(y @ y)
            assert res[r]["status"] == 0 and res[r]["gap"] <= tol * 0.5 * yy, res[r]
            lam_abs = res[r]["lambda"]
            assert abs(lam_abs - lams[0][r] * res[r]["lambda_max"]) <= 1e-12 * lam_abs
            o = oracle.solve(D32, y, lam_abs, test="none", tol=1e-13, max_iter=200000)
            p_star = o["primal"]
            x = Xs[0][r].double().cpu().numpy()
            p = _primal(D32, y, x, lam_abs)
            # the certified gap bounds the suboptimality (plus the FP32 rounding of x)
            assert p - p_star <= 1.05 * tol * 0.5 * yy + 1e-9 * yy, (r, p - p_star)
            assert p - p_star >= -1e-9 * yy
    finally:
        for d in dicts:
            ds.ds_dict_destroy(d)


def test_multi_rhs_degenerate_cases(ctx):
    D, Y, lam = _instance(303, 200, 700, 8)
    lam[1] = 1.0     # lambda = lambda_*: x = 0
    lam[5] = 1.7     # above lambda_*
    opt = ds.ds_options_default(test="dst3", tol_gap_rel=1e-9, max_iter=25, lambda_rel=1)
    dicts, Ys, Xs, lams, res, layout = _run_batch(ctx, [(D, Y, lam)], opt)
    try:
        assert layout["multi_rhs_blocks"] == 1
        for r in range(8):
            x = Xs[0][r].double().cpu().numpy()
            if r in (1, 5):
                assert res[r]["iters"] == 0 and res[r]["status"] == 0 and not x.any()
                assert res[r]["gap"] == 0.0
            else:
                # the cap stops every other problem before its tiny tolerance
                assert res[r]["iters"] == 25 and res[r]["status"] == ds.DS_ERR_NOT_CONVERGED, res[r]
                assert np.isfinite(x).all()
    finally:
        for d in dicts:
            ds.ds_dict_destroy(d)


def test_multi_rhs_one_cta_teams(ctx):
    # more blocks than SMs, teams of one CTA (ds_options.team_size): each takes several blocks in turn
    g = gen.rng(304)
    insts = []
    for k in range(170):
        N = int(g.integers(40, 130))
        K = int(g.integers(100, 400))
        insts.append(_instance(1000 + k, N, K, 2))
    opt = ds.ds_options_default(test="dst3", tol_gap_rel=0.0, max_iter=120, lambda_rel=1, team_size=1)
    dicts, Ys, Xs, lams, res, layout = _run_batch(ctx, insts, opt)
    try:
        assert layout["multi_rhs_blocks"] == 170 and layout["multi_rhs_team_size"] == 1, layout
        i = 0
        for k, (D, Y, lam) in enumerate(insts):
            for r in range(2):
                if k % 17 == 0:
                    x1 = torch.zeros(D.shape[1], device="cuda")
                    one = ds.ds_solve(ctx, dicts[k], Ys[k][r].contiguous(), lams[k][r], opt, x1)
                    a = x1.double().cpu().numpy()
                    b = Xs[k][r].double().cpu().numpy()
                    assert res[i]["iters"] == one["iters"] == 120
                    assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1e-30), (k, r)
                i += 1
    finally:
        for d in dicts:
            ds.ds_dict_destroy(d)


def test_multi_rhs_can_be_turned_off(ctx):
    insts = [_instance(305, 150, 500, 4)]
    opt = ds.ds_options_default(test="dst3", tol_gap_rel=1e-6, max_iter=5000, lambda_rel=1)
    opt.batch_multi_rhs = 0
    dicts, Ys, Xs, lams, res, layout = _run_batch(ctx, insts, opt)
    try:
        assert layout["multi_rhs_blocks"] == 0 and layout["single_problems"] == 4
        assert all(r["status"] == 0 for r in res)
    finally:
        for d in dicts:
            ds.ds_dict_destroy(d)


def _run_batch_dicts(ctx, dicts, insts, opt):
    Ys = [torch.from_numpy(Y).to("cuda", torch.float32) for (D, Y, lam) in insts]
    Xs = [torch.full((Y.shape[0], D.shape[1]), float("nan"), device="cuda") for (D, Y, lam) in insts]
    plan = ds.ds_batch_create(ctx, dicts, Ys, [lam.copy() for (_, _, lam) in insts], opt, Xs)
    res = ds.ds_batch_run(plan)
    torch.cuda.synchronize()
    ds.ds_batch_destroy(plan)
    return Xs, res


@pytest.mark.parametrize("test", ["dst3", "dome"])
def test_multi_rhs_tensor_core_bulk_matches_fp32(ctx, test):
    # BF16 copy: the bulk iterations contract on the tensor cores (theta split in BF16 hi + lo),
    # then the block finishes on the FP32 master; at a fixed iteration count the solutions
    # equal the FP32 block's within the parity tolerance
    insts = [_instance(306, 300, 1500, 70)]
    D = insts[0][0]
    Dt = _dev_dict(D)
    d32 = ds.ds_dict_create(ctx, Dt)
    dbf = ds.ds_dict_create(ctx, Dt, work_prec=ds.DS_BF16)
    try:
        opt = ds.ds_options_default(test=test, tol_gap_rel=0.0, max_iter=3000, lambda_rel=1)
        xa, ra = _run_batch_dicts(ctx, [d32], insts, opt)
        xb, rb = _run_batch_dicts(ctx, [dbf], insts, opt)
        a = xa[0].double().cpu().numpy()
        b = xb[0].double().cpu().numpy()
        assert np.isfinite(b).all()
        for r in range(a.shape[0]):
            assert rb[r]["iters"] == ra[r]["iters"] == 3000
            assert 0 < rb[r]["cols_lowp"] < rb[r]["cols_corr"], rb[r]
            assert np.abs(a[r] - b[r]).max() <= 1e-5 * max(np.abs(a[r]).max(), 1e-30), (r, np.abs(a[r] - b[r]).max())
        # with the gap rule the tensor-core block certifies the tolerance, at the oracle's optimum
        tol = 1e-6
        opt = ds.ds_options_default(test=test, tol_gap_rel=tol, max_iter=50000, lambda_rel=1)
        xc, rc = _run_batch_dicts(ctx, [dbf], insts, opt)
        D32 = D.astype(np.float32).astype(np.float64)
        Y = insts[0][1]
        for r in range(0, Y.shape[0], 7):
            y = Y[r].astype(np.float32).astype(np.float64)
            yy = float(y @ y)
            assert rc[r]["status"] == 0 and rc[r]["gap"] <= tol * 0.5 * yy, rc[r]
            o = oracle.solve(D32, y, rc[r]["lambda"], test="none", tol=1e-13, max_iter=200000)
            x = xc[0][r].double().cpu().numpy()
            p = _primal(D32, y, x, rc[r]["lambda"])
            assert p - o["primal"] <= 1.05 * tol * 0.5 * yy + 1e-9 * yy, (r, p - o["primal"])
    finally:
        ds.ds_dict_destroy(d32)
        ds.ds_dict_destroy(dbf)


def test_autotuner_keeps_a_valid_schedule_and_lambda_sorted_blocks_map_back(ctx):
    # two candidates: the default schedule, then blocks of 32 grouped by lambda; the last tuning
    # run (the lambda-sorted one) leaves its solutions in X, which must map back to the caller's
    # right-hand sides; the kept schedule must then solve the batch again
    insts = [_instance(307, 300, 1500, 70)]
    D, Y, lam = insts[0]
    d = ds.ds_dict_create(ctx, _dev_dict(D))
    try:
        Yt = torch.from_numpy(Y).to("cuda", torch.float32)
        X = torch.full((70, 1500), float("nan"), device="cuda")
        opt = ds.ds_options_default(test="dst3", tol_gap_rel=0.0, max_iter=200, lambda_rel=1)
        plan = ds.ds_batch_create(ctx, [d], [Yt], [lam.copy()], opt, [X])
        tune = ds.ds_batch_autotune(plan, max_candidates=2)
        assert len(tune["ms"]) == 2 and all(m > 0 for m in tune["ms"]), tune
        assert tune["chosen"] in (0, 1)
        for r in range(0, 70, 5):
            x1 = torch.zeros(1500, device="cuda")
            one = ds.ds_solve(ctx, d, Yt[r].contiguous(), float(lam[r]), opt, x1)
            a = x1.double().cpu().numpy()
            b = X[r].double().cpu().numpy()
            assert one["iters"] == 200
            assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1e-30), r
        X.fill_(float("nan"))
        res = ds.ds_batch_run(plan)
        assert all(rr["iters"] == 200 for rr in res)
        assert torch.isfinite(X).all()
        ds.ds_batch_destroy(plan)
    finally:
        ds.ds_dict_destroy(d)
