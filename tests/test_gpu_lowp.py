"""Precision variant: BF16 and FP8 (per-column scale) working copies.

The bulk iterations read the copy, screening radii are inflated by the copy's
rigorous error bound, and FP32 iterations on the master finish the solve; the
result must match the FP32 solve within the parity tolerance, the copy must
actually have been used, and the gap tolerance must be met."""
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


@pytest.mark.parametrize("prec", [ds.DS_BF16, ds.DS_FP8])
@pytest.mark.parametrize("ratio,test", [(0.3, "dst3"), (0.8, "dome"), (0.6, "safe")])
def test_lowp_matches_fp32(ctx, prec, ratio, test):
    D, y, _ = gen.lasso_problem(1100, 3000, seed=61, p=0.02)
    D = D.astype(np.float32).astype(np.float64)
    y = y.astype(np.float32)
    Dt = _dev_dict(D)
    d32 = ds.ds_dict_create(ctx, Dt)
    dlo = ds.ds_dict_create(ctx, Dt, work_prec=prec)
    try:
        yt = torch.from_numpy(y).cuda()
        o = ds.ds_options_default(test=test, tol_gap_rel=0.0, max_iter=3000, lambda_rel=1)
        xa = torch.zeros(3000, device="cuda")
        xb = torch.zeros(3000, device="cuda")
        ra = ds.ds_solve(ctx, d32, yt, ratio, o, xa)
        rb = ds.ds_solve(ctx, dlo, yt, ratio, o, xb)
        a = xa.double().cpu().numpy()
        b = xb.double().cpu().numpy()
        assert rb["cols_lowp"] > 0 and rb["cols_lowp"] < rb["cols_corr"]
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()
        # stopping on the gap: the low-precision run certifies the same tolerance
        o2 = ds.ds_options_default(test=test, tol_gap_rel=1e-6, max_iter=20000, lambda_rel=1)
        rc = ds.ds_solve(ctx, dlo, yt, ratio, o2, xb)
        assert rc["status"] == 0 and rc["gap"] <= 1e-6 * 0.5 * float(y.astype(np.float64) @ y.astype(np.float64))
        # safety: no atom of the FP64 solution was screened away (support recovered)
        lm, _, _ = oracle.lambda_max(D, y.astype(np.float64))
        ref = oracle.solve(D, y.astype(np.float64), ratio * lm, test="none", tol=1e-13, max_iter=100000)
        xs = xb.double().cpu().numpy()
        big = np.abs(ref["x"]) > 1e-3 * np.abs(ref["x"]).max()
        assert np.all(xs[big] != 0)
    finally:
        ds.ds_dict_destroy(d32)
        ds.ds_dict_destroy(dlo)


def test_lowp_group_lasso(ctx):
    D, y, _, goff, w = gen.config3(62, N=600, K=1800, gsize=10, n_active=6)
    D = D.astype(np.float32).astype(np.float64)
    Dt = _dev_dict(D)
    d32 = ds.ds_dict_create(ctx, Dt, goff, w)
    dlo = ds.ds_dict_create(ctx, Dt, goff, w, work_prec=ds.DS_BF16)
    try:
        yt = torch.from_numpy(y.astype(np.float32)).cuda()
        o = ds.ds_options_default(test="dgst3", tol_gap_rel=0.0, max_iter=2500, lambda_rel=1)
        xa = torch.zeros(1800, device="cuda")
        xb = torch.zeros(1800, device="cuda")
        ds.ds_solve(ctx, d32, yt, 0.5, o, xa)
        rb = ds.ds_solve(ctx, dlo, yt, 0.5, o, xb)
        a = xa.double().cpu().numpy()
        b = xb.double().cpu().numpy()
        assert rb["cols_lowp"] > 0
        assert np.abs(a - b).max() <= 1e-5 * np.abs(a).max()
    finally:
        ds.ds_dict_destroy(d32)
        ds.ds_dict_destroy(dlo)
