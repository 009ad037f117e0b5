"""Failure detection on the GPU without a fault: a kernel whose grid barrier can
never complete (one CTA never arrives, as if it were lost) gives up after the
barrier's time limit, returns a status the host reads, and leaves the context
usable for the next solve."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_1412_4080_gb300 as ds

pytestmark = pytest.mark.gpu


def test_barrier_wait_gives_up_and_reports_timeout():
    status, ms = ds.ds_selftest_wait_timeout(0)
    assert status == ds.DS_ERR_TIMEOUT
    # the wait is bounded by a 2 s clock limit (a few polls of slack)
    assert 1900.0 <= ms <= 10000.0, ms


def test_device_still_solves_after_a_timed_out_launch():
    status, _ = ds.ds_selftest_wait_timeout(0)
    assert status == ds.DS_ERR_TIMEOUT
    N, K = 200, 700
    D, y, _ = gen.lasso_problem(N, K, seed=77, p=0.02)
    D, y = D.astype(np.float32).astype(np.float64), y.astype(np.float32).astype(np.float64)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = 0.5 * lm
    ref = oracle.solve(D, y, lam, alg="fista", test="dst3", tol=1e-12, max_iter=100000)
    ctx = ds.ds_create(0, None)
    Dt = torch.from_numpy(np.ascontiguousarray(D.T)).to("cuda", torch.float32).t()
    dct = ds.ds_dict_create(ctx, Dt)
    try:
        o = ds.ds_options_default(test="dst3", tol_gap_rel=1e-7, max_iter=20000)
        x = torch.empty(K, device="cuda")
        r = ds.ds_solve(ctx, dct, torch.from_numpy(y).to("cuda", torch.float32), lam, o, x)
    finally:
        ds.ds_dict_destroy(dct)
        ds.ds_destroy(ctx)
    assert r["status"] == 0
    xs = x.double().cpu().numpy()
    assert np.abs(xs - ref["x"]).max() <= 1e-3 * np.abs(ref["x"]).max()
