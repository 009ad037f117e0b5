"""Batched solves (one persistent multi-team launch) against single solves.

Instances of uneven sizes (Lasso and Group-Lasso dictionaries of different N
and K) with several right-hand sides and lambda values each; every batched
solution must match the single-solve entry point on the same problem within
the parity tolerance, on two runs of the same plan (the second with new y
values and lambdas written in place).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import gen
import paper_1412_4080_gb300 as ds

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = ds.ds_create(0, None)
    yield c
    ds.ds_destroy(c)


def _dev_dict(D):
    return torch.from_numpy(np.ascontiguousarray(D.T)).to("cuda", torch.float32).t()


def _instances(seed):
    g = gen.rng(seed)
    out = []
    for (N, K, groups, nrhs) in ((300, 1500, False, 3), (700, 2100, False, 2), (520, 1200, True, 2), (129, 640, False, 4)):
        D = gen.gaussian_dict(N, K, g)
        goff = gen.contiguous_groups(K, 8) if groups else None
        Y = np.stack([gen.observe(D, gen.bernoulli_gaussian_x0(K, 0.02, g), g) for _ in range(nrhs)])
        lam = g.uniform(0.2, 0.9, size=nrhs)
        out.append((D, goff, Y, lam))
    return out


@pytest.mark.parametrize("alg", ["fista", "cp"])
@pytest.mark.parametrize("test", ["none", "dst3"])
def test_batch_matches_single_solves(ctx, test, alg):
    inst = _instances(77)
    dicts = [ds.ds_dict_create(ctx, _dev_dict(D), goff) for (D, goff, Y, lam) in inst]
    try:
        Ys = [torch.from_numpy(Y).to("cuda", torch.float32) for (D, goff, Y, lam) in inst]
        Xs = [torch.zeros((Y.shape[0], D.shape[1]), device="cuda") for (D, goff, Y, lam) in inst]
        lams = [lam.copy() for (D, goff, Y, lam) in inst]
        t_group = "dgst3" if test == "dst3" else "none"
        # one options set for all: group dictionaries read DST3 as its group form
        # (Chambolle-Pock problems run one per team; FISTA Lasso instances as multi-RHS blocks)
        opt = ds.ds_options_default(alg=alg, test=t_group, tol_gap_rel=0.0, max_iter=1500, lambda_rel=1)
        plan = ds.ds_batch_create(ctx, dicts, Ys, lams, opt, Xs)
        info = ds.ds_batch_info(plan)
        print("batch plan:", info)
        for run in range(2):
            if run == 1:
                g = gen.rng(5)
                for k, (D, goff, Y, lam) in enumerate(inst):
                    Ynew = np.stack([gen.observe(D, gen.bernoulli_gaussian_x0(D.shape[1], 0.02, g), g)
                                     for _ in range(Y.shape[0])])
                    Ys[k].copy_(torch.from_numpy(Ynew))
                    lams[k][:] = g.uniform(0.2, 0.9, size=Y.shape[0])
            res = ds.ds_batch_run(plan)
            torch.cuda.synchronize()
            i = 0
            for k, (D, goff, Y, lam) in enumerate(inst):
                for r in range(Y.shape[0]):
                    x1 = torch.zeros(D.shape[1], device="cuda")
                    one = ds.ds_solve(ctx, dicts[k], Ys[k][r].contiguous(), lams[k][r], opt, x1)
                    a = x1.double().cpu().numpy()
                    b = Xs[k][r].double().cpu().numpy()
                    assert res[i]["status"] == 0 and res[i]["iters"] == one["iters"] == 1500
                    assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1e-30), (k, r, run)
                    assert abs(res[i]["lambda_max"] - one["lambda_max"]) <= 1e-12 * one["lambda_max"]
                    i += 1
        ds.ds_batch_destroy(plan)
    finally:
        for d in dicts:
            ds.ds_dict_destroy(d)


def test_solve_batch_one_shot_converges(ctx):
    inst = _instances(78)
    dicts = [ds.ds_dict_create(ctx, _dev_dict(D), goff) for (D, goff, Y, lam) in inst]
    try:
        Ys = [torch.from_numpy(Y).to("cuda", torch.float32) for (D, goff, Y, lam) in inst]
        Xs = [torch.zeros((Y.shape[0], D.shape[1]), device="cuda") for (D, goff, Y, lam) in inst]
        opt = ds.ds_options_default(test="gsafe", tol_gap_rel=1e-6, max_iter=20000, lambda_rel=1)
        res = ds.ds_solve_batch(ctx, dicts, Ys, [l for (_, _, _, l) in inst], opt, Xs)
        for (D, goff, Y, lam), k0 in zip(inst, np.cumsum([0] + [i[2].shape[0] for i in inst])[:-1]):
            for r in range(Y.shape[0]):
                rr = res[k0 + r]
                assert rr["status"] == 0 and rr["gap"] <= 1e-6 * 0.5 * float(Y[r].astype(np.float32) @ Y[r].astype(np.float32)) * 1.001
    finally:
        for d in dicts:
            ds.ds_dict_destroy(d)
