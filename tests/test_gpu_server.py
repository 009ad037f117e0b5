"""Continuous-batching server: every request gives the same result alone and in
a mix of concurrent requests (Lasso and Group-Lasso, different sizes and
lambdas), and matches the single-solve entry point within the parity
tolerance."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import gen
import paper_1412_4080_gb300 as ds

pytestmark = pytest.mark.gpu


def _dev_dict(D):
    return torch.from_numpy(np.ascontiguousarray(D.T)).to("cuda", torch.float32).t()


def _wait(server, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = ds.ds_server_poll(server, t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "server requests did not complete"
        time.sleep(0.0005)
    return [out[t] for t in tickets]


def test_server_alone_equals_mix_and_single_solves():
    g = gen.rng(303)
    ctx = ds.ds_create(0, None)
    specs = [(600, 2400, None), (512, 2048, 8), (257, 1024, None)]
    dicts, mats = [], []
    for (N, K, gs) in specs:
        D = gen.gaussian_dict(N, K, g)
        goff = gen.contiguous_groups(K, gs) if gs else None
        dicts.append(ds.ds_dict_create(ctx, _dev_dict(D), goff))
        mats.append((D, goff))
    reqs = []
    for k in range(12):
        di = k % len(specs)
        D, goff = mats[di]
        y = gen.observe(D, gen.bernoulli_gaussian_x0(D.shape[1], 0.02, g), g).astype(np.float32)
        ratio = float(g.uniform(0.3, 0.9))
        test = "dgst3" if goff is not None else ("dst3", "dome", "safe")[k % 3]
        reqs.append((di, y, ratio, test))
    server = ds.ds_server_create(ctx, 256 << 20, 1024, 4096, 4)
    try:
        def opt(test):
            return ds.ds_options_default(test=test, tol_gap_rel=0.0, max_iter=700, lambda_rel=1)
        # alone: one request in flight at a time
        alone = []
        for (di, y, ratio, test) in reqs:
            x = np.zeros(mats[di][0].shape[1], dtype=np.float32)
            t = ds.ds_server_submit(server, dicts[di], y, ratio, opt(test), x)
            r = _wait(server, [t])[0]
            alone.append((x, r))
        # mix: all requests in flight together
        xs, ts = [], []
        for (di, y, ratio, test) in reqs:
            x = np.zeros(mats[di][0].shape[1], dtype=np.float32)
            xs.append(x)
            ts.append(ds.ds_server_submit(server, dicts[di], y, ratio, opt(test), x))
        mix = _wait(server, ts)
        st = ds.ds_server_stats(server)
        print("server stats:", st)
        for k, (di, y, ratio, test) in enumerate(reqs):
            xa, ra = alone[k]
            assert ra["status"] == 0 and mix[k]["status"] == 0
            # same team size, fixed-order reductions: bitwise the same alone and in the mix
            np.testing.assert_array_equal(xa, xs[k])
            assert ra["iters"] == mix[k]["iters"] == 700
            # and the single-solve entry point agrees within the parity tolerance
            x1 = torch.zeros(mats[di][0].shape[1], device="cuda")
            ds.ds_solve(ctx, dicts[di], torch.from_numpy(y).cuda(), ratio, opt(test), x1)
            a = x1.double().cpu().numpy()
            assert np.abs(a - xa.astype(np.float64)).max() <= 1e-5 * max(np.abs(a).max(), 1e-30)
    finally:
        ds.ds_server_destroy(server)
        for d in dicts:
            ds.ds_dict_destroy(d)
        ds.ds_destroy(ctx)


def test_server_rejects_oversized_and_admits_by_pool():
    g = gen.rng(304)
    ctx = ds.ds_create(0, None)
    D = gen.gaussian_dict(700, 3000, g)
    dct = ds.ds_dict_create(ctx, _dev_dict(D))
    server = ds.ds_server_create(ctx, 8 << 20, 512, 4096, 2)  # N above 512 is refused; a small pool
    try:
        y = gen.observe(D, gen.bernoulli_gaussian_x0(3000, 0.02, g), g).astype(np.float32)
        x = np.zeros(3000, dtype=np.float32)
        with pytest.raises(ds.DscreenError) as e:
            ds.ds_server_submit(server, dct, y, 0.5, ds.ds_options_default(lambda_rel=1), x)
        assert e.value.status == ds.DS_ERR_UNSUPPORTED
    finally:
        ds.ds_server_destroy(server)
        ds.ds_dict_destroy(dct)
        ds.ds_destroy(ctx)


def test_server_requests_after_a_lull_run_side_by_side():
    # A long request keeps one team busy while the others wait long enough to count themselves
    # idle; requests submitted then must still be spread over all teams (the launch ends only when
    # every team is idle), not queued behind the busy team.
    g = gen.rng(304)
    ctx = ds.ds_create(0, None)
    N, K = 700, 4000
    D = gen.gaussian_dict(N, K, g)
    d = ds.ds_dict_create(ctx, _dev_dict(D))
    ys = [gen.observe(D, gen.bernoulli_gaussian_x0(K, 0.02, g), g).astype(np.float32) for _ in range(9)]
    o = ds.ds_options_default(test="dst3", tol_gap_rel=0.0, max_iter=4000, lambda_rel=1)
    srv = ds.ds_server_create(ctx, 1 << 30, N, K, 4)
    try:
        x = np.zeros(K, dtype=np.float32)
        t0 = time.time()
        (r0,) = _wait(srv, [ds.ds_server_submit(srv, d, ys[0], 0.5, o, x)])
        t_one = time.time() - t0
        long_x = np.zeros(K, dtype=np.float32)
        o_long = ds.ds_options_default(test="dst3", tol_gap_rel=0.0, max_iter=40000, lambda_rel=1)
        t_long = ds.ds_server_submit(srv, d, ys[0], 0.5, o_long, long_x)
        time.sleep(0.2)  # the idle teams pass their idle limit meanwhile
        xs = [np.zeros(K, dtype=np.float32) for _ in range(8)]
        t1 = time.time()
        res = _wait(srv, [ds.ds_server_submit(srv, d, ys[k + 1], 0.5, o, xs[k]) for k in range(8)])
        t_eight = time.time() - t1
        _wait(srv, [t_long])
        assert all(r["iters"] == 4000 for r in res)
        # side by side: eight requests take about as long as one (queued they would take eight times as long)
        assert t_eight < 4.0 * t_one, (t_eight, t_one)
    finally:
        ds.ds_server_destroy(srv)
        ds.ds_dict_destroy(d)
        ds.ds_destroy(ctx)


def test_server_mixes_fixed_and_adaptive_step_requests():
    """Requests with the adaptive-step rows (SpaRSA, TwIST, FISTA with backtracking) between
    fixed-step ones: the server runs each on the kernel instance that has its code (an adaptive
    request waits for such a launch), and every result matches ds_solve with the same options."""
    g = gen.rng(305)
    ctx = ds.ds_create(0, None)
    D = gen.gaussian_dict(400, 1600, g)
    dct = ds.ds_dict_create(ctx, _dev_dict(D))
    server = ds.ds_server_create(ctx, 256 << 20, 1024, 4096, 8)
    kinds = [dict(alg="fista"), dict(alg="sparsa"), dict(alg="fista"), dict(alg="twist"),
             dict(alg="fista", step_backtracking=1), dict(alg="ista"), dict(alg="sparsa")]
    try:
        reqs = []
        for k, kw in enumerate(kinds):
            y = gen.observe(D, gen.bernoulli_gaussian_x0(1600, 0.02, g), g).astype(np.float32)
            o = ds.ds_options_default(test="dst3", tol_gap_rel=1e-7, max_iter=50000, lambda_rel=1, **kw)
            x = np.zeros(1600, dtype=np.float32)
            reqs.append((y, o, x, ds.ds_server_submit(server, dct, y, 0.4 + 0.05 * k, o, x)))
        res = _wait(server, [r[3] for r in reqs])
        for k, (y, o, x, _) in enumerate(reqs):
            assert res[k]["status"] == 0
            xd = torch.zeros(1600, device="cuda")
            ref = ds.ds_solve(ctx, dct, torch.from_numpy(y).cuda(), 0.4 + 0.05 * k, o, xd)
            xr = xd.double().cpu().numpy()
            assert ref["status"] == 0
            assert np.abs(x - xr).max() <= 1e-4 * np.abs(xr).max(), (k, kinds[k])
    finally:
        ds.ds_server_destroy(server)
        ds.ds_dict_destroy(dct)
        ds.ds_destroy(ctx)
