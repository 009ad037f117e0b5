#!/usr/bin/env python
"""Benchmark of the dynamic-screening Lasso solver on one GB300 (or N, one per rank).

Workload (one "step"): the 2000 x 10000 FP32 Lasso problem of the paper's
synthetic experiments -- Gaussian dictionary with unit-norm columns,
Bernoulli(0.01)-Gaussian x0, y = D x0 + noise at exactly 20 dB (seed 1002) --
solved by FISTA with dynamic SAFE, DST3 and Dome screening for
lambda / lambda_max in {0.1, 0.3, 0.5, 0.7, 0.9}, each to duality gap
1e-6 * 1/2 ||y||^2: 15 solves.  The step also registers the dictionary
(column norms and the Lanczos step bound), so it measures the whole job from
D and y resident in HBM to the 15 solutions.

Metric: solves per second (whole job; N ranks each run the step on their own
GPU, weak scaling, no collective on the data path).  The L2 (129 MB) is
flushed by a 256 MB write before every timed step, since D (80 MB) fits in it.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

RATIOS = (0.1, 0.3, 0.5, 0.7, 0.9)
TESTS = ("safe", "dst3", "dome")
TOL = 1e-6
METRIC = "Lasso solves/s to gap 1e-6 (batched+served vs plain); HBM GB/s; p50/p99 latency"
WORKLOAD = ("Lasso FISTA + dynamic SAFE/DST3/Dome, FP32, D 2000x10000 Gaussian unit-norm columns, "
            "x0 Bernoulli(0.01)-Gaussian, y = D x0 + noise at 20 dB (seed 1002), "
            "lambda/lambda_max in {0.1,0.3,0.5,0.7,0.9}, gap 1e-6 * 1/2||y||^2; step = dictionary "
            "precompute + 15 solves")


def _strip_comments(src):
    """C++ source without its comments and blank lines (a comment edit leaves the kernel as it was)."""
    import re
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())


def solve_kernel_source_hash():
    """sha256 (16 hex digits) of the solve kernel's sources without comments, recorded beside
    each ncu capture."""
    import hashlib
    src = "".join(_strip_comments(open(os.path.join(ROOT, "paper_1412_4080_gb300", "csrc", f)).read())
                  for f in ("ds_solve.cu", "ds_solve_body.cuh", "ds_common.cuh"))
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def _kernel_traffic(name="solve_kernel_config2.md", key="dram_bytes_per_launch:"):
    """A DRAM-bytes figure from a committed ncu summary, if the kernel sources still
    hash to the value recorded there (else None)."""
    prof = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(prof):
        return None
    rec, val = None, None
    for line in open(prof):
        if line.startswith("source-sha256:"):
            rec = line.split()[1]
        if line.startswith(key):
            val = float(line.split()[1])
    return val if rec == solve_kernel_source_hash() else None


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # the samples go to a scratch file; their summary goes into the JSON line
        self.path = os.path.join(tempfile.gettempdir(), f"dscreen_clocks_{os.getpid()}_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def problem():
    import gen
    D, y, _ = gen.config2(1002)
    return D.astype(np.float32), y.astype(np.float32)


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    """The FP64 oracle timed on the host cores (one core: it is single-threaded)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    D32, y32 = problem()
    D = D32.astype(np.float64)
    y = y32.astype(np.float64)
    L = float(np.linalg.norm(D, 2) ** 2) * (1 + 1e-6)
    oracle.build()

    def step(k):
        test = TESTS[k % len(TESTS)]
        lm, _, _ = oracle.lambda_max(D, y)
        n = 0
        for r in RATIOS:
            oracle.solve(D, y, r * lm, alg="fista", test=test, tol=TOL, max_iter=20000, L=L)
            n += 1
        return n

    for k in range(args.warmup):
        step(k)
    t0 = time.perf_counter()
    solves = 0
    for k in range(args.steps):
        solves += step(k)
    dt = time.perf_counter() - t0
    v = solves / dt
    sample = ("oracle FISTA to gap 1e-6 on the same 2000x10000 problem, 5 lambda values per step with one "
              "test per step (SAFE, DST3, Dome in turn); step constant from LAPACK, untimed")
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": {"workload": WORKLOAD},
                      "cpu_baseline": {"value": v, "unit": "solves/s", "cores": 1, "kind": "oracle", "sample": sample},
                      "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def cpu_baseline(D32, y32, budget_s=30.0):
    """Oracle solves of a bounded sample of the workload (DST3, the 5 lambda values)."""
    import oracle
    D = D32.astype(np.float64)
    y = y32.astype(np.float64)
    L = float(np.linalg.norm(D, 2) ** 2) * (1 + 1e-6)
    oracle.build()
    lm, _, _ = oracle.lambda_max(D, y)
    t0 = time.perf_counter()
    n = 0
    for r in (0.9, 0.7, 0.5, 0.3, 0.1):
        oracle.solve(D, y, r * lm, alg="fista", test="dst3", tol=TOL, max_iter=20000, L=L)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    # the small FP64 case of small_fp64_latency, one solve at a time
    import gen
    D1, y1, _ = gen.config1(1001)
    L1 = float(np.linalg.norm(D1, 2) ** 2) * (1 + 1e-6)
    lm1, _, _ = oracle.lambda_max(D1, y1)
    ms1 = []
    for _ in range(3):
        t1 = time.perf_counter()
        oracle.solve(D1, y1, 0.5 * lm1, alg="ista", test="dst3", tol=1e-8, max_iter=100000, L=L1)
        ms1.append(1e3 * (time.perf_counter() - t1))
    return {"value": n / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} oracle FISTA+DST3 solves (lambda/lambda_max = 0.9, 0.7, 0.5, 0.3, 0.1 in turn) of the "
                      f"same problem in {dt:.1f} s, single thread",
            "small_fp64_latency_ms": statistics.median(ms1)}


def _oracle_core(k, L, budget_s, barrier, q):
    """One host core: oracle FISTA + DST3 solves of the 2000 x 10000 workload, lambda ratios
    0.9, 0.7, ..., 0.1 in turn from an offset k, starting no new solve after the budget."""
    import oracle
    D32, y32 = problem()
    D, y = D32.astype(np.float64), y32.astype(np.float64)
    lm, _, _ = oracle.lambda_max(D, y)
    seq = (0.9, 0.7, 0.5, 0.3, 0.1)
    barrier.wait()  # every core has its data: the timed region starts here
    t0 = time.time()
    n = 0
    while time.time() - t0 < budget_s:
        oracle.solve(D, y, seq[(k + n) % 5] * lm, alg="fista", test="dst3", tol=TOL, max_iter=20000, L=L)
        n += 1
    q.put((n, time.time()))


def cpu_baseline_all_cores(budget_s=20.0):
    """Throughput of independent oracle solves over every host core this process may use
    (os.sched_getaffinity): one single-threaded oracle per core, in spawned processes that
    load the problem first and start together at a barrier."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    D32, _ = problem()
    L = float(np.linalg.norm(D32.astype(np.float64), 2) ** 2) * (1 + 1e-6)
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores + 1)
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_core, args=(k, L, budget_s, barrier, q)) for k in range(cores)]
    for p_ in procs:
        p_.start()
    barrier.wait()
    t0 = time.time()
    got = [q.get() for _ in procs]
    for p_ in procs:
        p_.join()
    n = sum(g[0] for g in got)
    dt = max(g[1] for g in got) - t0
    return {"value": n / dt, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} oracle FISTA+DST3 solves of the 2000x10000 workload (lambda/lambda_max cycling "
                      f"0.9..0.1) on {cores} host cores in {dt:.1f} s, one single-threaded oracle process per "
                      f"core, {budget_s:.0f} s budget per core; problem set-up untimed"}


def precision_error(ds, dev, D32, y32, ratio=0.5):
    """Error against the FP64 oracle per result: the 2000 x 10000 workload at lambda =
    ratio lambda_max, FISTA + DST3 to gap 1e-6, from the FP32 master and from the BF16 and
    FP8 working copies; ||x - x_oracle||_inf / ||x_oracle||_inf, the FP64 duality gap of the
    returned x, and the columns read from the copy."""
    import torch
    import oracle
    D, y = D32.astype(np.float64), y32.astype(np.float64)
    lm, _, _ = oracle.lambda_max(D, y)
    lam = ratio * lm
    ref = oracle.solve(D, y, lam, alg="fista", test="dst3", tol=1e-12, max_iter=100000)
    xs = ref["x"]
    ctx = ds.ds_create(dev.index or 0, torch.cuda.current_stream(dev))
    Dt = torch.from_numpy(np.ascontiguousarray(D32.T)).to(dev).t()
    yt = torch.from_numpy(y32).to(dev)
    x = torch.empty(D32.shape[1], device=dev)
    o = ds.ds_options_default(test="dst3", tol_gap_rel=TOL, max_iter=20000)
    out = {"workload": f"2000x10000 (seed 1002), lambda = {ratio} lambda_max, FISTA + DST3 to gap 1e-6; oracle "
                       "FP64 to gap 1e-12", "oracle_iters": ref["iters"]}
    yy = float(y @ y)
    for name, prec in (("fp32", None), ("bf16", ds.DS_BF16), ("fp8", ds.DS_FP8)):
        dct = ds.ds_dict_create(ctx, Dt, work_prec=prec)
        r = ds.ds_solve(ctx, dct, yt, lam, o, x)
        ds.ds_dict_destroy(dct)
        xg = x.double().cpu().numpy()
        res = y - D @ xg
        c = D.T @ res
        v = res * min(1.0 / lam, 1.0 / np.abs(c).max())
        gap = 0.5 * res @ res + lam * np.abs(xg).sum() - (0.5 * yy - 0.5 * lam * lam * np.sum((v - y / lam) ** 2))
        out[name] = {"rel_err_inf": float(np.abs(xg - xs).max() / np.abs(xs).max()),
                     "gap_rel_fp64": float(gap / (0.5 * yy)), "iters": r["iters"],
                     "lowp_columns_fraction": r["cols_lowp"] / max(1, r["cols_corr"])}
    ds.ds_destroy(ctx)
    return out


# ------------------------------------------------------------------------ our arm

def job_throughput(total_ms, solves_per_step, steps, world, dist=None, device="cpu"):
    """Whole-job solves/s when each of `world` ranks ran `steps` steps of `solves_per_step`
    independent solves on its own GPU (weak scaling, no collective on the data path): the
    slowest rank's time, a max over ranks, sets the job's time.  Returns (value, job_ms)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return solves_per_step * steps * world / (total_ms / 1e3), total_ms


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-large", action="store_true", help="skip the 8192x65536 HBM roofline run")
    ap.add_argument("--no-modes", action="store_true", help="skip the batched and served measurements")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--profile-one", action="store_true",
                    help="register the dictionary and run one 5-lambda DST3 path, then exit (profiling)")
    ap.add_argument("--profile-large", action="store_true",
                    help="register a 4096x32768 FP32 dictionary (512 MB > L2) and run one FISTA + DST3 solve, then "
                         "exit (profiling the DRAM traffic of the solve kernel)")
    ap.add_argument("--profile-batch", action="store_true",
                    help="run one 64-rhs multi-RHS batch on the BF16 copy of the dictionary, then exit (profiling)")
    ap.add_argument("--profile-small", action="store_true",
                    help="run the 100x500 FP64 solve (one-cluster kernel) three times, then exit (profiling)")
    ap.add_argument("--group-only", action="store_true",
                    help="the Group-Lasso workload alone (the default run measures it last)")
    ap.add_argument("--paper", action="store_true",
                    help="the paper's screening comparison (no screening / static / dynamic, ISTA / FISTA, "
                         "Pnoise / Gaussian) on the GPU, then exit")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_one:
        profile_one()
        return
    if args.profile_batch:
        profile_batch()
        return
    if args.profile_large:
        profile_large()
        return
    if args.profile_small:
        profile_small()
        return
    if args.paper:
        paper_accounting()
        return
    if args.group_only:
        print(json.dumps(group_measure()))
        return

    import torch
    import paper_1412_4080_gb300 as ds

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        import datetime
        # a lost rank ends the others' next collective within this limit instead of the default 10 min
        dist.init_process_group("nccl", device_id=torch.device("cuda", local), timeout=datetime.timedelta(seconds=300))
    ds.lib()

    D32, y32 = problem()
    N, K = D32.shape
    dev = torch.device("cuda", local)
    Dt = torch.from_numpy(np.ascontiguousarray(D32.T)).to(dev).t()  # column-major (N, K)
    yt = torch.from_numpy(y32).to(dev)
    X = torch.empty((len(RATIOS), K), device=dev)
    flush = torch.empty(64 * 1024 * 1024, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)
    ctx = ds.ds_create(local, stream)
    ratios = np.array(RATIOS)
    opts = {t: ds.ds_options_default(test=t, alg="fista", tol_gap_rel=TOL, max_iter=20000, lambda_rel=1)
            for t in TESTS}

    def step(y=yt, Xo=X, D=Dt):
        dct = ds.ds_dict_create(ctx, D)
        out = []
        for t in TESTS:
            out += ds.ds_solve_path(ctx, dct, y, ratios, opts[t], Xo)
        ds.ds_dict_destroy(dct)
        return out

    for _ in range(args.warmup):
        res = step()
    bad = [r for r in res if r["status"] != 0]
    if bad:
        raise SystemExit(f"solves did not converge: {bad[:2]}")

    launches0 = ds.ds_ctx_kernel_launches(ctx)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_ms = 0.0
    kern_ms = 0.0
    cols = 0
    iters = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            ev0.record(stream)
            res = step()
            ev1.record(stream)
            torch.cuda.synchronize()
            total_ms += ev0.elapsed_time(ev1)
            kern_ms += sum(r["ms"] for r in res)
            cols += sum(r["cols_corr"] + r["cols_synth"] for r in res)
            iters += [r["iters"] for r in res]
    torch.cuda.synchronize()
    launches = ds.ds_ctx_kernel_launches(ctx) - launches0
    if dist:
        dist.barrier()
    solves_per_step = len(TESTS) * len(RATIOS)
    value, total_ms = job_throughput(total_ms, solves_per_step, args.steps, world, dist, dev)

    # roofline of the dominant kernel (the persistent solve kernel): algorithmic bytes =
    # dictionary columns read (correlations + syntheses) x N x 4 bytes
    peak, peak_kind = _peaks()
    bytes_alg = cols * N * 4
    achieved = bytes_alg / (kern_ms / 1e3) / 1e9
    n_launch = args.steps * len(TESTS)
    traffic = _kernel_traffic()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind, "kernel": "solve_kernel<float>",
            "bytes_per_launch": bytes_alg / n_launch, "served_from": "L2",
            "note": "D (80 MB) fits in the 129 MB L2 and stays resident across the iterations of a solve, so "
                    "most algorithmic bytes are L2 hits; frac compares them with the HBM copy peak. "
                    "roofline_large measures D > L2 (8192x65536)"}
    if traffic:
        roof["dram_gbs"] = traffic * n_launch / (kern_ms / 1e3) / 1e9
        roof["dram_frac"] = roof["dram_gbs"] / peak

    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "solves_per_step": solves_per_step, "N": N, "K": K,
                      "l2": "flushed before each timed step (256 MB write)", "parallelism": f"replicas{world}"},
           "roofline": roof, "gpu_launches": launches, "clocks": clk.summary(),
           "iters": {"min": min(iters), "median": statistics.median(iters), "max": max(iters)},
           "solve_kernel_ms_per_step": kern_ms / args.steps}

    # ------------------------------------------------ e2e through the C ABI, host buffers
    Dh = torch.from_numpy(np.asfortranarray(D32).T.copy()).pin_memory()  # (K, N) rows = atoms
    Dh_np = Dh.numpy().T  # Fortran-ordered (N, K) view of pinned memory
    yh = torch.from_numpy(y32.copy()).pin_memory().numpy()
    Xh = torch.empty((len(RATIOS), K), dtype=torch.float32).pin_memory().numpy()
    step(yh, Xh, Dh_np)
    e2e_t = []
    for _ in range(args.e2e_steps):
        t0 = time.perf_counter()
        step(yh, Xh, Dh_np)
        e2e_t.append(time.perf_counter() - t0)
    # whole job: the slowest rank's time, as for the device-timed value (every rank gets here)
    e2e_value = job_throughput(1e3 * sum(e2e_t), solves_per_step, len(e2e_t), world, dist, dev)[0] \
        if e2e_t else None
    out["e2e"] = {"value": e2e_value, "unit": "solves/s",
                  "h2d_bytes_per_step": int(D32.nbytes + len(TESTS) * y32.nbytes),
                  "d2h_bytes_per_step": int(len(TESTS) * Xh.nbytes)}

    # ------------------------------------------------ HBM roofline with D larger than L2
    if not args.no_large:
        out["roofline_large"] = large_roofline(ds, ctx, dev, stream, peak, peak_kind)

    if not args.no_modes:
        # the uneven batch is sharded by instance over the ranks (no collective on the data path)
        out["batched_uneven"] = batched_uneven_measure(ds, ctx, dev, flush, rank, world, dist)
    if world == 1 and not args.no_modes:
        out["batched"] = batched_measure(ds, ctx, D32, dev, flush)
        out["served"] = served_measure(ds, ctx, dev)
    ds.ds_destroy(ctx)
    if world == 1 and not args.no_modes:
        try:
            out["precision_error"] = precision_error(ds, dev, D32, y32)
        except Exception as e:
            out["precision_error"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and not args.no_cpu and world == 1:
        out["cpu_baseline"] = cpu_baseline(D32, y32)
        out["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores()
    if world == 1 and not args.no_modes:
        # last, once every figure above is taken: a failure here is reported in its own entry
        for key, fn in (("group_lasso", group_measure), ("small_fp64_latency", config1_latency),
                        ("group_sizes", lambda: group_size_sweep(ds, dev))):
            try:
                out[key] = fn()
            except Exception as e:
                out[key] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def profile_batch():
    """One launch of the multi-RHS kernel: 64 right-hand sides on the 2000 x 10000 dictionary
    with its BF16 copy (tensor-core bulk phase, FP32 polish), FISTA + DST3 to gap 1e-6."""
    import torch
    import paper_1412_4080_gb300 as ds
    D32, _ = problem()
    g = np.random.default_rng(2002)
    Y, ratios = _rhs_block(D32, 64, g)
    Dt = torch.from_numpy(np.ascontiguousarray(D32.T)).cuda().t()
    ctx = ds.ds_create(0, torch.cuda.current_stream())
    dct = ds.ds_dict_create(ctx, Dt, work_prec=ds.DS_BF16)
    Yt = torch.from_numpy(Y).cuda()
    X = torch.zeros((64, D32.shape[1]), device="cuda")
    opt = ds.ds_options_default(test="dst3", tol_gap_rel=TOL, max_iter=20000, lambda_rel=1)
    plan = ds.ds_batch_create(ctx, [dct], [Yt], [ratios], opt, [X])
    res = ds.ds_batch_run(plan)
    ds.ds_batch_destroy(plan)
    ds.ds_dict_destroy(dct)
    ds.ds_destroy(ctx)
    print(json.dumps({"solves": len(res), "converged": sum(r["status"] == 0 for r in res),
                      "iters_max": max(r["iters"] for r in res), "ms": res[0]["ms"],
                      "cols_corr": sum(r["cols_corr"] for r in res), "cols_lowp": sum(r["cols_lowp"] for r in res)}))


PAPER_RATIOS = (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9)
PAPER_STRATEGIES = (("none", 1), ("dst3", 0), ("safe", 1), ("dst3", 1), ("dome", 1))


def paper_accounting():
    """The comparison of Sec. 4.3-4.5 on the GPU: for a Pnoise and a Gaussian 2000 x 10000
    dictionary, an observation drawn like the atoms (Sec. 4.2), ISTA, FISTA and Chambolle-Pock run for 200
    iterations (the paper's cap) with no screening, static ST3 (Algorithm 1) and dynamic SAFE,
    ST3 and Dome (Algorithm 3), at lambda / lambda_* = 0.1 ... 0.9.  Reported per run: the
    dictionary columns read (correlations + syntheses; 2 N flops each, the paper's flops_D /
    flops_N when divided by the unscreened count) and the kernel time against no screening."""
    import torch
    import gen
    import paper_1412_4080_gb300 as ds
    out = {"workload": "2000x10000, y drawn like the atoms (Sec. 4.2), 200 iterations, FP32", "runs": []}
    ctx = ds.ds_create(0, torch.cuda.current_stream())
    for kind, seed in (("pnoise", 1010), ("gaussian", 1011)):
        g = gen.rng(seed)
        D = gen.pnoise_dict(2000, 10000, g) if kind == "pnoise" else gen.gaussian_dict(2000, 10000, g)
        y = gen.atom_like_y(2000, kind, g)
        Dt = torch.from_numpy(np.ascontiguousarray(D.T.astype(np.float32))).cuda().t()
        yt = torch.from_numpy(y.astype(np.float32)).cuda()
        dct = ds.ds_dict_create(ctx, Dt)
        x = torch.empty(D.shape[1], device="cuda")
        try:
            for alg in ("ista", "fista", "cp"):
                for ratio in PAPER_RATIOS:
                    base = None
                    for test, dyn in PAPER_STRATEGIES:
                        o = ds.ds_options_default(alg=alg, test=test, dynamic=dyn, tol_gap_rel=0.0, max_iter=200,
                                                  lambda_rel=1)
                        ds.ds_solve(ctx, dct, yt, ratio, o, x)  # warm the caches for the timed run
                        r = ds.ds_solve(ctx, dct, yt, ratio, o, x)
                        cols = r["cols_corr"] + r["cols_synth"]
                        if base is None:
                            base = (cols, r["ms"])
                        out["runs"].append({"dict": kind, "alg": alg, "ratio": ratio, "test": test,
                                            "dynamic": dyn, "iters": r["iters"], "n_active": r["n_active"],
                                            "gap_rel": r["gap"] / (0.5 * float(y @ y)), "ms": round(r["ms"], 4),
                                            "flops_ratio": cols / base[0], "time_ratio": r["ms"] / base[1]})
        finally:
            ds.ds_dict_destroy(dct)
    ds.ds_destroy(ctx)
    out["group_sizes"] = group_size_sweep(ds, torch.device("cuda", 0))
    print(json.dumps(out))


GROUP_SIZES = (5, 10, 50, 100)


def group_size_sweep(ds, dev, ratios=(0.3, 0.5, 0.8), iters=200):
    """The paper's Group-Lasso comparison over group sizes (Sec. 4.4): Pnoise 2000 x 10000
    dictionaries with groups of 5, 10, 50 and 100 atoms (w_g = sqrt(size)), groups active with
    probability 0.05, unit-norm y at 20 dB (Sec. 4.2); FISTA for 200 iterations (the paper's
    cap) with no screening, dynamic GSAFE and dynamic DGST3.  Per run: the dictionary columns
    read against no screening (the paper's normalised flops) and the kernel time against no
    screening (its normalised running time)."""
    import torch
    import gen
    ctx = ds.ds_create(dev.index or 0, torch.cuda.current_stream(dev))
    out = {"workload": "Pnoise 2000x10000, groups of 5/10/50/100, Bernoulli(0.05) active groups, unit y at 20 dB, "
                       "FISTA 200 iterations, FP32; entries: flops ratio / time ratio against no screening",
           "runs": []}
    try:
        for gs in GROUP_SIZES:
            D, y, _, goff, w = gen.paper_group_problem(gs, seed=1100 + gs)
            Dt = torch.from_numpy(np.ascontiguousarray(D.T.astype(np.float32))).to(dev).t()
            yt = torch.from_numpy(y.astype(np.float32)).to(dev)
            dct = ds.ds_dict_create(ctx, Dt, goff, w)
            x = torch.empty(D.shape[1], device=dev)
            try:
                for ratio in ratios:
                    base = None
                    for test in ("none", "gsafe", "dgst3"):
                        o = ds.ds_options_default(test=test, tol_gap_rel=0.0, max_iter=iters, lambda_rel=1)
                        ds.ds_solve(ctx, dct, yt, ratio, o, x)  # warm the caches for the timed run
                        r = ds.ds_solve(ctx, dct, yt, ratio, o, x)
                        cols = r["cols_corr"] + r["cols_synth"]
                        if base is None:
                            base = (cols, r["ms"])
                        out["runs"].append({"group_size": gs, "ratio": ratio, "test": test, "n_active": r["n_active"],
                                            "ms": round(r["ms"], 4), "flops_ratio": round(cols / base[0], 4),
                                            "time_ratio": round(r["ms"] / base[1], 4)})
            finally:
                ds.ds_dict_destroy(dct)
            del Dt
    finally:
        ds.ds_destroy(ctx)
    return out


def profile_large(N=4096, K=32768):
    """One solve launch (lambda = 0.5 lambda_max, FISTA + DST3 to gap 1e-6) on an N x K FP32
    Gaussian unit-norm dictionary larger than L2, generated as in large_roofline; prints the
    algorithmic bytes of the launch (columns read x N x 4 B) for the ncu traffic ratio."""
    import torch
    import paper_1412_4080_gb300 as ds
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(1103)
    D = torch.randn((K, N), device=dev, generator=g)
    D /= D.norm(dim=1, keepdim=True)
    x0 = torch.zeros(K, device=dev)
    m = torch.rand(K, device=dev, generator=g) < 0.01
    x0[m] = torch.randn(int(m.sum()), device=dev, generator=g)
    s_ = D.t() @ x0
    e = torch.randn(N, device=dev, generator=g)
    y = s_ + e * (s_.norm() / e.norm()) * 0.1
    ctx = ds.ds_create(0, torch.cuda.current_stream(dev))
    dct = ds.ds_dict_create(ctx, D.t())
    x = torch.empty(K, device=dev)
    o = ds.ds_options_default(test="dst3", tol_gap_rel=TOL, max_iter=20000, lambda_rel=1)
    r = ds.ds_solve(ctx, dct, y, 0.5, o, x)
    ds.ds_dict_destroy(dct)
    ds.ds_destroy(ctx)
    print(json.dumps({"N": N, "K": K, "iters": r["iters"], "status": r["status"], "ms": r["ms"],
                      "algorithmic_bytes": (r["cols_corr"] + r["cols_synth"]) * N * 4}))


def profile_one():
    import torch
    import paper_1412_4080_gb300 as ds
    D32, y32 = problem()
    Dt = torch.from_numpy(np.ascontiguousarray(D32.T)).cuda().t()
    yt = torch.from_numpy(y32).cuda()
    ctx = ds.ds_create(0, torch.cuda.current_stream())
    dct = ds.ds_dict_create(ctx, Dt)
    X = torch.empty((len(RATIOS), D32.shape[1]), device="cuda")
    o = ds.ds_options_default(test="dst3", tol_gap_rel=TOL, max_iter=20000, lambda_rel=1)
    res = ds.ds_solve_path(ctx, dct, yt, np.array(RATIOS), o, X)
    ds.ds_dict_destroy(dct)
    ds.ds_destroy(ctx)
    yy = float(y32.astype(np.float64) @ y32.astype(np.float64))
    print(json.dumps([{**{k: r[k] for k in ("iters", "status", "ms", "n_active", "nnz", "cols_corr", "cols_synth")},
                       "gap_rel": r["gap"] / (0.5 * yy)} for r in res]))


def profile_small(reps=3):
    """The small FP64 case (100 x 500, ISTA + DST3 at 0.5 lambda_max to gap 1e-8) solved `reps` times on
    the one-cluster kernel; prints the iterations and times (profiling)."""
    import torch
    import gen
    import paper_1412_4080_gb300 as ds
    D, y, _ = gen.config1(1001)
    Dt = torch.from_numpy(np.ascontiguousarray(D.T)).cuda().t()
    yt = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    x = torch.empty(D.shape[1], dtype=torch.float64, device="cuda")
    ctx = ds.ds_create(0, torch.cuda.current_stream())
    dct = ds.ds_dict_create(ctx, Dt)
    o = ds.ds_options_default(alg="ista", test="dst3", tol_gap_rel=1e-8, max_iter=100000, lambda_rel=1)
    res = [ds.ds_solve(ctx, dct, yt, 0.5, o, x) for _ in range(reps)]
    ds.ds_dict_destroy(dct)
    ds.ds_destroy(ctx)
    print(json.dumps([{k: r[k] for k in ("iters", "status", "ms", "n_active", "nnz")} for r in res]))


def _rhs_block(D, R, g, lo=0.1, hi=0.9):
    """R right-hand sides y = D x0 + e at 20 dB (x0 Bernoulli(0.01)-Gaussian), lambda/lambda_max ~ U[lo, hi]."""
    N, K = D.shape
    X0 = np.zeros((K, R))
    mask = g.uniform(size=(K, R)) < 0.01
    X0[mask] = g.standard_normal(int(mask.sum()))
    S = D.astype(np.float64) @ X0
    E = g.standard_normal((N, R))
    Y = (S + E * (np.linalg.norm(S, axis=0) / np.maximum(np.linalg.norm(E, axis=0), 1e-300)) * 0.1).T
    # row r = right-hand side r, contiguous: the library reads each y as N consecutive floats
    return np.ascontiguousarray(Y, dtype=np.float32), g.uniform(lo, hi, size=R)


def _time_batch(ds, plan, flush, reps=2):
    import torch
    ds.ds_batch_run(plan)  # warm
    best, res = None, None
    for k in range(reps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        res = ds.ds_batch_run(plan)
        ev1.record()
        torch.cuda.synchronize()
        t = ev0.elapsed_time(ev1) / 1e3
        best = t if best is None else min(best, t)
    return best, res


def batched_measure(ds, ctx, D32, dev, flush):
    """Batching: 64 right-hand sides on the 2000 x 10000 dictionary (Bernoulli(0.01)-Gaussian
    x0, 20 dB, lambda/lambda_max ~ U[0.1, 0.9]), FISTA + DST3 to gap 1e-6.  The batch solves
    the 64 problems as one multi-RHS block (one graph-replayed persistent launch): from the
    FP32 master alone, and with the BF16 working copy whose bulk iterations contract on the
    tensor cores.  The plain form solves the same 64 problems one at a time."""
    import torch
    R = 64
    g = np.random.default_rng(2002)
    N, K = D32.shape
    Y, ratios = _rhs_block(D32, R, g)
    Dt = torch.from_numpy(np.ascontiguousarray(D32.T)).to(dev).t()
    d32 = ds.ds_dict_create(ctx, Dt)
    dbf = ds.ds_dict_create(ctx, Dt, work_prec=ds.DS_BF16)
    Yt = torch.from_numpy(Y).to(dev)
    Xb = torch.zeros((R, K), device=dev)
    opt = ds.ds_options_default(test="dst3", tol_gap_rel=TOL, max_iter=20000, lambda_rel=1)
    out = {}
    for name, dct in (("bf16_tensor", dbf), ("fp32", d32), ("autotuned", dbf)):
        plan = ds.ds_batch_create(ctx, [dct], [Yt], [ratios], opt, [Xb])
        tune = ds.ds_batch_autotune(plan, 5) if name == "autotuned" else None
        t, res = _time_batch(ds, plan, flush)
        out[name] = {"solves_per_s": R / t, "ms": t * 1e3, "layout": ds.ds_batch_layout(plan),
                     "converged": all(r["status"] == 0 for r in res),
                     "iters_median": float(np.median([r["iters"] for r in res])),
                     "iters_max": int(max(r["iters"] for r in res)),
                     "lowp_column_fraction": float(np.mean([r["cols_lowp"] / max(r["cols_corr"], 1) for r in res]))}
        if tune:
            out[name]["tuning"] = tune
        ds.ds_batch_destroy(plan)
    # plain form: one solve at a time, FP32 master
    x1 = torch.zeros(K, device=dev)
    flush.fill_(2.0)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for r in range(R):
        ds.ds_solve(ctx, d32, Yt[r], float(ratios[r]), opt, x1)
    ev1.record()
    torch.cuda.synchronize()
    t_plain = ev0.elapsed_time(ev1) / 1e3
    ds.ds_dict_destroy(d32)
    ds.ds_dict_destroy(dbf)
    best = out["autotuned"]["solves_per_s"]
    return {"value": best, "unit": "solves/s", "plain_value": R / t_plain, "vs_plain": best * t_plain / R,
            "modes": out,
            "workload": "64 rhs x 2000x10000 FP32 Gaussian dictionary (+ BF16 copy), lambda/lambda_max ~ "
                        "U[0.1,0.9], FISTA+DST3, gap 1e-6; multi-RHS blocks in a graph-replayed persistent "
                        "launch (schedule from ds_batch_autotune) vs 64 sequential ds_solve on the FP32 master"}


def uneven_instances(n_inst=256, seed=1004):
    """The uneven batch workload's shapes: instance i has N ~ U{256..4096}, K ~ U{1024..32768},
    64 right-hand sides with lambda/lambda_max ~ U[0.1, 0.9] (host RNG, seeded)."""
    g = np.random.default_rng(seed)
    shapes = [(int(g.integers(256, 4097)), int(g.integers(1024, 32769))) for _ in range(n_inst)]
    lams = [g.uniform(0.1, 0.9, size=64) for _ in range(n_inst)]
    return shapes, lams


def shard(n, rank, world):
    """Instances of rank `rank` out of `world`: every world-th one (no data exchange between ranks)."""
    return list(range(rank, n, world))


def batched_uneven_measure(ds, ctx, dev, flush, rank=0, world=1, dist=None, n_inst=256, team_size=0):
    """The uneven batch workload at its stated size: 256 instances with N ~ U{256..4096},
    K ~ U{1024..32768} (Gaussian unit-norm columns), 64 right-hand sides each (Bernoulli(0.01)-
    Gaussian x0, 20 dB), FP32 master + BF16 working copy, FISTA + DST3 to gap 1e-6, one batch
    plan (persistent launch replayed from a CUDA graph).  With several ranks the instances are
    sharded (rank r takes instances r, r + world, ...), each rank solves its own, and the job's
    time is the slowest rank's.  The plain form is timed on the first right-hand side of every
    instance of the shard, solved one at a time."""
    import torch
    shapes, lams_all = uneven_instances(n_inst)
    mine = shard(n_inst, rank, world)
    dicts, Ys, Xs, lams = [], [], [], []
    for i in mine:
        N, K = shapes[i]
        # generated on the device (seeded per instance): D column-major with unit-norm columns, x0, 20 dB noise
        tg = torch.Generator(device=dev).manual_seed(10040 + i)
        Dt = torch.randn((K, N), device=dev, generator=tg)
        Dt /= Dt.norm(dim=1, keepdim=True)
        Dt = Dt.t()  # (N, K) column-major view
        X0 = torch.randn((64, K), device=dev, generator=tg) * (torch.rand((64, K), device=dev, generator=tg) < 0.01)
        S = X0 @ Dt.t()  # (64, N)
        E = torch.randn((64, N), device=dev, generator=tg)
        Y = S + E * (S.norm(dim=1, keepdim=True) / E.norm(dim=1, keepdim=True)) * 0.1
        dicts.append(ds.ds_dict_create(ctx, Dt, work_prec=ds.DS_BF16))
        Ys.append(Y.contiguous())
        Xs.append(torch.zeros((64, K), device=dev))
        lams.append(lams_all[i])
        del Dt, X0, S, E
    torch.cuda.empty_cache()
    opt = ds.ds_options_default(test="dst3", tol_gap_rel=TOL, max_iter=20000, lambda_rel=1, team_size=team_size)
    plan = ds.ds_batch_create(ctx, dicts, Ys, lams, opt, Xs)
    layout = ds.ds_batch_layout(plan)
    if dist is not None:
        dist.barrier()
    flush.fill_(4.0)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    res = ds.ds_batch_run(plan)
    ev1.record()
    torch.cuda.synchronize()
    t_ms = ev0.elapsed_time(ev1)
    ds.ds_batch_destroy(plan)
    n_mine = 64 * len(mine)
    value, job_ms = job_throughput(t_ms, n_inst * 64 / world, 1, world, dist, dev)
    # plain: the first right-hand side of every instance of the shard, one at a time
    flush.fill_(3.0)
    torch.cuda.synchronize()
    ev0.record()
    for k in range(len(mine)):
        x1 = torch.zeros(Xs[k].shape[1], device=dev)
        ds.ds_solve(ctx, dicts[k], Ys[k][0], float(lams[k][0]), opt, x1)
    ev1.record()
    torch.cuda.synchronize()
    t_plain = ev0.elapsed_time(ev1) / 1e3
    for d in dicts:
        ds.ds_dict_destroy(d)
    del Ys, Xs
    torch.cuda.empty_cache()
    plain = len(mine) / t_plain
    return {"value": value, "unit": "solves/s", "ms": job_ms, "plain_value": plain * world,
            "vs_plain": value / (plain * world), "converged": all(r["status"] == 0 for r in res),
            "not_converged": sum(r["status"] != 0 for r in res), "layout": layout, "solves": n_inst * 64,
            "ranks": world, "solves_this_rank": n_mine, "scaling": "weak" if world == 1 else "strong",
            "sample": f"all {n_inst} instances x 64 rhs ({n_inst * 64} solves), sharded over {world} rank(s); "
                      f"default multi-RHS schedule (tensor-core bulk on the BF16 copy, blocks of 64); plain "
                      f"timed on the first rhs of each instance ({len(mine)} solves on this rank)"}


def ar1_dict_device(N, K, rho, tg, dev, block=64):
    """AR(1) columns along the signal axis (d[0] = e_0, d[n] = rho d[n-1] + sqrt(1 - rho^2) e_n),
    normalised, generated on the device: the recursion over a block of rows is one small
    lower-triangular matrix product (rho^(j-i) weights) plus the carry from the previous block."""
    import torch
    E = torch.randn((N, K), device=dev, generator=tg)
    s = (1.0 - rho * rho) ** 0.5
    j = torch.arange(block, device=dev, dtype=torch.float32)
    Tm = torch.tril(rho ** (j[:, None] - j[None, :]).clamp(min=0)) * s
    carry_w = rho ** (j + 1)
    D = torch.empty_like(E)
    D[0] = E[0]
    n0 = 1
    while n0 < N:
        b = min(block, N - n0)
        D[n0:n0 + b] = Tm[:b, :b] @ E[n0:n0 + b] + carry_w[:b, None] * D[n0 - 1][None, :]
        n0 += b
    del E
    D /= D.norm(dim=0, keepdim=True)
    return D


def _serve_stream(ds, ctx, pool, opts, team_size, seconds, rate, drain_s, budget_gib):
    """One open-loop Poisson stream through a server with teams of team_size CTAs (see served_measure)."""
    import time
    g = np.random.default_rng(2007)
    server = ds.ds_server_create(ctx, budget_gib << 30, 8192, 65536, team_size)
    N, K, lasso, group, Ys = pool[0]  # warm the server (kernel load, first launch)
    xw = np.zeros(K, dtype=np.float32)
    tw = ds.ds_server_submit(server, lasso, Ys["lasso"][0], 0.9, opts["lasso"], xw)
    while ds.ds_server_poll(server, tw) is None:
        time.sleep(0.001)
    arrivals = np.cumsum(g.exponential(1.0 / rate, size=int(rate * seconds * 1.5)))
    arrivals = arrivals[arrivals < seconds]
    outstanding, lat, keep, kinds = {}, [], [], {"lasso": 0, "group": 0}
    t0 = time.perf_counter()
    i = 0
    while i < len(arrivals) or outstanding:
        now = time.perf_counter() - t0
        if now > seconds + drain_s:
            break  # saturated: what is still outstanding is reported, not hidden
        while i < len(arrivals) and arrivals[i] <= now:
            N, K, lasso, group, Ys = pool[g.integers(len(pool))]
            kind = "group" if g.uniform() < 0.2 else "lasso"
            x = np.zeros(K, dtype=np.float32)
            t = ds.ds_server_submit(server, group if kind == "group" else lasso,
                                    Ys[kind][g.integers(Ys[kind].shape[0])], float(g.uniform(0.1, 0.9)),
                                    opts[kind], x)
            outstanding[t] = (x, kind)
            i += 1
        for t in list(outstanding):
            r = ds.ds_server_poll(server, t)
            if r is not None:
                lat.append(r["ms"])
                keep.append(r["status"])
                kinds[outstanding[t][1]] += 1
                del outstanding[t]
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    unfinished = len(outstanding)
    st = ds.ds_server_stats(server)
    ds.ds_server_destroy(server)
    outstanding.clear()
    lat_a = np.array(lat) if lat else np.array([float("nan")])
    return {"team_size": team_size, "submitted": int(len(arrivals)), "completed": int(len(keep)),
            "completed_by_kind": kinds, "unfinished_at_deadline": unfinished, "wall_s": wall,
            "solves_per_s": len(keep) / wall, "p50_ms": float(np.percentile(lat_a, 50)),
            "p99_ms": float(np.percentile(lat_a, 99)), "converged": int(sum(1 for s_ in keep if s_ == 0)),
            "kernel_launches": st["launches"]}


def _serve_closed(ds, ctx, pool, opts, team_size, reqs, budget_gib):
    """A fixed set of requests submitted at once and drained completely through a server with teams of
    team_size CTAs; returns the wall time and the results."""
    import time
    server = ds.ds_server_create(ctx, budget_gib << 30, 8192, 65536, team_size)
    N, K, lasso, group, Ys = pool[0]  # warm the server (kernel load, first launch)
    xw = np.zeros(K, dtype=np.float32)
    tw = ds.ds_server_submit(server, lasso, Ys["lasso"][0], 0.9, opts["lasso"], xw)
    while ds.ds_server_poll(server, tw) is None:
        time.sleep(0.001)
    outs, res = {}, []
    t0 = time.perf_counter()
    for (pi, kind, yi, ratio) in reqs:
        N, K, lasso, group, Ys = pool[pi]
        x = np.zeros(K, dtype=np.float32)
        t = ds.ds_server_submit(server, group if kind == "group" else lasso, Ys[kind][yi], ratio, opts[kind], x)
        outs[t] = x
    while outs:
        for t in list(outs):
            r = ds.ds_server_poll(server, t)
            if r is not None:
                res.append(r)
                del outs[t]
        time.sleep(0.0005)
    wall = time.perf_counter() - t0
    ds.ds_server_destroy(server)
    return wall, res


def served_measure(ds, ctx, dev, seconds=5.0, rate=2000.0, drain_s=10.0, plain_n=8, team_sizes=(38,), n_pool=32,
                   budget_gib=8, closed_n=48, closed_team_sizes=(19, 38, 76)):
    """The served mixed stream at its stated shapes: a pool of n_pool AR(1) dictionaries (rho = 0.9,
    unit-norm columns) with N ~ U{512..8192} and K ~ U{4096..65536} (K a multiple of 8), each
    registered twice (Lasso, and Group-Lasso with groups of 8) with an FP8 e4m3 working copy
    (scale per column) next to the FP32 master; open-loop Poisson arrivals at `rate` req/s for
    `seconds`, 80% Lasso / 20% Group-Lasso, each request drawing a pool dictionary and one of
    its observations (1% active atoms or groups, 20 dB) and lambda/lambda_max ~ U[0.1, 0.9],
    gap 1e-6; HBM-budget admission.  Requests still unfinished `drain_s` after the window are
    counted, not hidden.  The plain form solves plain_n requests of the same mix one at a time."""
    import time
    import torch
    g = np.random.default_rng(2005)
    tg = torch.Generator(device=dev).manual_seed(2005)
    pool = []
    t_reg = time.perf_counter()
    for _ in range(n_pool):
        N = int(g.integers(512, 8193))
        K = int(g.integers(4096, 65537)) // 8 * 8
        D = ar1_dict_device(N, K, 0.9, tg, dev)
        Dc = D.t().contiguous().t()  # column-major
        del D
        lasso = ds.ds_dict_create(ctx, Dc, work_prec=ds.DS_FP8)
        goff = np.arange(0, K + 1, 8, dtype=np.int64)
        group = ds.ds_dict_create(ctx, Dc, goff, work_prec=ds.DS_FP8)
        B = 8  # observations per dictionary: 1% active atoms (Lasso) / groups (Group-Lasso), 20 dB
        Ys = {}
        for kind in ("lasso", "group"):
            if kind == "lasso":
                X0 = torch.randn((K, B), device=dev, generator=tg) * (
                    torch.rand((K, B), device=dev, generator=tg) < 0.01)
            else:
                act = (torch.rand((K // 8, B), device=dev, generator=tg) < 0.01).repeat_interleave(8, dim=0)
                X0 = torch.randn((K, B), device=dev, generator=tg) * act
            S = Dc @ X0
            Nz = torch.randn(S.shape, device=dev, generator=tg)
            Ys[kind] = (S + Nz * (S.norm(dim=0) / Nz.norm(dim=0).clamp(min=1e-30)) * 0.1).t().contiguous().cpu().numpy()
        pool.append((N, K, lasso, group, Ys))
        del Dc
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    reg_s = time.perf_counter() - t_reg
    opts = {"lasso": ds.ds_options_default(test="dst3", tol_gap_rel=TOL, max_iter=20000, lambda_rel=1),
            "group": ds.ds_options_default(test="dgst3", tol_gap_rel=TOL, max_iter=20000, lambda_rel=1)}
    runs = {}
    for team_size in team_sizes:
        runs[team_size] = _serve_stream(ds, ctx, pool, opts, team_size, seconds, rate, drain_s, budget_gib)
    best_ts = max(runs, key=lambda k: runs[k]["completed"] / runs[k]["wall_s"])
    best = runs[best_ts]
    # like for like: one fixed set of closed_n requests of the same mix, drained completely through the
    # server and solved one at a time by ds_solve (the plain form) -- the open stream above cannot drain
    # at 2000 req/s, and its completions favour the short requests
    gc = np.random.default_rng(2008)
    reqs = []
    for _ in range(closed_n):
        pi = int(gc.integers(len(pool)))
        kind = "group" if gc.uniform() < 0.2 else "lasso"
        reqs.append((pi, kind, int(gc.integers(pool[pi][4][kind].shape[0])), float(gc.uniform(0.1, 0.9))))
    closed = {}
    for ts in closed_team_sizes:
        w_, r_ = _serve_closed(ds, ctx, pool, opts, ts, reqs, budget_gib)
        closed[ts] = {"wall_s": w_, "solves_per_s": closed_n / w_,
                      "converged": sum(1 for q in r_ if q["status"] == 0)}
    torch.cuda.synchronize()
    tq0 = time.perf_counter()
    for (pi, kind, yi, ratio) in reqs:
        N, K, lasso, group, Ys = pool[pi]
        yd = torch.from_numpy(Ys[kind][yi].copy()).to(dev)
        xd = torch.zeros(K, device=dev)
        ds.ds_solve(ctx, group if kind == "group" else lasso, yd, ratio, opts[kind], xd)
    torch.cuda.synchronize()
    closed_plain = closed_n / (time.perf_counter() - tq0)
    best_closed = max(closed, key=lambda k: closed[k]["solves_per_s"])
    # plain form: requests of the same mix, one at a time (the whole GPU per solve)
    gp = np.random.default_rng(2006)
    torch.cuda.synchronize()
    tp0 = time.perf_counter()
    for _ in range(plain_n):
        N, K, lasso, group, Ys = pool[gp.integers(len(pool))]
        kind = "group" if gp.uniform() < 0.2 else "lasso"
        yd = torch.from_numpy(Ys[kind][gp.integers(Ys[kind].shape[0])].copy()).to(dev)
        xd = torch.zeros(K, device=dev)
        ds.ds_solve(ctx, group if kind == "group" else lasso, yd, float(gp.uniform(0.1, 0.9)), opts[kind], xd)
    torch.cuda.synchronize()
    plain = plain_n / (time.perf_counter() - tp0)
    shapes = [(p_[0], p_[1]) for p_ in pool]
    for (_, _, lasso, group, _) in pool:
        ds.ds_dict_destroy(lasso)
        ds.ds_dict_destroy(group)
    torch.cuda.empty_cache()
    return {"value": closed[best_closed]["solves_per_s"], "unit": "solves/s", "plain_value": closed_plain,
            "vs_plain": closed[best_closed]["solves_per_s"] / closed_plain,
            "closed_set": {"requests": closed_n, "team_size": best_closed,
                           "by_team_size": {str(k): {kk: round(vv, 4) for kk, vv in v.items()} for k, v in
                                            closed.items()},
                           "note": "value / plain_value: the same requests drained through the server and "
                                   "solved one at a time"},
            "stream": {"solves_per_s": best["solves_per_s"], "plain_sample_solves_per_s": plain,
                       "note": "open-loop stream at the offered rate: completions within the window, which "
                               "favour short requests; latency from submission"},
            "offered_rate": rate, "window_s": seconds, "drain_s": drain_s,
            **{k: best[k] for k in ("team_size", "submitted", "completed", "completed_by_kind",
                                    "unfinished_at_deadline", "wall_s", "p50_ms", "p99_ms", "converged",
                                    "kernel_launches")},
            "team_sizes_tried": {str(k): round(v["solves_per_s"], 3) for k, v in runs.items()},
            "registration_s": reg_s, "pool_elements_mean": float(np.mean([a * b for a, b in shapes])),
            "workload": f"Poisson arrivals at {rate:.0f} req/s for {seconds:.0f} s (then {drain_s:.0f} s to drain), "
                        f"80% Lasso / 20% Group-Lasso (groups of 8), pool of {n_pool} AR(1) rho=0.9 dictionaries "
                        "N ~ U{512..8192}, K ~ U{4096..65536}, lambda/lambda_max ~ U[0.1,0.9], FP8 e4m3 copy with "
                        "per-column scale + FP32 master, gap 1e-6, FISTA + DST3/DGST3, "
                        f"{budget_gib} GiB pool; saturated: throughput is completions / wall time, the best of the "
                        f"team sizes tried; plain: {plain_n} requests of the same mix solved one at a time"}


GROUP_RATIOS = (0.2, 0.5, 0.8)
GROUP_TESTS = ("gsafe", "dgst3")


def config1_latency(reps=10, warmup=3):
    """Latency of the small FP64 case (100 x 500 Gaussian unit-norm D, 10 nonzeros, sigma 0.01,
    seed 1001): ISTA + dynamic DST3 at lambda = 0.5 lambda_max to gap 1e-8 * 1/2 ||y||^2, one
    ds_solve at a time, CUDA events on the library's stream (D fits in cache: no flush).
    team_size 0 takes the one-cluster solve (4 CTAs for this size); team_size > 0 the grid kernel."""
    import torch
    import gen
    import paper_1412_4080_gb300 as ds
    D, y, _ = gen.config1(1001)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    Dt = torch.from_numpy(np.ascontiguousarray(D.T)).to(dev).t()  # column-major (N, K), FP64
    yt = torch.from_numpy(np.ascontiguousarray(y)).to(dev)
    x = torch.empty(D.shape[1], dtype=torch.float64, device=dev)
    ctx = ds.ds_create(0, stream)
    dct = ds.ds_dict_create(ctx, Dt)
    def timed(team_size):
        o = ds.ds_options_default(alg="ista", test="dst3", tol_gap_rel=1e-8, max_iter=100000, lambda_rel=1,
                                  team_size=team_size)
        for _ in range(warmup):
            ds.ds_solve(ctx, dct, yt, 0.5, o, x)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, res = [], []
        for _ in range(reps):
            torch.cuda.synchronize()
            ev0.record(stream)
            res.append(ds.ds_solve(ctx, dct, yt, 0.5, o, x))
            ev1.record(stream)
            torch.cuda.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        return ms, res

    ms, res = timed(0)  # the grid the library picks for this size
    by_grid = {str(gsz): round(statistics.median(timed(gsz)[0]), 4) for gsz in (1, 4, 152)}
    ds.ds_dict_destroy(dct)
    ds.ds_destroy(ctx)
    return {"median_ms": statistics.median(ms), "min_ms": min(ms), "iters": res[-1]["iters"],
            "path": "one thread-block cluster (the dictionary in shared memory as float-float pairs)",
            "median_ms_by_grid_ctas": by_grid,
            "converged": all(r["status"] == 0 for r in res),
            "workload": "100x500 FP64 Gaussian, 10 nonzeros, sigma 0.01 (seed 1001), ISTA + dynamic DST3, "
                        "lambda = 0.5 lambda_max, gap 1e-8; one solve per call"}


def group_measure(steps=3, warmup=3):
    """The Group-Lasso workload (2000 x 10000 Gaussian unit-norm D, contiguous groups of 10 with
    w_g = sqrt(10), 10 active groups of N(0,1) entries, 20 dB, seed 1003): FISTA with dynamic
    GSAFE and DGST3 at lambda / lambda_max in {0.2, 0.5, 0.8}, each to gap 1e-6 * 1/2 ||y||^2.
    A step is the 6 solves, timed with CUDA events on the library's stream after an L2 flush;
    the dictionary precompute (norms, group spectral norms, Lanczos) is timed apart."""
    import torch
    import gen
    import paper_1412_4080_gb300 as ds
    D, y, _, goff, w = gen.config3(1003)
    D32, y32 = D.astype(np.float32), y.astype(np.float32)
    N, K = D32.shape
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    Dt = torch.from_numpy(np.ascontiguousarray(D32.T)).to(dev).t()  # column-major (N, K)
    yt = torch.from_numpy(y32).to(dev)
    x = torch.empty(K, device=dev)
    flush = torch.empty(64 * 1024 * 1024, device=dev)  # 256 MB > L2
    ctx = ds.ds_create(0, stream)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    dct = ds.ds_dict_create(ctx, Dt, goff, w)
    ev1.record(stream)
    torch.cuda.synchronize()
    pre_ms = ev0.elapsed_time(ev1)
    opts = {t: ds.ds_options_default(test=t, alg="fista", tol_gap_rel=TOL, max_iter=20000, lambda_rel=1)
            for t in GROUP_TESTS}

    def step():
        return [ds.ds_solve(ctx, dct, yt, r, opts[t], x) for t in GROUP_TESTS for r in GROUP_RATIOS]

    for _ in range(warmup):
        step()
    total_ms, kern_ms, cols, res = 0.0, 0.0, 0, []
    for k in range(steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        ev0.record(stream)
        rs = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        total_ms += ev0.elapsed_time(ev1)
        kern_ms += sum(r["ms"] for r in rs)
        cols += sum(r["cols_corr"] + r["cols_synth"] for r in rs)
        res += rs
    ds.ds_dict_destroy(dct)
    ds.ds_destroy(ctx)
    peak, peak_kind = _peaks()
    achieved = cols * N * 4 / (kern_ms / 1e3) / 1e9
    n = len(GROUP_TESTS) * len(GROUP_RATIOS) * steps
    return {"value": n / (total_ms / 1e3), "unit": "solves/s", "ms_per_step": total_ms / steps,
                      "steps": steps, "warmup": warmup, "precompute_ms": pre_ms,
                      "converged": all(r["status"] == 0 for r in res),
                      "iters": {"min": min(r["iters"] for r in res), "max": max(r["iters"] for r in res)},
                      "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                   "frac": achieved / peak, "peak_kind": peak_kind},
                      "workload": "Group-Lasso 2000x10000 Gaussian, groups of 10, w_g = sqrt(10), 10 active groups, "
                                  "20 dB (seed 1003), FISTA + dynamic GSAFE/DGST3, lambda/lambda_max in "
                                  "{0.2,0.5,0.8}, gap 1e-6; L2 flushed before each step; precompute timed apart"}


def large_roofline(ds, ctx, dev, stream, peak, peak_kind, repeats=5, N=8192, K=65536):
    """Solves (lambda = 0.5 lambda_max, the median of `repeats` timed runs after a warm-up)
    on an 8192 x 65536 FP32 Gaussian unit-norm dictionary (2.1 GB > L2): algorithmic GB/s
    of the solve kernel, from the FP32 master and from the BF16 / FP8 working copies."""
    import torch
    g = torch.Generator(device=dev).manual_seed(1102)
    D = torch.randn((K, N), device=dev, generator=g)
    D /= D.norm(dim=1, keepdim=True)
    x0 = torch.zeros(K, device=dev)
    m = torch.rand(K, device=dev, generator=g) < 0.01
    x0[m] = torch.randn(int(m.sum()), device=dev, generator=g)
    s = D.t() @ x0
    e = torch.randn(N, device=dev, generator=g)
    y = s + e * (s.norm() / e.norm()) * 0.1
    Dt = D.t()  # column-major (N, K)
    x = torch.empty(K, device=dev)
    o = ds.ds_options_default(test="dst3", tol_gap_rel=TOL, max_iter=20000, lambda_rel=1)
    out = {}
    for name, prec, es in (("fp32", None, 4), ("bf16", ds.DS_BF16, 2), ("fp8", ds.DS_FP8, 1)):
        dct = ds.ds_dict_create(ctx, Dt, work_prec=prec)
        ds.ds_solve_path(ctx, dct, y, np.array([0.5]), o, x)  # warm
        runs = [ds.ds_solve_path(ctx, dct, y, np.array([0.5]), o, x)[0] for _ in range(repeats)]
        ds.ds_dict_destroy(dct)
        r = runs[0]
        ms = statistics.median(q["ms"] for q in runs)
        # algorithmic bytes: FP32 columns at 4 B/entry, copy columns at 2 or 1 B/entry
        byt = ((r["cols_corr"] - r["cols_lowp"] + r["cols_synth"]) * 4 + r["cols_lowp"] * es) * N
        gbs = byt / (ms / 1e3) / 1e9
        out[name] = {"achieved": gbs, "frac": gbs / peak, "iters": r["iters"], "kernel_ms": ms,
                     "kernel_ms_all": [round(q["ms"], 4) for q in runs], "bytes_per_launch": byt,
                     "lowp_columns_fraction": r["cols_lowp"] / max(1, r["cols_corr"]), "status": r["status"]}
    del D, Dt
    torch.cuda.empty_cache()
    f = out["fp32"]
    # DRAM traffic: ncu's dram bytes per algorithmic byte on a 4096 x 32768 launch (512 MB > L2),
    # scaled to this launch's algorithmic bytes (the traffic of a column stream grows with it)
    ratio = _kernel_traffic("solve_kernel_large.md", "dram_bytes_per_algorithmic_byte:")
    return {"bound": "hbm", "achieved": f["achieved"], "peak": peak, "unit": "GB/s", "frac": f["frac"],
            "peak_kind": peak_kind, "traffic": ratio * f["bytes_per_launch"] if ratio else None,
            "traffic_source": "ncu dram__bytes_read+write on 4096x32768, per algorithmic byte, scaled",
            "workload": "8192x65536 FP32 Gaussian, FISTA+DST3, lambda = 0.5 lambda_max, gap 1e-6",
            "iters": f["iters"], "kernel_ms": f["kernel_ms"], "repeats": repeats, "timing": "median of repeats",
            "precision_variant": {k: out[k] for k in ("bf16", "fp8")}}


if __name__ == "__main__":
    main()
