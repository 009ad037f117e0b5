/*
 * dscreen.h -- C ABI of a GB300 (sm_103a) solver for the Lasso and the
 * Group-Lasso with dynamic screening (Bonnefoy, Emiya, Ralaivola, Gribonval,
 * "Dynamic Screening: Accelerating First-Order Algorithms for the Lasso and
 * Group-Lasso", arXiv 1412.4080).
 *
 * Problem (eq. 1):   x~ = argmin_x 1/2 ||D x - y||_2^2 + lambda * Omega(x)
 *   Lasso (eq. lasso):              Omega(x) = ||x||_1
 *   Group-Lasso (eq. group-lasso):  Omega(x) = sum_g w_g ||x_g||_2, G a partition
 * D is N x K, y has N entries.  The solver runs ISTA, FISTA or Chambolle-Pock
 * (Table 1) and, inside every iteration, a safe screening test (Lemmas 2-7,
 * dual scaling by Lemma 8) that removes atoms from the working dictionary
 * (Algorithm 3).
 *
 * Conventions shared by every call:
 *  - Layout: D is column-major (atom i is the contiguous column D[:, i]),
 *    with leading dimension ld >= N elements.  Vectors are contiguous.
 *  - Element type: the dictionary's dtype (DS_FP32 -> float, DS_FP64 ->
 *    double) is also the type of y, x0 and x_out.
 *  - Pointers may be host or device memory; the library detects which with
 *    cudaPointerGetAttributes and copies host data itself (pinned host
 *    memory is fastest).  The caller owns every buffer it passes in and may
 *    free it when the call returns (ds_dict_create copies D).
 *  - Every call is ordered on the context's CUDA stream and returns when its
 *    results are in the caller's buffers (synchronous), except where noted.
 *  - Errors are returned as ds_status codes; nothing is thrown across the
 *    ABI.  A failed call leaves its outputs unspecified.
 *  - Not thread-safe per context: one call at a time on a given ds_ctx.
 */
#ifndef DSCREEN_H
#define DSCREEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ds_ctx ds_ctx;
typedef struct ds_dict ds_dict;

typedef enum {
    DS_OK = 0,
    DS_ERR_INVALID = 1,       /* bad argument: null pointer, N/K <= 0, lambda <= 0, bad groups ... */
    DS_ERR_OOM = 2,           /* device or pinned allocation failed */
    DS_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    DS_ERR_TIMEOUT = 4,       /* a bounded device-side wait (grid barrier) gave up */
    DS_ERR_NOT_CONVERGED = 5, /* (ds_result.status only) max_iter reached above the gap tolerance */
    DS_ERR_UNSUPPORTED = 6,   /* valid request outside what this build handles (e.g. N too large) */
    DS_PENDING = 7            /* (ds_server_poll only) the request has not completed yet */
} ds_status;

/* Table 1 rows: ISTA, FISTA, Chambolle-Pock, SpaRSA (ISTA with the Barzilai-Borwein step
 * and its nonmonotone acceptance test) and TwIST (two-step shrinkage, monotone variant). */
typedef enum { DS_ISTA = 0, DS_FISTA = 1, DS_CP = 2, DS_SPARSA = 3, DS_TWIST = 4 } ds_alg;

typedef enum {
    DS_TEST_NONE = 0,
    DS_SAFE = 1,  /* Lemma 2 (Lasso) */
    DS_DST3 = 2,  /* Lemma 3 (Lasso) */
    DS_DOME = 3,  /* Lemma 4 (Lasso), dynamic form of the dome maximum */
    DS_GSAFE = 4, /* Lemma 5 (Group-Lasso; on a Lasso dictionary: singleton groups) */
    DS_DGST3 = 5  /* Lemma 6 (Group-Lasso; on a Lasso dictionary: singleton groups) */
} ds_test;

typedef enum { DS_FP64 = 0, DS_FP32 = 1, DS_BF16 = 2, DS_FP8 = 3 } ds_prec;

typedef struct {
    int alg;            /* ds_alg */
    int test;           /* ds_test */
    int dynamic;        /* 1: test at every iteration (Algorithm 3); 0: once at theta = -y (Algorithm 1) */
    int max_iter;       /* iteration cap (>= 1) */
    double tol_gap_rel; /* stop when gap <= tol * 1/2 ||y||^2; 0 runs exactly max_iter iterations */
    double L;           /* step constant; <= 0 uses the dictionary's ||D||_2^2 upper estimate */
    int lambda_rel;     /* 1: lambda values are fractions of lambda_max (computed in the call) */
    double lowp_switch; /* dictionaries with a BF16/FP8 copy: relative nominal gap at which a solve leaves
                           the copy for the FP32 master, restarting FISTA from the bulk iterate (also left
                           after 25 iterations without 1% progress); <= 0: 1e-3, or the gap tolerance if
                           that is coarser */
    int batch_multi_rhs; /* batches: 1 (default) solves the right-hand sides of an FP32 Lasso instance
                            together, up to 64 per block, so each dictionary column read serves them all;
                            0 runs every (instance, rhs) problem on its own */
    int warm_start;      /* ds_solve_path: 1 starts each lambda from the previous lambda's solution (a
                            regularization path; the screening tests of each lambda stay those of its own
                            dual problem, so they remain safe); 0 (default) starts every lambda from x0 */
    double cp_tau;       /* DS_CP (Table 1): tau_0 and sigma_0 of the primal and dual steps (<= 0: 0.99 / sqrt(L)
                            each, so that tau_0 sigma_0 ||D||^2 < 1); the dual iterate starts at 0 */
    double cp_sigma;
    double cp_gamma;     /* DS_CP: gamma >= 0 of phi_t = 1 / sqrt(1 + 2 gamma tau_{t-1}); 0 (default) keeps
                            phi_t = 1 (the Lasso's penalty is not strongly convex: a positive gamma drives
                            tau_t to 0) */
    int step_backtracking; /* DS_ISTA / DS_FISTA: 1 sets L_t by backtracking (Beck-Teboulle, the rule Table 1
                              cites): starting from bt_L0, L is doubled until ||D (x_t - u)||^2 <= L ||x_t - u||^2
                              (the quadratic upper model of the loss); 0 (default) keeps the fixed L */
    double bt_L0;          /* first L of the backtracking (<= 0: 1) */
    double twist_xi1;      /* DS_TWIST: lower bound xi_1 of the eigenvalues of D^T D / L that sets TwIST's
                              alpha = rho^2 + 1, beta = 2 alpha / (1 + xi_1), rho = (1 - sqrt(xi_1)) /
                              (1 + sqrt(xi_1)) (<= 0: 1e-4) */
    int gap_every;         /* the stopping rule (duality gap) is evaluated every gap_every iterations
                              (<= 1: every iteration) */
    int team_size;         /* CTAs that run one solve: ds_solve / ds_solve_path (0: one per SM, except
                              that a small FP64 Lasso problem -- N <= 256, K <= 2048, ISTA or FISTA at
                              a fixed step, one lambda, no history -- runs on one thread-block cluster
                              of 2 to 8 CTAs holding the dictionary in shared memory) and the multi-RHS
                              blocks of batches (0: automatic); > 0 always runs the grid of that size */
} ds_options;

typedef struct {
    int iters;          /* iterations run */
    int status;         /* DS_OK, DS_ERR_NOT_CONVERGED or DS_ERR_TIMEOUT */
    int64_t n_active;   /* atoms not screened at exit */
    int64_t nnz;        /* nonzeros of the returned x */
    double gap;         /* P(x) - Dual(mu theta) at exit (absolute) */
    double primal;      /* P(x) */
    double dual;        /* Dual(mu theta) */
    double lambda;      /* absolute lambda used */
    double lambda_max;  /* lambda_* (Sec. 2.2.2 / eq. gstar) */
    double ms;          /* device time of the solve kernel, milliseconds (path: shared equally) */
    int64_t cols_corr;  /* dictionary columns read by correlations D_A^T theta (incl. D^T y, D^T n) */
    int64_t cols_synth; /* dictionary columns read by the sparse syntheses D_A u, D_A x */
    int64_t cols_lowp;  /* of cols_corr, the columns read from the BF16/FP8 working copy */
} ds_result;

/* Human-readable name of a status code (static string, never NULL). */
const char* ds_status_str(ds_status s);

/* Fill *opt with defaults: FISTA, DST3, dynamic, max_iter 10000, tol 1e-6,
 * L from the dictionary, absolute lambda, fixed step, gap checked every
 * iteration, automatic team size.  DS_ERR_INVALID if opt is NULL. */
ds_status ds_options_default(ds_options* opt);

/* Create a context on CUDA device `device`, ordered on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The context owns the
 * solver workspaces (grown on demand).  Errors: DS_ERR_INVALID (out == NULL or
 * no such device), DS_ERR_CUDA. */
ds_status ds_create(int device, void* cuda_stream, ds_ctx** out);

/* Release a context and its workspaces (NULL is a no-op). */
ds_status ds_destroy(ds_ctx* ctx);

/* Register a dictionary D (N x K, column-major, leading dimension ld >= N,
 * element type dtype = DS_FP32 or DS_FP64; host or device pointer).  The
 * library copies D into a zero-padded device copy (16-byte aligned columns)
 * and precomputes what does not depend on y or lambda (the Sec. 4.1 remark
 * that the group norms ||D_g|| depend on the dictionary only):
 *   - column norms ||d_i||;
 *   - L = an upper estimate of ||D||_2^2 (Lanczos on D D^T with a residual bound);
 *   - for Group-Lasso, ||D_g||_2 of every group (Gram matrix + Jacobi,
 *     rounded up), used by Lemmas 5-7.
 * Groups (eq. group-lasso): group_offsets (host, n_groups + 1 entries,
 * 0 = off_0 < off_1 < ... < off_G = K) lists contiguous column ranges; weights
 * (host, n_groups entries, > 0; NULL = sqrt(group size)).  group_offsets NULL
 * = the Lasso.  Group sizes are limited to 128 columns (DS_ERR_UNSUPPORTED).
 * work_prec: dtype, or (FP32 dictionaries) DS_BF16 / DS_FP8 for the precision
 * variant: the library also keeps a BF16 copy or an FP8 e4m3 copy with one
 * scale per column (max|d_i| / 448) and the exact error norms ||d_i - copy_i||;
 * solves then run their bulk iterations on the copy (2 or 1 bytes per entry),
 * with every screening radius inflated by the copy's error bound so the tests
 * stay safe, and finish with FP32 iterations on the surviving atoms.
 * Errors: DS_ERR_INVALID,
 * DS_ERR_UNSUPPORTED (N > the shared-memory limit, group > 128, work_prec),
 * DS_ERR_OOM, DS_ERR_CUDA, DS_ERR_TIMEOUT. */
ds_status ds_dict_create(ds_ctx* ctx, const void* D, int64_t N, int64_t K, int64_t ld, ds_prec dtype,
                         const int64_t* group_offsets, const double* weights, int64_t n_groups,
                         ds_prec work_prec, ds_dict** out);

/* Release a dictionary (NULL is a no-op). */
ds_status ds_dict_destroy(ds_dict* dict);

/* Read back the dictionary's step constant L (>= ||D||_2^2 estimate).
 * Errors: DS_ERR_INVALID (NULL dict or L). */
ds_status ds_dict_lipschitz(const ds_dict* dict, double* L);

/* lambda_* of y (Sec. 2.2.2: ||D^T y||_inf; eq. gstar: max_g ||D_g^T y|| / w_g)
 * computed on the device with compensated FP32 (or FP64) dot products.
 * y: N elements of the dictionary's type, host or device.  Errors:
 * DS_ERR_INVALID, DS_ERR_CUDA, DS_ERR_TIMEOUT. */
ds_status ds_lambda_max(ds_ctx* ctx, const ds_dict* dict, const void* y, double* lambda_max);

/* Solve eq. (1) for one y and one lambda > 0 with dynamic (or static)
 * screening; one persistent cooperative kernel runs the whole solve.
 * x0 (nullable, K elements): warm start.  x_out: K elements.  res (host):
 * iterations, gap, status, ...  lambda >= lambda_max returns x = 0 with 0
 * iterations.  The call returns DS_OK when the solve ran (res->status tells
 * whether the gap tolerance was met).  Errors: DS_ERR_INVALID (null y/x_out/
 * opt/res, lambda <= 0, max_iter < 1, test not valid for the dictionary),
 * DS_ERR_OOM, DS_ERR_CUDA, DS_ERR_TIMEOUT. */
ds_status ds_solve(ds_ctx* ctx, const ds_dict* dict, const void* y, double lambda, const ds_options* opt,
                   const void* x0, void* x_out, ds_result* res);

/* Same as ds_solve for n_lambda values of lambda sharing one y (the precompute
 * of D^T y, lambda_* and the test centres runs once).  lambdas: host array
 * (absolute, or fractions of lambda_max when opt->lambda_rel).  X_out: K x
 * n_lambda, column j = solution for lambdas[j].  res: n_lambda entries.
 * Errors: those of ds_solve, and DS_ERR_INVALID for n_lambda < 1, a NULL
 * lambdas array or a lambda that is not finite and positive. */
ds_status ds_solve_path(ds_ctx* ctx, const ds_dict* dict, const void* y, int n_lambda, const double* lambdas,
                        const ds_options* opt, const void* x0, void* X_out, ds_result* res);

/* ----------------------------------------------------------------- batches
 * Many solves in one persistent launch.  n instances; instance i has a
 * registered dictionary dicts[i] (all of one dtype, on this context),
 * n_rhs[i] right-hand sides Y[i] (device, N_i x n_rhs[i], column r contiguous)
 * and one lambda per right-hand side lambdas[i][r] (host; absolute, or
 * fractions of each y's lambda_max when opt->lambda_rel).  Solutions go to
 * X_out[i] (device, K_i x n_rhs[i]).  Every (instance, rhs) pair is one problem
 * of Algorithm 3; a persistent kernel splits the GPU into teams of CTAs that
 * take problems from a queue, largest instances first, so uneven problems run
 * side by side; problems of one instance run next to each other and share its
 * dictionary through the L2.  The device work of a run (descriptor upload,
 * counters, the launch, result download) is captured once into a CUDA graph by
 * ds_batch_create and replayed by every ds_batch_run; buffers are read at run
 * time, so new y values (same addresses) and new lambdas (same host arrays)
 * are picked up.  res: host, sum(n_rhs) entries, instance-major.
 * Errors: DS_ERR_INVALID, DS_ERR_OOM, DS_ERR_CUDA, DS_ERR_UNSUPPORTED,
 * DS_ERR_TIMEOUT. */
typedef struct ds_batch ds_batch;
ds_status ds_batch_create(ds_ctx* ctx, int n, const ds_dict* const* dicts, const void* const* Y, const int* n_rhs,
                          const double* const* lambdas, const ds_options* opt, void* const* X_out, ds_batch** out);
/* Run the batch; res as above.  Errors: DS_ERR_INVALID (NULL batch or res),
 * DS_ERR_CUDA, DS_ERR_TIMEOUT. */
ds_status ds_batch_run(ds_batch* batch, ds_result* res);
/* Whether the run replays a CUDA graph, and the team layout chosen.
 * Errors: DS_ERR_INVALID on NULL batch. */
ds_status ds_batch_info(const ds_batch* batch, int* uses_graph, int* teams, int* team_size);
/* How the batch's problems run (any output pointer may be NULL):
 *   multi_rhs_blocks: blocks of up to 64 right-hand sides of one FP32 Lasso
 *     instance solved together (opt->batch_multi_rhs, tests NONE/SAFE/DST3/DOME,
 *     instances with >= 2 right-hand sides).  A block runs Algorithm 3 for all
 *     its problems in lockstep: the correlation of every iteration is one
 *     contraction D_A^T [theta_1 ... theta_R] over the union A of their active
 *     sets, so each dictionary column read serves all of them; screening,
 *     iterates, gaps and stopping stay per problem, and a problem leaves the
 *     block when its gap is met.  multi_rhs_teams / multi_rhs_team_size: the
 *     persistent launch that runs the blocks;
 *   single_problems: (instance, rhs) problems run one per team as above.
 * Errors: DS_ERR_INVALID on NULL batch. */
ds_status ds_batch_layout(const ds_batch* batch, int* multi_rhs_blocks, int* multi_rhs_teams, int* multi_rhs_team_size,
                          int* single_problems);
/* Autotuner of the multi-RHS schedule.  Runs the batch once under each of up to
 * max_candidates schedules -- the plan's own first, then: blocks of 32 right-hand sides
 * grouped by lambda (similar iteration counts and screened sets per block), and, when a
 * dictionary has a BF16 copy, the tensor-core bulk phase turned off / on and a coarser
 * switch level (1e-2) -- timing each run on the device, and keeps the fastest for the
 * following ds_batch_run calls (the batch's handle stays valid).  Every tuning run
 * solves the batch, so X_out holds a valid solution afterwards.  ms_tried (nullable,
 * max_candidates entries) receives each run's device time in ms (-1 when a candidate
 * could not be built); *chosen the index of the kept schedule (0: unchanged).
 * Errors: DS_ERR_INVALID, and the errors of ds_batch_run for the plan's own run. */
ds_status ds_batch_autotune(ds_batch* batch, int max_candidates, int* chosen, int* n_tried, float* ms_tried);
/* The batch's current multi-RHS schedule (any output pointer may be NULL).
 * Errors: DS_ERR_INVALID on NULL batch. */
ds_status ds_batch_schedule(const ds_batch* batch, int* tensor_bulk, int* block_rhs, int* sort_lambda,
                            double* lowp_switch);
/* Release a batch (NULL is a no-op). */
ds_status ds_batch_destroy(ds_batch* batch);
/* One-shot form: create, run once, destroy. */
ds_status ds_solve_batch(ds_ctx* ctx, int n, const ds_dict* const* dicts, const void* const* Y, const int* n_rhs,
                         const double* const* lambdas, const ds_options* opt, void* const* X_out, ds_result* res);

/* ----------------------------------------------------------------- serving
 * A continuous-batching server: requests (one y and one lambda on a registered
 * FP32 dictionary, Lasso or Group-Lasso) are admitted while others run.  A
 * persistent kernel splits the GPU into teams of team_size CTAs (0 = 4); each
 * team takes the next admitted request, keeps its iterate, residual and
 * shrinking active set on the device, and retires it when the duality gap is
 * met, then takes another.  A request is admitted when a ring slot is free and
 * its workspace (sized for its N and K) fits in the hbm_budget_bytes pool
 * (admission by HBM footprint); otherwise it waits in a host queue.  When no
 * work arrives for a while the kernel exits and the next submission relaunches
 * it.  Requests of any N <= max_N, K <= max_K mix freely.
 *   ds_server_submit: y (host, N floats) is copied during the call; x_out (host,
 *     K floats) must stay valid until ds_server_poll returns DS_OK for the
 *     ticket.  Returns a ticket.  DS_ERR_UNSUPPORTED beyond max_N / max_K or
 *     for an FP64 dictionary.
 *   ds_server_poll: DS_PENDING while the request runs; DS_OK fills res
 *     (res->ms = latency from submission to completion) and forgets the ticket.
 *   ds_server_stats: completed, in flight, waiting, kernel launches, pool bytes.
 * team_size: CTAs per team, 0 (= 4) to the number of SMs; large requests (HBM-bound) want larger
 * teams, many small ones smaller teams.
 * A server drives its own CUDA stream; calls are serialised internally.
 * Errors: DS_ERR_INVALID (null arguments, a dictionary of another context, a
 * Lasso test on a group dictionary, an unknown ticket), DS_ERR_UNSUPPORTED (as
 * above), DS_ERR_OOM, DS_ERR_CUDA; ds_server_destroy(NULL) is a no-op. */
typedef struct ds_server ds_server;
ds_status ds_server_create(ds_ctx* ctx, size_t hbm_budget_bytes, int64_t max_N, int64_t max_K, int team_size,
                           ds_server** out);
ds_status ds_server_submit(ds_server* server, const ds_dict* dict, const void* y, double lambda, const ds_options* opt,
                           void* x_out, uint64_t* ticket);
ds_status ds_server_poll(ds_server* server, uint64_t ticket, ds_result* res);
ds_status ds_server_stats(ds_server* server, int64_t* completed, int64_t* in_flight, int64_t* pending,
                          int64_t* launches, size_t* pool_in_use);
ds_status ds_server_destroy(ds_server* server);

/* Allocation-free Lasso solve.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- a framework whose
 * caching allocator owns all device memory, a service with a fixed memory
 * budget committed up front, or a latency-critical loop that must not pay for
 * cudaMalloc/cudaFree (cudaFree can synchronize the whole device).  It calls no
 * cudaMalloc, cudaFree or allocating library routine: the solver's scratch is
 * one fixed 3 MiB array in device memory that every GPU loading this library
 * holds until the process exits.
 *
 * Same computation as ds_solve with a Lasso dictionary (ISTA, FISTA or
 * Chambolle-Pock, any test;
 * DS_GSAFE / DS_DGST3 act as singleton groups), run on `device` and ordered on
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 *   D      device memory of `device` (or managed memory), FP32, column-major
 *          N x K, leading dimension ld with N <= ld <= N rounded up to a
 *          multiple of 512 and ld % 4 == 0, D 16-byte aligned; rows N..ld-1, if
 *          any, are not part of the atoms and must hold finite values (a row
 *          slice of a taller column-major matrix qualifies).  A larger ld is
 *          rejected with DS_ERR_UNSUPPORTED.
 *   y      device, FP32, N entries.      x_out  device, FP32, K entries
 *          (both on `device`, or managed).
 *   opt    host; opt->L > 0 is required (e.g. ds_dict_lipschitz of a
 *          registered copy of D, or any upper bound of ||D||_2^2).
 *   res    host.
 * Limits: N <= 4096 and K <= 16384, else DS_ERR_UNSUPPORTED (the fixed
 * scratch would be too small; a message names the limits).
 * The first call on a device resolves the scratch array's device address
 * (set-up, once per device); make that first call before any stream capture.
 * Every call shares the one scratch array per device and it keeps the last
 * call's contents; the call clears what must start at zero.  Calls whose GPU
 * work overlaps (concurrent streams, several host threads) race on the array:
 * serialise them.  Synchronous like ds_solve.  The caller's current device is
 * restored before the call returns.  Errors: DS_ERR_INVALID (null or host
 * pointers, pointers to another GPU's memory, bad sizes or alignment,
 * lambda <= 0, opt->L <= 0), DS_ERR_UNSUPPORTED, DS_ERR_CUDA, DS_ERR_TIMEOUT. */
ds_status ds_solve_lasso_noalloc(int device, void* cuda_stream, const float* D, int64_t N, int64_t K, int64_t ld,
                                 const float* y, double lambda, const ds_options* opt, float* x_out, ds_result* res);

/* Self-test of the failure detection; the paper has no counterpart (its
 * solvers run on one CPU and wait for nothing).  Every wait of the persistent
 * kernels on other CTAs (grid barriers) gives up after a time limit (2 s),
 * raises an error flag that the other CTAs see, and the kernel returns; the
 * host then reports DS_ERR_TIMEOUT and the context stays usable.  This call
 * launches a two-CTA kernel on `device` in which one CTA never arrives at the
 * barrier, so the other's wait runs out: *status receives DS_ERR_TIMEOUT when
 * the wait gave up as designed (DS_OK would mean it completed), *waited_ms the
 * kernel's duration.  No fault, trap or endless loop is involved.  Errors:
 * DS_ERR_INVALID (null pointer, no such device), DS_ERR_OOM, DS_ERR_CUDA. */
ds_status ds_selftest_wait_timeout(int device, int* status, double* waited_ms);

/* Number of CUDA kernels this context has launched so far (solves, lambda_max
 * queries and dictionary precomputes).  Errors: DS_ERR_INVALID on NULL. */
ds_status ds_ctx_kernel_launches(const ds_ctx* ctx, int64_t* n);

/* Record per-iteration history of the following solves into hist (device,
 * max_rows x 6 doubles, row t-1 = iteration t: active atoms, nnz(x), R,
 * test radius, gap, mu), or stop recording (hist NULL).  Only the first
 * lambda of a path is recorded.  Errors: DS_ERR_INVALID (NULL ctx, or hist
 * with max_rows < 1). */
ds_status ds_set_history(ds_ctx* ctx, double* hist, int max_rows);

/* Record, for the following solves, which test iteration screened each atom
 * (Algorithm 3's cumulative set I_t, atom by atom): scr_iter (device, capacity
 * int32 values) receives, for each lambda j of a solve or path with
 * (j + 1) * K <= capacity, K values at scr_iter + j * K: t >= 1 when the test
 * of iteration t screened the atom (its group), -1 when the static test of
 * Algorithm 1 did (dynamic = 0), 0 when the atom was never screened.  Passing
 * NULL stops recording.  The buffer must stay valid while solves run; it is
 * written by the solve kernels only (batches and servers do not record).
 * Errors: DS_ERR_INVALID (NULL ctx, or scr_iter with capacity < 1). */
ds_status ds_set_screen_log(ds_ctx* ctx, int32_t* scr_iter, int64_t capacity);

#ifdef __cplusplus
}
#endif
#endif /* DSCREEN_H */
