// ds_solve.cu -- persistent cooperative kernel running a whole screened
// ISTA/FISTA solve (Algorithm 3 with the Table 1 updates) on one GB300.
//
// One CTA per SM stays resident for the whole solve.  Every iteration t is
// two grid phases separated by bounded grid barriers:
//
//   (A) test + synthesis      the Lemma 8 dual scaling and the radius of the
//                             chosen test (Lemmas 2-7) from the partials of
//                             t-1, the test itself on each CTA's slice of the
//                             atoms (Algorithm 3), and theta_t = D ubar_{t-1} - y
//                             and D xbar_{t-1} over the nonzeros only (row
//                             tiles), with the partials of theta^T y,
//                             ||theta||^2 and ||D xbar - y||^2;
//   (B) correlation + prox    the gap of iteration t-1 and the stopping rule
//                             (an adaptive step's acceptance test, and its redo,
//                             first), the compaction of the atoms the test kept,
//                             z = D_A^T theta_t over them (the dominant stream,
//                             theta staged in shared memory, 16-byte vector
//                             loads, warp-shuffle dots), the proximal step (soft
//                             threshold or group soft threshold), the FISTA
//                             extrapolation, the max |z| (or max ||z_g|| / w_g)
//                             partials and the per-CTA nonzero lists.
//
// Reductions are per-CTA partials summed in a fixed order by every CTA, so all
// CTAs take identical decisions and the results do not depend on timing.
#include <cmath>
#include <cstring>

#include "ds_solve_body.cuh"

namespace ds {

// the one-cluster solve of small FP64 Lasso problems (ds_small.cu)
int small_cluster_size(const SolveP<double>& P, size_t smem_optin, int* pitch);
cudaError_t launch_small(const SolveP<double>& P, int C, int pitch, size_t smem_optin, cudaStream_t s);

// ADAPT: the kernel also runs the adaptive-step rows (backtracking, SpaRSA, TwIST); fixed-step solves
// launch the instance without that code.  GRP: the instance for Group-Lasso (1) or Lasso (0)
// dictionaries, so that neither carries the other's code and register pressure.
template <typename T, bool ADAPT, int GRP>
__global__ void __launch_bounds__(kThreads, 1) solve_kernel(const SolveP<T> P)
{
    unsigned int gen = 0;  // running barrier target, used by thread 0 only
    if (!solve_body<T, ADAPT, GRP>(P, blockIdx.x, gridDim.x, P.ws.bar, gen) && blockIdx.x == 0 && threadIdx.x == 0) {
        const int n = P.n_lambda > 0 ? P.n_lambda : 1;
        for (int j = 0; j < n; j++) P.res[j].status = kDevTimeout;
    }
}

// ------------------------------------------------------------ host launcher


template <typename T>
size_t solve_ws_bytes_t(const DictDesc& dd, int num_sms, size_t smem_optin, int n_lambda)
{
    Geometry g;
    if (geometry<T>(dd, num_sms, smem_optin, &g) != DS_OK) return 0;
    Ws<T> w;
    double* l;
    DevResult* r;
    double* c;
    return layout<T>(nullptr, dd, g, n_lambda, &w, &l, &r, &c);
}

size_t solve_ws_bytes(const DictDesc& dd, int num_sms, size_t smem_optin, int n_lambda)
{
    return dd.dtype == DS_FP32 ? solve_ws_bytes_t<float>(dd, num_sms, smem_optin, n_lambda)
                               : solve_ws_bytes_t<double>(dd, num_sms, smem_optin, n_lambda);
}

// Results of a launched solve: copied back on the solve's stream, then the kernel time.
static ds_status finish_solve(const SolveEnv& env, DevResult* res_host, const DevResult* res_dev, int n_lambda,
                              float* ms)
{
    cudaStream_t s = env.stream;
    const int nr = std::max(n_lambda, 1);
    // through the context's pinned buffer when there is one (an asynchronous copy, not a staged one)
    DevResult* dst = res_host;
    if (env.ctx) {
        if (env.ctx->res_cap < (size_t)nr) {
            if (env.ctx->h_res) cudaFreeHost(env.ctx->h_res);
            env.ctx->h_res = nullptr;
            env.ctx->res_cap = 0;
            if (cudaMallocHost(&env.ctx->h_res, sizeof(DevResult) * nr) == cudaSuccess) env.ctx->res_cap = nr;
        }
        if (env.ctx->h_res) dst = static_cast<DevResult*>(env.ctx->h_res);
    }
    if (cudaMemcpyAsync(dst, res_dev, sizeof(DevResult) * nr, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DS_ERR_CUDA;
    if (dst != res_host) std::memcpy(res_host, dst, sizeof(DevResult) * nr);
    if (ms) {
        *ms = 0.f;
        if (env.ctx) cudaEventElapsedTime(ms, env.ctx->ev0, env.ctx->ev1);
    }
    for (int j = 0; j < std::max(n_lambda, 1); j++)
        if (res_host[j].status == kDevTimeout) return DS_ERR_TIMEOUT;
    return DS_OK;
}

template <typename T>
static ds_status launch_env_t(const SolveEnv& env, const DictDesc& dd, const void* y_dev, const void* x0_dev,
                              int n_lambda, const double* lambdas_host, const ds_options* opt, void* xout_dev,
                              int64_t ldx, DevResult* res_host, float* ms)
{
    constexpr int EV = 16 / sizeof(T);
    Geometry g;
    ds_status st = geometry<T>(dd, env.num_sms, env.smem_optin, &g);
    if (st != DS_OK) return st;
    // grid: one CTA per SM (a small problem is not faster on fewer: its iteration is bound by serial
    // steps and barrier waits, not by the number of arrivals); opt->team_size > 0 sets the count
    if (opt && opt->team_size > 0) g.G = std::max(1, std::min(g.G, opt->team_size));
    Ws<T> w;
    double* lam_dev;
    DevResult* res_dev;
    double* colnorm_w;
    const size_t need = layout<T>(nullptr, dd, g, n_lambda, &w, &lam_dev, &res_dev, &colnorm_w);
    char* base = reinterpret_cast<char*>(env.ws);
    if (env.ctx) {
        st = ctx_reserve(env.ctx, need);
        if (st != DS_OK) return st;
        base = reinterpret_cast<char*>(env.ctx->ws);
    } else if (!base || env.ws_bytes < need) {
        return DS_ERR_UNSUPPORTED;
    }
    layout<T>(base, dd, g, n_lambda, &w, &lam_dev, &res_dev, &colnorm_w);

    SolveP<T> P;
    fill_params<T>(P, dd, g, opt);
    P.fista = env.fista;
    P.fista_n = env.fista_n;
    P.colnorm_w = colnorm_w;
    P.y = reinterpret_cast<const T*>(y_dev);
    P.x0 = reinterpret_cast<const T*>(x0_dev);
    P.n_lambda = n_lambda;
    P.lambdas = lam_dev;
    P.x_out = reinterpret_cast<T*>(xout_dev);
    P.ldx = ldx;
    P.res = res_dev;
    P.hist = env.hist;
    P.hist_rows = env.hist_rows;
    P.scr_log = env.scr_log;
    P.scr_rows = env.scr_log ? (int)std::min<int64_t>(env.scr_cap / std::max(dd.K, 1), 1 << 30) : 0;
    P.ws = w;

    cudaStream_t s = env.stream;
    if constexpr (sizeof(T) == 8) {
        // a small FP64 Lasso problem runs on one thread-block cluster (team_size > 0 keeps the grid); its
        // lambda travels in the parameters, and it needs no grid barrier
        int pitch = 0;
        const int C = (opt && opt->team_size > 0) ? 0 : small_cluster_size(P, env.smem_optin, &pitch);
        if (C > 0) {
            P.lam0 = lambdas_host[0];
            if (env.ctx) {
                env.ctx->launches++;
                cudaEventRecord(env.ctx->ev0, s);
            }
            const cudaError_t e = launch_small(P, C, pitch, env.smem_optin, s);
            if (e != cudaSuccess) {
                fprintf(stderr, "dscreen: small solve launch failed: %s\n", cudaGetErrorString(e));
                return DS_ERR_CUDA;
            }
            if (env.ctx) cudaEventRecord(env.ctx->ev1, s);
            return finish_solve(env, res_host, res_dev, n_lambda, ms);
        }
    }
    if (n_lambda > 0 &&
        cudaMemcpyAsync(lam_dev, lambdas_host, sizeof(double) * n_lambda, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaMemsetAsync(w.bar, 0, sizeof(GridBarrier), s) != cudaSuccess) return DS_ERR_CUDA;
    if (cudaMemsetAsync(res_dev, 0, sizeof(DevResult) * std::max(n_lambda, 1), s) != cudaSuccess) return DS_ERR_CUDA;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DS_ERR_CUDA;
    const bool adapt = P.step_mode != 0;
    const int grp = P.is_group ? 1 : 0;
    const void* kfn = adapt ? (grp ? (const void*)solve_kernel<T, true, 1> : (const void*)solve_kernel<T, true, 0>)
                            : (grp ? (const void*)solve_kernel<T, false, 1> : (const void*)solve_kernel<T, false, 0>);
    static bool attr_set[2][2][64] = {};
    if (dev < 64 && !attr_set[adapt][grp][dev]) {
        if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(env.smem_optin - 40 * 1024)) != cudaSuccess)
            return DS_ERR_CUDA;
        attr_set[adapt][grp][dev] = true;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kThreads, g.smem) != cudaSuccess)
        return DS_ERR_CUDA;
    if (occ < 1) return DS_ERR_UNSUPPORTED;

    void* args[] = {(void*)&P};
    if (env.ctx) {
        env.ctx->launches++;
        cudaEventRecord(env.ctx->ev0, s);
    }
    cudaError_t e = cudaLaunchCooperativeKernel(kfn, dim3(g.G), dim3(kThreads), args, g.smem, s);
    if (e != cudaSuccess) {
        fprintf(stderr, "dscreen: solve launch failed: %s\n", cudaGetErrorString(e));
        return DS_ERR_CUDA;
    }
    if (env.ctx) cudaEventRecord(env.ctx->ev1, s);
    (void)EV;
    return finish_solve(env, res_host, res_dev, n_lambda, ms);
}

ds_status launch_solve_env(const SolveEnv& env, const DictDesc& dd, const void* y_dev, const void* x0_dev, int n_lambda,
                           const double* lambdas_host, const ds_options* opt, void* xout_dev, int64_t ldx,
                           DevResult* res_host, float* ms)
{
    if (dd.dtype == DS_FP32)
        return launch_env_t<float>(env, dd, y_dev, x0_dev, n_lambda, lambdas_host, opt, xout_dev, ldx, res_host, ms);
    return launch_env_t<double>(env, dd, y_dev, x0_dev, n_lambda, lambdas_host, opt, xout_dev, ldx, res_host, ms);
}

DictDesc dict_desc(const ds_dict* d)
{
    DictDesc dd;
    dd.D = d->D;
    dd.dtype = d->dtype;
    dd.N = (int)d->N;
    dd.K = (int)d->K;
    dd.ld = (int)d->ld;
    dd.nG = d->nG;
    dd.is_group = d->is_group;
    dd.max_gsize = d->max_gsize;
    dd.goff = d->goff;
    dd.w = d->w;
    dd.spec = d->spec;
    dd.colnorm = d->colnorm;
    dd.fmax = d->fmax;
    dd.L = d->L;
    dd.norms_in_kernel = false;
    dd.lo_kind = d->lo_kind;
    dd.Dlo = d->Dlo;
    dd.ld_lo = (int)d->ld_lo;
    dd.lo_scale = d->lo_scale;
    dd.emax = d->emax;
    dd.Dff = d->Dff;
    return dd;
}

ds_status launch_solve(ds_ctx* ctx, const ds_dict* dict, const void* y_dev, const void* x0_dev, int n_lambda,
                       const double* lambdas_host, const ds_options* opt, void* xout_dev, int64_t ldx,
                       DevResult* res_host, float* ms)
{
    if (opt && opt->alg == DS_FISTA) {
        ds_status fs = ctx_fista_table(ctx, opt->max_iter);
        if (fs != DS_OK) return fs;
    }
    SolveEnv env;
    env.stream = ctx->stream;
    env.num_sms = ctx->num_sms;
    env.smem_optin = ctx->smem_optin;
    env.ws = nullptr;
    env.ws_bytes = 0;
    env.ctx = ctx;
    env.fista = ctx->fista;
    env.fista_n = ctx->fista_n;
    env.hist = ctx->hist;
    env.hist_rows = ctx->hist_rows;
    env.scr_log = ctx->scr_log;
    env.scr_cap = ctx->scr_cap;
    return launch_solve_env(env, dict_desc(dict), y_dev, x0_dev, n_lambda, lambdas_host, opt, xout_dev, ldx, res_host,
                            ms);
}

ds_status launch_lambda_max(ds_ctx* ctx, const ds_dict* dict, const void* y_dev, double* lmax)
{
    DevResult r[1];
    ds_status st = launch_solve(ctx, dict, y_dev, nullptr, 0, nullptr, nullptr, nullptr, 0, r, nullptr);
    if (st == DS_OK) *lmax = r[0].lambda_max;
    return st;
}

}  // namespace ds
