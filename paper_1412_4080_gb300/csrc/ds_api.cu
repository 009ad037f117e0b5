// ds_api.cu -- the C ABI declared in include/dscreen.h: argument checks,
// host/device pointer handling, workspace management and dispatch to the
// kernel launchers.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ds_internal.h"

using namespace ds;

namespace {

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t elem_size(int dtype) { return dtype == DS_FP64 ? 8 : 4; }

ds_status ensure_io(ds_ctx* ctx, size_t bytes)
{
    if (bytes <= ctx->io_bytes) return DS_OK;
    if (ctx->d_io) cudaFree(ctx->d_io);
    ctx->d_io = nullptr;
    ctx->io_bytes = 0;
    if (cudaMalloc(&ctx->d_io, bytes) != cudaSuccess) return DS_ERR_OOM;
    ctx->io_bytes = bytes;
    return DS_OK;
}

bool valid_opt(const ds_options* o)
{
    return o && o->alg >= DS_ISTA && o->alg <= DS_TWIST && o->test >= DS_TEST_NONE &&
           o->test <= DS_DGST3 && o->max_iter >= 1 && o->tol_gap_rel >= 0.0 && std::isfinite(o->tol_gap_rel) &&
           std::isfinite(o->cp_tau) && std::isfinite(o->cp_sigma) && o->cp_gamma >= 0.0 && std::isfinite(o->cp_gamma) &&
           std::isfinite(o->bt_L0) && std::isfinite(o->twist_xi1) && o->twist_xi1 < 1.0 && o->team_size >= 0;
}

}  // namespace

namespace ds {

ds_status ctx_reserve(ds_ctx* ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes) return DS_OK;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return DS_ERR_CUDA;
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    size_t want = align_up(bytes, 1 << 20);
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
        cudaGetLastError();
        return DS_ERR_OOM;
    }
    ctx->ws_bytes = want;
    return DS_OK;
}

// The FISTA extrapolation coefficients depend on the iteration number only
// (Table 1: l_0 = 1, l_t = (1 + sqrt(1 + 4 l_{t-1}^2)) / 2, coefficient
// (l_{t-1} - 1) / l_t); they are tabulated once per context in FP64 on the host.
ds_status ctx_fista_table(ds_ctx* ctx, int n)
{
    const int cap = 1 << 20;
    n = std::min(std::max(n, 1024), cap);
    if (ctx->fista_n >= n) return DS_OK;
    std::vector<double> tab(2 * (size_t)n);
    double l = 1.0;
    for (int t = 0; t < n; t++) {
        const double ln = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * l * l));
        tab[2 * t] = (l - 1.0) / ln;
        tab[2 * t + 1] = ln;
        l = ln;
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return DS_ERR_CUDA;
    if (ctx->fista) cudaFree(ctx->fista);
    ctx->fista = nullptr;
    ctx->fista_n = 0;
    if (cudaMalloc(&ctx->fista, sizeof(double) * tab.size()) != cudaSuccess) return DS_ERR_OOM;
    if (cudaMemcpy(ctx->fista, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return DS_ERR_CUDA;
    ctx->fista_n = n;
    return DS_OK;
}

}  // namespace ds

extern "C" {

const char* ds_status_str(ds_status s)
{
    switch (s) {
    case DS_OK: return "DS_OK";
    case DS_ERR_INVALID: return "DS_ERR_INVALID";
    case DS_ERR_OOM: return "DS_ERR_OOM";
    case DS_ERR_CUDA: return "DS_ERR_CUDA";
    case DS_ERR_TIMEOUT: return "DS_ERR_TIMEOUT";
    case DS_ERR_NOT_CONVERGED: return "DS_ERR_NOT_CONVERGED";
    case DS_ERR_UNSUPPORTED: return "DS_ERR_UNSUPPORTED";
    case DS_PENDING: return "DS_PENDING";
    }
    return "DS_ERR_UNKNOWN";
}

ds_status ds_options_default(ds_options* opt)
{
    if (!opt) return DS_ERR_INVALID;
    opt->alg = DS_FISTA;
    opt->test = DS_DST3;
    opt->dynamic = 1;
    opt->max_iter = 10000;
    opt->tol_gap_rel = 1e-6;
    opt->L = 0.0;
    opt->lambda_rel = 0;
    opt->lowp_switch = 0.0;
    opt->batch_multi_rhs = 1;
    opt->warm_start = 0;
    opt->cp_tau = 0.0;
    opt->cp_sigma = 0.0;
    opt->cp_gamma = 0.0;
    opt->step_backtracking = 0;
    opt->bt_L0 = 0.0;
    opt->twist_xi1 = 0.0;
    opt->gap_every = 1;
    opt->team_size = 0;
    return DS_OK;
}

ds_status ds_create(int device, void* cuda_stream, ds_ctx** out)
{
    if (!out) return DS_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        cudaGetLastError();
        return DS_ERR_CUDA;
    }
    if (device < 0 || device >= n) return DS_ERR_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return DS_ERR_CUDA;
    ds_ctx* c = new (std::nothrow) ds_ctx();
    if (!c) return DS_ERR_OOM;
    c->device = device;
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return DS_ERR_CUDA;
    }
    c->num_sms = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    if (!prop.cooperativeLaunch) {
        delete c;
        return DS_ERR_UNSUPPORTED;
    }
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
        delete c;
        return DS_ERR_CUDA;
    }
    *out = c;
    return DS_OK;
}

ds_status ds_destroy(ds_ctx* c)
{
    if (!c) return DS_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->ws) cudaFree(c->ws);
    if (c->d_io) cudaFree(c->d_io);
    if (c->h_res) cudaFreeHost(c->h_res);
    if (c->fista) cudaFree(c->fista);
    cudaEventDestroy(c->ev0);
    cudaEventDestroy(c->ev1);
    delete c;
    return DS_OK;
}

ds_status ds_ctx_kernel_launches(const ds_ctx* ctx, int64_t* n)
{
    if (!ctx || !n) return DS_ERR_INVALID;
    *n = ctx->launches;
    return DS_OK;
}

ds_status ds_set_history(ds_ctx* ctx, double* hist, int max_rows)
{
    if (!ctx || (hist && max_rows < 1)) return DS_ERR_INVALID;
    ctx->hist = hist;
    ctx->hist_rows = hist ? max_rows : 0;
    return DS_OK;
}

ds_status ds_set_screen_log(ds_ctx* ctx, int32_t* scr_iter, int64_t capacity)
{
    if (!ctx || (scr_iter && capacity < 1)) return DS_ERR_INVALID;
    ctx->scr_log = scr_iter;
    ctx->scr_cap = scr_iter ? capacity : 0;
    return DS_OK;
}

ds_status ds_dict_create(ds_ctx* ctx, const void* D, int64_t N, int64_t K, int64_t ld, ds_prec dtype,
                         const int64_t* group_offsets, const double* weights, int64_t n_groups, ds_prec work_prec,
                         ds_dict** out)
{
    if (!ctx || !D || !out || N <= 0 || K <= 0 || ld < N) return DS_ERR_INVALID;
    *out = nullptr;
    if (dtype != DS_FP32 && dtype != DS_FP64) return DS_ERR_INVALID;
    if (work_prec != dtype && !(dtype == DS_FP32 && (work_prec == DS_BF16 || work_prec == DS_FP8)))
        return DS_ERR_UNSUPPORTED;
    if (K >= (1ll << 31) || N >= (1ll << 30)) return DS_ERR_UNSUPPORTED;
    int max_gsize = 1;
    if (group_offsets) {
        if (n_groups <= 0 || group_offsets[0] != 0 || group_offsets[n_groups] != K) return DS_ERR_INVALID;
        for (int64_t g = 0; g < n_groups; g++) {
            int64_t sz = group_offsets[g + 1] - group_offsets[g];
            if (sz <= 0) return DS_ERR_INVALID;
            if (weights && !(weights[g] > 0.0 && std::isfinite(weights[g]))) return DS_ERR_INVALID;
            max_gsize = (int)std::max<int64_t>(max_gsize, sz);
        }
        if (max_gsize > kMaxGroup) return DS_ERR_UNSUPPORTED;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return DS_ERR_CUDA;
    const size_t es = elem_size(dtype);
    const int64_t align = 16 / (int64_t)es;
    const int64_t ldp = (N + align - 1) / align * align;
    ds_dict* d = new (std::nothrow) ds_dict();
    if (!d) return DS_ERR_OOM;
    d->ctx = ctx;
    d->dtype = dtype;
    d->N = N;
    d->K = K;
    d->ld = ldp;
    d->is_group = group_offsets != nullptr;
    d->nG = (int)(group_offsets ? n_groups : K);
    d->max_gsize = max_gsize;
    auto fail = [&](ds_status s) {
        ds_dict_destroy(d);
        return s;
    };
    cudaStream_t s = ctx->stream;
    if (cudaMalloc(&d->D, (size_t)ldp * K * es) != cudaSuccess) return fail(DS_ERR_OOM);
    if (cudaMalloc(&d->colnorm, sizeof(double) * K) != cudaSuccess) return fail(DS_ERR_OOM);
    if (cudaMemsetAsync(d->D, 0, (size_t)ldp * K * es, s) != cudaSuccess) return fail(DS_ERR_CUDA);
    cudaMemcpyKind kind = is_device_ptr(D) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpy2DAsync(d->D, ldp * es, D, ld * es, N * es, K, kind, s) != cudaSuccess) return fail(DS_ERR_CUDA);
    std::vector<double> wh;
    if (d->is_group) {
        std::vector<int> go(n_groups + 1);
        for (int64_t g = 0; g <= n_groups; g++) go[g] = (int)group_offsets[g];
        wh.resize(n_groups);
        for (int64_t g = 0; g < n_groups; g++)
            wh[g] = weights ? weights[g] : std::sqrt((double)(group_offsets[g + 1] - group_offsets[g]));
        if (cudaMalloc(&d->goff, sizeof(int) * (n_groups + 1)) != cudaSuccess) return fail(DS_ERR_OOM);
        if (cudaMalloc(&d->w, sizeof(double) * n_groups) != cudaSuccess) return fail(DS_ERR_OOM);
        if (cudaMalloc(&d->spec, sizeof(double) * n_groups) != cudaSuccess) return fail(DS_ERR_OOM);
        if (cudaMemcpyAsync(d->goff, go.data(), sizeof(int) * (n_groups + 1), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d->w, wh.data(), sizeof(double) * n_groups, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(DS_ERR_CUDA);
        if (cudaStreamSynchronize(s) != cudaSuccess) return fail(DS_ERR_CUDA);
    }
    ds_status st = dict_precompute(ctx, d, wh.empty() ? nullptr : wh.data());
    if (st != DS_OK) return fail(st);
    if (small_dict_eligible(dtype, d->is_group, N, K)) {
        if (cudaMalloc(&d->Dff, sizeof(float2) * (size_t)N * K) != cudaSuccess) return fail(DS_ERR_OOM);
        if (small_dict_split(static_cast<const double*>(d->D), ldp, (int)N, (int)K, d->Dff, s) != cudaSuccess)
            return fail(DS_ERR_CUDA);
    }
    if (work_prec == DS_BF16 || work_prec == DS_FP8) {
        st = dict_lowp(ctx, d, work_prec == DS_BF16 ? 1 : 2);
        if (st != DS_OK) return fail(st);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(DS_ERR_CUDA);
    *out = d;
    return DS_OK;
}

ds_status ds_dict_destroy(ds_dict* d)
{
    if (!d) return DS_OK;
    if (d->ctx) {
        cudaSetDevice(d->ctx->device);
        cudaStreamSynchronize(d->ctx->stream);
    }
    if (d->D) cudaFree(d->D);
    if (d->colnorm) cudaFree(d->colnorm);
    if (d->goff) cudaFree(d->goff);
    if (d->w) cudaFree(d->w);
    if (d->spec) cudaFree(d->spec);
    if (d->Dlo) cudaFree(d->Dlo);
    if (d->lo_scale) cudaFree(d->lo_scale);
    if (d->Dff) cudaFree(d->Dff);
    delete d;
    return DS_OK;
}

ds_status ds_dict_lipschitz(const ds_dict* d, double* L)
{
    if (!d || !L) return DS_ERR_INVALID;
    *L = d->L;
    return DS_OK;
}

ds_status ds_lambda_max(ds_ctx* ctx, const ds_dict* d, const void* y, double* lambda_max)
{
    if (!ctx || !d || !y || !lambda_max || d->ctx != ctx) return DS_ERR_INVALID;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return DS_ERR_CUDA;
    const size_t es = elem_size(d->dtype);
    const void* yd = y;
    if (!is_device_ptr(y)) {
        ds_status st = ensure_io(ctx, d->N * es + 256);
        if (st != DS_OK) return st;
        if (cudaMemcpyAsync(ctx->d_io, y, d->N * es, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess)
            return DS_ERR_CUDA;
        yd = ctx->d_io;
    }
    return launch_lambda_max(ctx, d, yd, lambda_max);
}

ds_status ds_solve_path(ds_ctx* ctx, const ds_dict* d, const void* y, int n_lambda, const double* lambdas,
                        const ds_options* opt, const void* x0, void* X_out, ds_result* res)
{
    if (!ctx || !d || !y || !X_out || !res || !lambdas || n_lambda < 1 || d->ctx != ctx) return DS_ERR_INVALID;
    if (!valid_opt(opt)) return DS_ERR_INVALID;
    for (int j = 0; j < n_lambda; j++)
        if (!(lambdas[j] > 0.0) || !std::isfinite(lambdas[j])) return DS_ERR_INVALID;
    if (d->is_group && (opt->test == DS_SAFE || opt->test == DS_DST3 || opt->test == DS_DOME)) return DS_ERR_INVALID;
    if (opt->L < 0.0 || !std::isfinite(opt->L)) return DS_ERR_INVALID;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return DS_ERR_CUDA;
    const size_t es = elem_size(d->dtype);
    const bool y_dev = is_device_ptr(y), x0_dev = x0 ? is_device_ptr(x0) : true, xo_dev = is_device_ptr(X_out);
    size_t need = 0;
    size_t off_y = 0, off_x0 = 0, off_xo = 0;
    if (!y_dev) { off_y = need; need = align_up(need + d->N * es, 256); }
    if (!x0_dev) { off_x0 = need; need = align_up(need + d->K * es, 256); }
    if (!xo_dev) { off_xo = need; need = align_up(need + (size_t)d->K * n_lambda * es, 256); }
    if (need) {
        ds_status st = ensure_io(ctx, need);
        if (st != DS_OK) return st;
    }
    char* io = reinterpret_cast<char*>(ctx->d_io);
    cudaStream_t s = ctx->stream;
    const void* yd = y;
    const void* x0d = x0;
    void* xod = X_out;
    if (!y_dev) {
        if (cudaMemcpyAsync(io + off_y, y, d->N * es, cudaMemcpyHostToDevice, s) != cudaSuccess) return DS_ERR_CUDA;
        yd = io + off_y;
    }
    if (!x0_dev) {
        if (cudaMemcpyAsync(io + off_x0, x0, d->K * es, cudaMemcpyHostToDevice, s) != cudaSuccess) return DS_ERR_CUDA;
        x0d = io + off_x0;
    }
    if (!xo_dev) xod = io + off_xo;
    std::vector<DevResult> r(n_lambda);
    float ms = 0.f;
    ds_status st = launch_solve(ctx, d, yd, x0d, n_lambda, lambdas, opt, xod, d->K, r.data(), &ms);
    if (st != DS_OK && st != DS_ERR_TIMEOUT) return st;
    if (!xo_dev) {
        if (cudaMemcpyAsync(X_out, xod, (size_t)d->K * n_lambda * es, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return DS_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return DS_ERR_CUDA;
    }
    for (int j = 0; j < n_lambda; j++) {
        res[j].iters = r[j].iters;
        res[j].status = r[j].status;
        res[j].n_active = r[j].n_active;
        res[j].nnz = r[j].nnz;
        res[j].gap = r[j].gap;
        res[j].primal = r[j].primal;
        res[j].dual = r[j].dual;
        res[j].lambda = r[j].lambda;
        res[j].lambda_max = r[j].lambda_max;
        res[j].ms = ms / n_lambda;
        res[j].cols_corr = r[j].cols_corr;
        res[j].cols_synth = r[j].cols_synth;
        res[j].cols_lowp = r[j].cols_lowp;
    }
    return st;
}

ds_status ds_solve(ds_ctx* ctx, const ds_dict* d, const void* y, double lambda, const ds_options* opt, const void* x0,
                   void* x_out, ds_result* res)
{
    return ds_solve_path(ctx, d, y, 1, &lambda, opt, x0, x_out, res);
}

}  // extern "C"
