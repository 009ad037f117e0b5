// ds_internal.h -- structures shared by the translation units of libdscreen
// (host side of the C ABI and the kernel launchers).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dscreen.h"
#include "ds_common.cuh"

struct ds_ctx {
    int device;
    cudaStream_t stream;
    int num_sms;
    size_t smem_optin;
    // solve workspace (grown on demand, bump-allocated)
    void* ws;
    size_t ws_bytes;
    // device-side result staging and pinned host copy
    void* d_res;
    void* h_res;
    size_t res_cap;  // in results
    // staging for host y / x0 / x_out
    void* d_io;
    size_t io_bytes;
    double* hist;
    int hist_rows;
    int* scr_log;       // per-atom screening log of the following solves (device), scr_cap ints
    int64_t scr_cap;
    long long launches;
    double* fista;  // device table of the FISTA sequence (coefficient, l_t), t = 1..fista_n
    int fista_n;
    cudaEvent_t ev0, ev1;
};

struct ds_dict {
    ds_ctx* ctx;
    int dtype;        // DS_FP32 or DS_FP64
    int64_t N, K, ld; // ld: padded leading dimension of the owned copy (elements)
    void* D;          // device copy, ld * K elements, zero rows N..ld-1
    double* colnorm;  // device, K: ||d_i||
    int is_group;
    int nG;           // groups (Lasso: K)
    int max_gsize;
    int* goff;        // device, nG + 1 (Lasso: nullptr)
    double* w;        // device, nG (Lasso: nullptr)
    double* spec;     // device, nG: upper estimate of ||D_g||_2 (Lasso: nullptr)
    double fmax;      // max_g ||D_g||_F / w_g (Lasso: max_i ||d_i||)
    double L;         // upper estimate of ||D||_2^2
    // low-precision working copy (work_prec BF16 or FP8), next to the FP32 master
    int lo_kind;      // 0 none, 1 BF16, 2 FP8 e4m3 with a per-column scale
    void* Dlo;        // ld_lo * K elements, zero rows N..ld_lo-1
    int64_t ld_lo;
    float* lo_scale;  // FP8: per-column scale (d_i ~ scale_i * q_i)
    double emax;      // max_g ||D_g - Dlo_g||_F / w_g: rounding of the copy, for the radius bound
    // FP64 dictionaries small enough for the one-cluster solve: each entry as a float-float pair
    // (hi, lo), K columns of N, made once here so that no solve converts on the FP64 pipe
    float2* Dff;
};

namespace ds {

constexpr int kMaxGroup = 128;  // largest group (columns) of a Group-Lasso dictionary

// Per-solve result written by the solve kernel (one per lambda).
struct DevResult {
    int iters;
    int status;
    long long n_active;
    long long nnz;
    double gap, primal, dual, lambda, lambda_max;
    long long cols_corr, cols_synth, cols_lowp;
};

// Error codes raised inside kernels (DevResult.status).
constexpr int kDevOk = 0;
constexpr int kDevNotConverged = 5;
constexpr int kDevTimeout = 4;

// Dictionary as the solve kernel sees it.
struct DictDesc {
    const void* D;
    int dtype;
    int N, K, ld, nG, is_group, max_gsize;
    const int* goff;
    const double* w;
    const double* spec;
    const double* colnorm;  // may be null when norms_in_kernel
    double fmax, L;
    bool norms_in_kernel;   // Lasso only: the kernel computes ||d_i|| and their max itself
    int lo_kind;            // low-precision copy: 0 none, 1 BF16, 2 FP8
    const void* Dlo;
    int ld_lo;
    const float* lo_scale;
    double emax;
    const float2* Dff;      // FP64 dictionaries: the float-float copy (or null)
};

// Where and how a solve runs: a context (workspace reserved on demand, timing
// events, FISTA table) or, with ctx == nullptr, a caller-provided workspace.
struct SolveEnv {
    cudaStream_t stream;
    int num_sms;
    size_t smem_optin;
    void* ws;
    size_t ws_bytes;
    ds_ctx* ctx;
    const double* fista;
    int fista_n;
    double* hist;
    int hist_rows;
    int* scr_log;
    int64_t scr_cap;
};

size_t solve_ws_bytes(const DictDesc& dd, int num_sms, size_t smem_optin, int n_lambda);
DictDesc dict_desc(const ds_dict* d);
ds_status launch_solve_env(const SolveEnv& env, const DictDesc& dd, const void* y_dev, const void* x0_dev, int n_lambda,
                           const double* lambdas_host, const ds_options* opt, void* xout_dev, int64_t ldx,
                           DevResult* res_host, float* ms);

// Host-side launchers (defined in ds_solve.cu / ds_dict.cu).
ds_status launch_solve(ds_ctx* ctx, const ds_dict* dict, const void* y_dev, const void* x0_dev, int n_lambda,
                       const double* lambdas_host, const ds_options* opt, void* xout_dev, int64_t ldx,
                       DevResult* res_host, float* ms);
ds_status launch_lambda_max(ds_ctx* ctx, const ds_dict* dict, const void* y_dev, double* lmax);
ds_status dict_precompute(ds_ctx* ctx, ds_dict* dict, const double* w_host);
ds_status dict_lowp(ds_ctx* ctx, ds_dict* dict, int kind);
// the one-cluster solve of small FP64 Lasso problems (ds_small.cu): which dictionaries get the
// float-float copy, and the kernel that makes it
bool small_dict_eligible(int dtype, int is_group, long long N, long long K);
cudaError_t small_dict_split(const double* D, long long ld, int N, int K, float2* out, cudaStream_t s);

// Right-hand sides sharing a dictionary, solved together (ds_mrhs.cu): a block
// is up to 64 problems of one FP32 Lasso instance; problem r of the block is the
// instance's right-hand side ridx[r] (y at Y + ridx[r] * N, x at X + ridx[r] * K).
constexpr int kMrhsMaxR = 64;
struct MrhsBlock {
    const ds_dict* dict;
    const void* Y;  // the instance's right-hand sides (column 0)
    int R;
    void* X;        // the instance's solutions (column 0)
    int inst;
    int ridx[kMrhsMaxR];
};
// Schedule choices of a plan (the batch autotuner varies them).
struct MrhsCfg {
    int allow_tc;      // bulk phase on the tensor cores when the dictionary has a BF16 copy
    double lo_switch;  // > 0: overrides the bulk-to-FP32 switch level
    int team_size;     // > 0: CTAs per team (else chosen from the block sizes)
};
struct MrhsPlan;
ds_status mrhs_plan_create(ds_ctx* ctx, int n_blocks, const MrhsBlock* blocks, const ds_options* opt,
                           const double* fista_dev, int fista_n, const MrhsCfg& cfg, MrhsPlan** out);
const MrhsBlock* mrhs_plan_blocks(const MrhsPlan* M, int* n);  // in job order
double* mrhs_plan_lambdas(MrhsPlan* M);                        // pinned, [job][kMrhsMaxR]
const DevResult* mrhs_plan_results(const MrhsPlan* M);         // pinned, [job][kMrhsMaxR]
ds_status mrhs_plan_enqueue(MrhsPlan* M, cudaStream_t s);
int* mrhs_plan_error_flag(MrhsPlan* M);                        // device int
void mrhs_plan_info(const MrhsPlan* M, int* teams, int* team_size);
void mrhs_plan_destroy(MrhsPlan* M);

// Workspace helpers (ds_api.cu).
ds_status ctx_reserve(ds_ctx* ctx, size_t bytes);
ds_status ctx_fista_table(ds_ctx* ctx, int n);
ds_status ctx_reserve_results(ds_ctx* ctx, size_t n);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Simple bump allocator over a workspace block.
struct Bump {
    char* base;
    size_t off;
    template <typename U>
    U* take(size_t n)
    {
        off = align_up(off, 256);
        U* p = reinterpret_cast<U*>(base ? base + off : nullptr);
        off += n * sizeof(U);
        return p;
    }
};

}  // namespace ds
