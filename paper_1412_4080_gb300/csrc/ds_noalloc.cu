// ds_noalloc.cu -- ds_solve_lasso_noalloc: a Lasso solve that allocates no
// memory at all.
//
// Some callers cannot call cudaMalloc: a framework whose caching allocator owns
// all device memory and forbids allocations behind its back, a service that
// commits a fixed memory budget up front, or a latency-critical loop that must
// not pay for cudaMalloc/cudaFree (cudaFree can synchronize the whole device).
// For them, the solver's scratch lives in one file-scope __device__ array of
// fixed size that every GPU loading this library holds until the process
// exits; the caller passes only inputs and outputs.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "ds_internal.h"

namespace {

// Size limits of the allocation-free path and its scratch array.
constexpr int64_t kNoAllocMaxN = 4096;
constexpr int64_t kNoAllocMaxK = 16384;
constexpr size_t kNoAllocScratchBytes = 3u << 20;  // >= the solve workspace at the limits above
constexpr int64_t kNoAllocChunk = 512;              // rows of one FP32 correlation chunk (32 lanes x 4 x 4)

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
    bool ready;
    void* scratch;  // device address of g_noalloc_scratch on this device
    int num_sms;
    size_t smem_optin;
};

constexpr int kMaxDevices = 64;
NoAllocDevice g_dev[kMaxDevices];
std::mutex g_mu;

// Once per device, with that device current: resolve the device address of the
// scratch array (the host-side symbol is only a stand-in and must never be
// passed to a kernel) and read the launch limits.
ds_status setup_device(int device, NoAllocDevice** out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    NoAllocDevice& d = g_dev[device];
    if (!d.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DS_ERR_CUDA;
        }
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return DS_ERR_CUDA;
        if (!prop.cooperativeLaunch) return DS_ERR_UNSUPPORTED;
        d.scratch = p;
        d.num_sms = prop.multiProcessorCount;
        d.smem_optin = prop.sharedMemPerBlockOptin;
        d.ready = true;
    }
    *out = &d;
    return DS_OK;
}

// A device (or managed) allocation that the kernel can read on `device`: memory of
// another GPU would be dereferenced without peer access.
bool on_device(const void* p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

// Restores the caller's current device when the entry point returns.
struct DeviceRestore {
    int prev = -1;
    ~DeviceRestore()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" ds_status ds_solve_lasso_noalloc(int device, void* cuda_stream, const float* D, int64_t N, int64_t K,
                                            int64_t ld, const float* y, double lambda, const ds_options* opt,
                                            float* x_out, ds_result* res)
{
    if (!D || !y || !x_out || !opt || !res || N <= 0 || K <= 0 || ld < N) return DS_ERR_INVALID;
    if (!(lambda > 0.0) || !(opt->L > 0.0) || opt->max_iter < 1 || !(opt->tol_gap_rel >= 0.0)) return DS_ERR_INVALID;
    if (opt->alg != DS_ISTA && opt->alg != DS_FISTA && opt->alg != DS_CP) return DS_ERR_INVALID;
    if (opt->test < DS_TEST_NONE || opt->test > DS_DGST3) return DS_ERR_INVALID;
    if (N > kNoAllocMaxN || K > kNoAllocMaxK) {
        fprintf(stderr, "ds_solve_lasso_noalloc: N=%lld K=%lld exceeds the fixed scratch limits N<=%lld K<=%lld\n",
                (long long)N, (long long)K, (long long)kNoAllocMaxN, (long long)kNoAllocMaxK);
        return DS_ERR_UNSUPPORTED;
    }
    // 16-byte vector loads: columns must start on 16-byte boundaries
    if (ld % 4 != 0 || (reinterpret_cast<uintptr_t>(D) & 15) != 0) return DS_ERR_INVALID;
    // The kernel stages y (and d_* in the DST3/Dome precompute) in shared vectors of
    // N rounded up to its 512-row correlation chunk, and walks each column of D up to
    // ld: a leading dimension beyond that rounding would read past those vectors.
    if (ld >= (int64_t(1) << 31) || ld > (N + kNoAllocChunk - 1) / kNoAllocChunk * kNoAllocChunk) {
        fprintf(stderr, "ds_solve_lasso_noalloc: ld=%lld exceeds N=%lld rounded up to a multiple of %lld\n",
                (long long)ld, (long long)N, (long long)kNoAllocChunk);
        return DS_ERR_UNSUPPORTED;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return DS_ERR_CUDA;
    }
    if (device < 0 || device >= ndev || device >= kMaxDevices) return DS_ERR_INVALID;
    DeviceRestore restore;
    if (cudaGetDevice(&restore.prev) != cudaSuccess) {
        cudaGetLastError();
        return DS_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return DS_ERR_CUDA;
    if (!on_device(D, device) || !on_device(y, device) || !on_device(x_out, device)) return DS_ERR_INVALID;
    NoAllocDevice* dev = nullptr;
    ds_status st = setup_device(device, &dev);
    if (st != DS_OK) return st;

    ds::DictDesc dd;
    std::memset(&dd, 0, sizeof(dd));
    dd.D = D;
    dd.dtype = DS_FP32;
    dd.N = (int)N;
    dd.K = (int)K;
    dd.ld = (int)ld;
    dd.nG = (int)K;
    dd.is_group = 0;
    dd.max_gsize = 1;
    dd.L = opt->L;
    dd.norms_in_kernel = true;
    if (ds::solve_ws_bytes(dd, dev->num_sms, dev->smem_optin, 1) > kNoAllocScratchBytes) return DS_ERR_UNSUPPORTED;

    ds::SolveEnv env;
    std::memset(&env, 0, sizeof(env));
    env.stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    env.num_sms = dev->num_sms;
    env.smem_optin = dev->smem_optin;
    env.ws = dev->scratch;
    env.ws_bytes = kNoAllocScratchBytes;
    env.ctx = nullptr;  // no context: no workspace growth, no FISTA table, no timing events
    ds::DevResult r;
    st = ds::launch_solve_env(env, dd, y, nullptr, 1, &lambda, opt, x_out, K, &r, nullptr);
    if (st != DS_OK && st != DS_ERR_TIMEOUT) return st;
    res->iters = r.iters;
    res->status = r.status;
    res->n_active = r.n_active;
    res->nnz = r.nnz;
    res->gap = r.gap;
    res->primal = r.primal;
    res->dual = r.dual;
    res->lambda = r.lambda;
    res->lambda_max = r.lambda_max;
    res->ms = 0.0;
    res->cols_corr = r.cols_corr;
    res->cols_synth = r.cols_synth;
    res->cols_lowp = r.cols_lowp;
    return st;
}
