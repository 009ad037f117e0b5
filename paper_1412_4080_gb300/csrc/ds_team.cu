// ds_team.cu -- many screened solves in one persistent launch.
//
// team_kernel splits the grid (one CTA per SM) into teams of T CTAs; each team
// takes problems from a queue and runs solve_body on them with its own
// barrier and workspace, so problems of uneven sizes run side by side and a
// team never waits for another.  Two queues feed it:
//   - batch: a device array of problems in a fixed order (largest first), for
//     ds_batch_* / ds_solve_batch.  The whole sequence (descriptor upload,
//     counter reset, the launch, result download) is captured once into a
//     CUDA graph and replayed;
//   - server: a ring of problem descriptors in mapped host memory that the host
//     fills while the kernel runs (continuous batching, ds_server_*).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "ds_solve_body.cuh"

namespace ds {

template <typename T>
struct TeamArgs {
    SolveP<T>* jobs;       // batch: device array; server: ring in mapped host memory
    int n_jobs;            // batch: problems; server: ring slots
    const Ws<T>* team_ws;  // one workspace per team (device)
    GridBarrier* bars;     // one barrier per team
    int* team_job;         // per team: the problem it took
    int* next_job;         // queue head (server: next sequence number to claim)
    int* error;            // set when a team's barrier timed out
    int team_size;
    int server;
    // server mode
    const volatile int* published;  // mapped host: number of problems published
    const volatile int* stop;       // mapped host: shutdown request
    volatile int* done;             // mapped host: per slot, sequence number + 1 when finished
    T* stage_y;                     // per team, max_N
    T* stage_x;                     // per team, max_K
    DevResult* stage_res;           // per team
    int max_N, max_K;
    long long idle_polls;           // server: give up waiting for work after this many polls
};

__device__ __forceinline__ int ld_acquire_sys(const volatile int* p)
{
    int v;
    asm volatile("ld.acquire.sys.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) team_kernel(const TeamArgs<T> A)
{
    __shared__ SolveP<T> sP;
    __shared__ int s_job;
    const int team = blockIdx.x / A.team_size, rank = blockIdx.x % A.team_size;
    GridBarrier* bar = A.bars + team;
    unsigned int gen = 0;  // running barrier target (thread 0)
    for (;;) {
        // ---- take the next problem (rank 0 of the team), tell the team
        if (threadIdx.x == 0 && rank == 0) {
            int j = -1;
            if (!A.server) {
                j = atomicAdd(A.next_job, 1);
                if (j >= A.n_jobs) j = -1;
            } else {
                long long polls = 0;
                while (!*A.stop) {
                    const int head = atomicAdd(A.next_job, 0);
                    if (head < ld_acquire_sys(A.published)) {
                        if (atomicCAS(A.next_job, head, head + 1) == head) {
                            j = head;
                            break;
                        }
                        continue;
                    }
                    if (++polls > A.idle_polls) break;  // idle: the host relaunches on the next request
                    __nanosleep(polls < 64 ? 200 : 2000);
                }
            }
            A.team_job[team] = j;
        }
        if (!grid_sync(bar, A.team_size, gen)) {
            if (threadIdx.x == 0) atomicExch(A.error, 1);
            return;
        }
        if (threadIdx.x == 0) s_job = __ldcg(A.team_job + team);
        __syncthreads();
        const int j = s_job;
        if (j < 0) return;
        const int slot = A.server ? j % A.n_jobs : j;
        T* host_x = nullptr;
        DevResult* host_res = nullptr;
        if (threadIdx.x == 0) {
            if (A.server) {
                // the descriptor lives in host memory: copy it word by word with volatile loads
                const volatile unsigned int* src = reinterpret_cast<const volatile unsigned int*>(A.jobs + slot);
                unsigned int* dst = reinterpret_cast<unsigned int*>(&sP);
                for (int k = 0; k < (int)(sizeof(SolveP<T>) / 4); k++) dst[k] = src[k];
            } else {
                sP = A.jobs[slot];
            }
            sP.ws = A.team_ws[team];
        }
        __syncthreads();
        if (A.server) {
            // stage y in device memory; outputs go to team staging, copied out at the end
            T* ys = A.stage_y + (size_t)team * A.max_N;
            const volatile T* yh = sP.y;
            for (int r = rank * kThreads + threadIdx.x; r < sP.N; r += A.team_size * kThreads) ys[r] = yh[r];
            host_x = sP.x_out;
            host_res = sP.res;
            __syncthreads();
            if (threadIdx.x == 0) {
                sP.y = ys;
                sP.x_out = A.stage_x + (size_t)team * A.max_K;
                sP.ldx = A.max_K;
                sP.res = A.stage_res + team;
            }
            if (!grid_sync(bar, A.team_size, gen)) {
                if (threadIdx.x == 0) atomicExch(A.error, 1);
                return;
            }
        }
        if (!solve_body<T>(sP, rank, A.team_size, bar, gen)) {
            if (threadIdx.x == 0) atomicExch(A.error, 1);
            if (threadIdx.x == 0 && rank == 0) sP.res[0].status = kDevTimeout;
            return;
        }
        if (A.server) {
            // copy x and the result to the caller's host buffers, then flag completion
            const T* xs = sP.x_out;
            for (int i = rank * kThreads + threadIdx.x; i < sP.K; i += A.team_size * kThreads) host_x[i] = xs[i];
            __threadfence_system();
            if (!grid_sync(bar, A.team_size, gen)) {
                if (threadIdx.x == 0) atomicExch(A.error, 1);
                return;
            }
            if (threadIdx.x == 0 && rank == 0) {
                *host_res = *sP.res;
                __threadfence_system();
                A.done[slot] = j + 1;
                __threadfence_system();
            }
        }
    }
}

// ------------------------------------------------------------ team geometry

// Team size: enough teams to keep every SM busy; a problem shared by fewer
// teams than SMs gets several CTAs.
static int pick_team_size(int n_jobs, int num_sms)
{
    int t = n_jobs >= num_sms ? 1 : std::max(1, num_sms / std::max(1, n_jobs));
    return std::min(t, 16);
}

}  // namespace ds

// ==================================================================== batch

struct ds_batch {
    ds_ctx* ctx;
    int dtype;
    int n_jobs;
    std::vector<int> order;            // job -> position in the caller's result array
    std::vector<int> job_inst, job_rhs;
    std::vector<const double*> lam_src;  // caller's lambda arrays (re-read before each run)
    int n_inst;
    std::vector<int> n_rhs;
    void* dmem;                        // device: team workspaces, jobs, lambdas, results, control
    size_t dbytes;
    void* hjobs;                       // pinned: job descriptors
    double* hlam;                      // pinned: lambdas in job order
    ds::DevResult* hres;               // pinned: results in job order
    void* djobs;
    double* dlam;
    ds::DevResult* dres;
    void* dctl;                        // bars + team_job + next_job + error
    size_t ctl_bytes;
    int* derr;
    void* args;                        // TeamArgs<T> (host copy)
    int grid, smem;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    bool use_graph;
    float ms_last;
};

namespace ds {

template <typename T>
static ds_status batch_create_t(ds_ctx* ctx, int n, const ds_dict* const* dicts, const void* const* Y,
                                const int* n_rhs, const double* const* lambdas, const ds_options* opt,
                                void* const* X_out, ds_batch* B)
{
    // problems (instance, rhs), instances ordered largest first
    std::vector<int> inst(n);
    std::iota(inst.begin(), inst.end(), 0);
    std::stable_sort(inst.begin(), inst.end(), [&](int a, int b) {
        return (double)dicts[a]->N * dicts[a]->K > (double)dicts[b]->N * dicts[b]->K;
    });
    std::vector<int> res_base(n, 0);
    for (int i = 1; i < n; i++) res_base[i] = res_base[i - 1] + n_rhs[i - 1];
    int n_jobs = 0, maxN = 1, maxK = 1, maxG = 1, maxgs = 1;
    for (int i = 0; i < n; i++) {
        n_jobs += n_rhs[i];
        maxN = std::max(maxN, (int)dicts[i]->N);
        maxK = std::max(maxK, (int)dicts[i]->K);
        maxG = std::max(maxG, dicts[i]->nG);
        maxgs = std::max(maxgs, dicts[i]->max_gsize);
    }
    B->n_jobs = n_jobs;
    const int team = pick_team_size(n_jobs, ctx->num_sms);
    const int n_teams = std::max(1, std::min(ctx->num_sms / team, n_jobs));
    // workspace of one team, sized for the largest problem
    DictDesc dmax = dict_desc(dicts[inst[0]]);
    dmax.N = maxN; dmax.K = maxK; dmax.nG = maxG; dmax.max_gsize = maxgs;
    dmax.is_group = maxgs > 1;
    Geometry gmax;
    ds_status st = geometry<T>(dmax, team, ctx->smem_optin, &gmax);
    if (st != DS_OK) return st;
    Ws<T> wtmp;
    double* ltmp;
    DevResult* rtmp;
    double* ctmp;
    const size_t ws_team = align_up(layout<T>(nullptr, dmax, gmax, 1, &wtmp, &ltmp, &rtmp, &ctmp), 256);
    const size_t jobs_bytes = align_up(sizeof(SolveP<T>) * n_jobs, 256);
    const size_t lam_bytes = align_up(sizeof(double) * n_jobs, 256);
    const size_t res_bytes = align_up(sizeof(DevResult) * n_jobs, 256);
    const size_t tws_bytes = align_up(sizeof(Ws<T>) * n_teams, 256);
    if (opt->alg == DS_FISTA) {
        st = ctx_fista_table(ctx, opt->max_iter);
        if (st != DS_OK) return st;
    }
    // the plan keeps its own copy of the FISTA table (the context's may be regrown)
    const size_t fista_bytes = align_up(sizeof(double) * 2 * (size_t)ctx->fista_n, 256);
    B->ctl_bytes = align_up(sizeof(GridBarrier) * n_teams + sizeof(int) * (n_teams + 2), 256);
    B->dbytes = ws_team * n_teams + jobs_bytes + lam_bytes + res_bytes + tws_bytes + B->ctl_bytes + fista_bytes;
    if (cudaMalloc(&B->dmem, B->dbytes) != cudaSuccess) {
        cudaGetLastError();
        B->dmem = nullptr;
        return DS_ERR_OOM;
    }
    if (cudaMallocHost(&B->hjobs, jobs_bytes) != cudaSuccess || cudaMallocHost((void**)&B->hlam, lam_bytes) != cudaSuccess ||
        cudaMallocHost((void**)&B->hres, res_bytes) != cudaSuccess)
        return DS_ERR_OOM;
    char* d = reinterpret_cast<char*>(B->dmem);
    char* wsbase = d;
    B->djobs = d + ws_team * n_teams;
    B->dlam = reinterpret_cast<double*>(d + ws_team * n_teams + jobs_bytes);
    B->dres = reinterpret_cast<DevResult*>(d + ws_team * n_teams + jobs_bytes + lam_bytes);
    Ws<T>* dtws = reinterpret_cast<Ws<T>*>(d + ws_team * n_teams + jobs_bytes + lam_bytes + res_bytes);
    B->dctl = d + ws_team * n_teams + jobs_bytes + lam_bytes + res_bytes + tws_bytes;
    GridBarrier* bars = reinterpret_cast<GridBarrier*>(B->dctl);
    int* team_job = reinterpret_cast<int*>(bars + n_teams);
    int* next_job = team_job + n_teams;
    B->derr = next_job + 1;
    double* dfista = reinterpret_cast<double*>(reinterpret_cast<char*>(B->dctl) + B->ctl_bytes);
    if (ctx->fista_n > 0 &&
        cudaMemcpy(dfista, ctx->fista, sizeof(double) * 2 * (size_t)ctx->fista_n, cudaMemcpyDeviceToDevice) != cudaSuccess)
        return DS_ERR_CUDA;
    // team workspaces
    std::vector<Ws<T>> tws(n_teams);
    for (int t = 0; t < n_teams; t++) layout<T>(wsbase + ws_team * t, dmax, gmax, 1, &tws[t], &ltmp, &rtmp, &ctmp);
    if (cudaMemcpy(dtws, tws.data(), sizeof(Ws<T>) * n_teams, cudaMemcpyHostToDevice) != cudaSuccess)
        return DS_ERR_CUDA;
    // problem descriptors
    SolveP<T>* hj = reinterpret_cast<SolveP<T>*>(B->hjobs);
    B->order.resize(n_jobs);
    B->job_inst.resize(n_jobs);
    B->job_rhs.resize(n_jobs);
    int j = 0;
    for (int ii = 0; ii < n; ii++) {
        const int i = inst[ii];
        const ds_dict* dc = dicts[i];
        DictDesc dd = dict_desc(dc);
        Geometry g;
        st = geometry<T>(dd, team, ctx->smem_optin, &g);
        if (st != DS_OK) return st;
        const size_t es = sizeof(T);
        for (int r = 0; r < n_rhs[i]; r++, j++) {
            SolveP<T> P;
            std::memset(&P, 0, sizeof(P));
            fill_params<T>(P, dd, g, opt);
            P.fista = dfista;
            P.fista_n = ctx->fista_n;
            P.y = reinterpret_cast<const T*>(reinterpret_cast<const char*>(Y[i]) + es * dc->N * r);
            P.n_lambda = 1;
            P.lambdas = B->dlam + j;
            P.x_out = reinterpret_cast<T*>(reinterpret_cast<char*>(X_out[i]) + es * dc->K * r);
            P.ldx = dc->K;
            P.res = B->dres + j;
            hj[j] = P;
            B->order[j] = res_base[i] + r;
            B->job_inst[j] = i;
            B->job_rhs[j] = r;
        }
    }
    B->lam_src.assign(lambdas, lambdas + n);
    B->n_inst = n;
    B->n_rhs.assign(n_rhs, n_rhs + n);
    // the persistent launch
    TeamArgs<T>* A = new TeamArgs<T>();
    std::memset(A, 0, sizeof(*A));
    A->jobs = reinterpret_cast<SolveP<T>*>(B->djobs);
    A->n_jobs = n_jobs;
    A->team_ws = dtws;
    A->bars = bars;
    A->team_job = team_job;
    A->next_job = next_job;
    A->error = B->derr;
    A->team_size = team;
    A->server = 0;
    B->args = A;
    B->grid = n_teams * team;
    B->smem = (int)gmax.smem;
    if (cudaFuncSetAttribute(team_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(ctx->smem_optin - 40 * 1024)) != cudaSuccess)
        return DS_ERR_CUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, team_kernel<T>, kThreads, B->smem) != cudaSuccess || occ < 1)
        return DS_ERR_UNSUPPORTED;
    return DS_OK;
}

// Device work of one run, in stream order (captured into the graph).
template <typename T>
static ds_status batch_enqueue_t(ds_batch* B, cudaStream_t s)
{
    TeamArgs<T>* A = reinterpret_cast<TeamArgs<T>*>(B->args);
    if (cudaMemcpyAsync(B->djobs, B->hjobs, sizeof(SolveP<T>) * B->n_jobs, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaMemcpyAsync(B->dlam, B->hlam, sizeof(double) * B->n_jobs, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaMemsetAsync(B->dctl, 0, B->ctl_bytes, s) != cudaSuccess) return DS_ERR_CUDA;
    if (cudaMemsetAsync(B->dres, 0, sizeof(DevResult) * B->n_jobs, s) != cudaSuccess) return DS_ERR_CUDA;
    void* args[] = {(void*)A};
    if (cudaLaunchCooperativeKernel((const void*)team_kernel<T>, dim3(B->grid), dim3(kThreads), args, B->smem, s) !=
        cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaMemcpyAsync(B->hres, B->dres, sizeof(DevResult) * B->n_jobs, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return DS_ERR_CUDA;
    return DS_OK;
}

static ds_status batch_enqueue(ds_batch* B, cudaStream_t s)
{
    return B->dtype == DS_FP32 ? batch_enqueue_t<float>(B, s) : batch_enqueue_t<double>(B, s);
}

}  // namespace ds

extern "C" {

ds_status ds_batch_destroy(ds_batch* B)
{
    if (!B) return DS_OK;
    if (B->ctx) {
        cudaSetDevice(B->ctx->device);
        cudaStreamSynchronize(B->ctx->stream);
    }
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->dmem) cudaFree(B->dmem);
    if (B->hjobs) cudaFreeHost(B->hjobs);
    if (B->hlam) cudaFreeHost(B->hlam);
    if (B->hres) cudaFreeHost(B->hres);
    if (B->args) {
        if (B->dtype == DS_FP32) delete reinterpret_cast<ds::TeamArgs<float>*>(B->args);
        else delete reinterpret_cast<ds::TeamArgs<double>*>(B->args);
    }
    delete B;
    return DS_OK;
}

ds_status ds_batch_create(ds_ctx* ctx, int n, const ds_dict* const* dicts, const void* const* Y, const int* n_rhs,
                          const double* const* lambdas, const ds_options* opt, void* const* X_out, ds_batch** out)
{
    if (!ctx || n < 1 || !dicts || !Y || !n_rhs || !lambdas || !opt || !X_out || !out) return DS_ERR_INVALID;
    *out = nullptr;
    if (opt->max_iter < 1 || !(opt->tol_gap_rel >= 0.0) || opt->test < DS_TEST_NONE || opt->test > DS_DGST3 ||
        (opt->alg != DS_ISTA && opt->alg != DS_FISTA) || opt->L < 0.0)
        return DS_ERR_INVALID;
    const int dtype = dicts[0] ? dicts[0]->dtype : -1;
    for (int i = 0; i < n; i++) {
        if (!dicts[i] || dicts[i]->ctx != ctx || dicts[i]->dtype != dtype || !Y[i] || !X_out[i] || !lambdas[i] ||
            n_rhs[i] < 1)
            return DS_ERR_INVALID;
        if (dicts[i]->is_group && (opt->test == DS_SAFE || opt->test == DS_DST3 || opt->test == DS_DOME))
            return DS_ERR_INVALID;
        for (int r = 0; r < n_rhs[i]; r++)
            if (!(lambdas[i][r] > 0.0)) return DS_ERR_INVALID;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return DS_ERR_CUDA;
    ds_batch* B = new (std::nothrow) ds_batch();
    if (!B) return DS_ERR_OOM;
    B->ctx = ctx;
    B->dtype = dtype;
    ds_status st = dtype == DS_FP32 ? ds::batch_create_t<float>(ctx, n, dicts, Y, n_rhs, lambdas, opt, X_out, B)
                                    : ds::batch_create_t<double>(ctx, n, dicts, Y, n_rhs, lambdas, opt, X_out, B);
    if (st != DS_OK) {
        ds_batch_destroy(B);
        return st;
    }
    // capture the run once into a CUDA graph; runs replay it
    B->use_graph = false;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) {
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            ds_status es = ds::batch_enqueue(B, cs);
            cudaGraph_t g = nullptr;
            cudaError_t ec = cudaStreamEndCapture(cs, &g);
            if (es == DS_OK && ec == cudaSuccess && g && cudaGraphInstantiate(&B->exec, g, 0) == cudaSuccess) {
                B->graph = g;
                B->use_graph = true;
            } else {
                if (g) cudaGraphDestroy(g);
                B->exec = nullptr;
            }
        }
        cudaGetLastError();
        cudaStreamDestroy(cs);
    }
    *out = B;
    return DS_OK;
}

ds_status ds_batch_run(ds_batch* B, ds_result* res)
{
    if (!B || !res) return DS_ERR_INVALID;
    if (cudaSetDevice(B->ctx->device) != cudaSuccess) return DS_ERR_CUDA;
    for (int j = 0; j < B->n_jobs; j++) B->hlam[j] = B->lam_src[B->job_inst[j]][B->job_rhs[j]];
    cudaStream_t s = B->ctx->stream;
    cudaEventRecord(B->ctx->ev0, s);
    if (B->use_graph) {
        if (cudaGraphLaunch(B->exec, s) != cudaSuccess) return DS_ERR_CUDA;
    } else {
        ds_status st = ds::batch_enqueue(B, s);
        if (st != DS_OK) return st;
    }
    cudaEventRecord(B->ctx->ev1, s);
    B->ctx->launches++;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DS_ERR_CUDA;
    cudaEventElapsedTime(&B->ms_last, B->ctx->ev0, B->ctx->ev1);
    int err = 0;
    if (cudaMemcpy(&err, B->derr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DS_ERR_CUDA;
    for (int j = 0; j < B->n_jobs; j++) {
        const ds::DevResult& r = B->hres[j];
        ds_result& o = res[B->order[j]];
        o.iters = r.iters;
        o.status = r.status;
        o.n_active = r.n_active;
        o.nnz = r.nnz;
        o.gap = r.gap;
        o.primal = r.primal;
        o.dual = r.dual;
        o.lambda = r.lambda;
        o.lambda_max = r.lambda_max;
        o.ms = B->ms_last;
        o.cols_corr = r.cols_corr;
        o.cols_synth = r.cols_synth;
    }
    return err ? DS_ERR_TIMEOUT : DS_OK;
}

ds_status ds_batch_info(const ds_batch* B, int* uses_graph, int* teams, int* team_size)
{
    if (!B) return DS_ERR_INVALID;
    const int ts = B->dtype == DS_FP32 ? reinterpret_cast<ds::TeamArgs<float>*>(B->args)->team_size
                                       : reinterpret_cast<ds::TeamArgs<double>*>(B->args)->team_size;
    if (uses_graph) *uses_graph = B->use_graph ? 1 : 0;
    if (team_size) *team_size = ts;
    if (teams) *teams = B->grid / ts;
    return DS_OK;
}

ds_status ds_solve_batch(ds_ctx* ctx, int n, const ds_dict* const* dicts, const void* const* Y, const int* n_rhs,
                         const double* const* lambdas, const ds_options* opt, void* const* X_out, ds_result* res)
{
    if (!res) return DS_ERR_INVALID;
    ds_batch* B = nullptr;
    ds_status st = ds_batch_create(ctx, n, dicts, Y, n_rhs, lambdas, opt, X_out, &B);
    if (st != DS_OK) return st;
    st = ds_batch_run(B, res);
    ds_batch_destroy(B);
    return st;
}

}  // extern "C"
