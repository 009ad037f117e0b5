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
#include <atomic>
#include <chrono>
#include <map>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "ds_solve_body.cuh"

namespace ds {

constexpr unsigned long long kServerWaitNs = 120000000000ull;  // 120 s

// A served request: solve parameters (with the request's own workspace, carved
// from the server's memory pool) and device staging for y, x and the result.
template <typename T>
struct ServerJob {
    SolveP<T> P;  // P.y, P.x_out, P.res point to mapped host memory; P.ws to the request's pool block
    T* y_dev;
    T* x_dev;
    DevResult* res_dev;
};

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
    ServerJob<T>* ring;             // mapped host: request descriptors, one per slot
    long long idle_polls;           // server: a team counts itself idle after this many empty polls
    int n_teams;                    // server: teams of the launch
    int* idle_teams;                // server: teams counted idle (zeroed per launch)
    int* exiting;                   // server: set when every team was idle (zeroed per launch)
};

__device__ __forceinline__ int ld_acquire_sys(const volatile int* p)
{
    int v;
    asm volatile("ld.acquire.sys.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ADAPT: the solves may use the adaptive-step rows (backtracking, SpaRSA, TwIST); a batch of fixed-step
// solves launches the instance without that code, the server (any request) the one with it.
template <typename T, bool ADAPT = true>
__global__ void __launch_bounds__(kThreads, 1) team_kernel(const TeamArgs<T> A)
{
    __shared__ SolveP<T> sP;
    __shared__ T* s_stage[2];
    __shared__ DevResult* s_res_dev;
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
                // the launch ends only when every team is idle: a team that has waited long enough
                // counts itself idle (and uncounts itself if work arrives); the team that sees all
                // teams idle raises `exiting`, which takes every team out, and the host relaunches on
                // the next request.  (A team leaving on its own would leave the rest of the launch
                // to its remaining teams, which would then serve every later request.)
                long long polls = 0;
                bool counted = false;
                while (!*A.stop) {
                    if (atomicAdd(A.exiting, 0)) break;
                    const int head = atomicAdd(A.next_job, 0);
                    if (head < ld_acquire_sys(A.published)) {
                        if (counted) {
                            atomicSub(A.idle_teams, 1);
                            counted = false;
                        }
                        if (atomicCAS(A.next_job, head, head + 1) == head) {
                            j = head;
                            break;
                        }
                        continue;
                    }
                    if (++polls > A.idle_polls && !counted) {
                        atomicAdd(A.idle_teams, 1);
                        counted = true;
                    }
                    if (counted && atomicAdd(A.idle_teams, 0) >= A.n_teams) {
                        atomicExch(A.exiting, 1);
                        break;
                    }
                    __nanosleep(polls < 64 ? 200 : 2000);
                }
            }
            A.team_job[team] = j;
        }
        // the team's other CTAs wait here while its leader looks for work, which may last as long as
        // another team's solve: this wait gets a longer limit than the barriers inside a solve
        if (!grid_sync(bar, A.team_size, gen, kServerWaitNs)) {
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
                const volatile unsigned int* src = reinterpret_cast<const volatile unsigned int*>(A.ring + slot);
                ServerJob<T> job;
                unsigned int* dst = reinterpret_cast<unsigned int*>(&job);
                for (int k = 0; k < (int)(sizeof(ServerJob<T>) / 4); k++) dst[k] = src[k];
                sP = job.P;
                s_stage[0] = job.y_dev;
                s_stage[1] = job.x_dev;
                s_res_dev = job.res_dev;
            } else {
                sP = A.jobs[slot];
                sP.ws = A.team_ws[team];
            }
        }
        __syncthreads();
        if (A.server) {
            // stage y in device memory; x and the result go to device staging, copied out at the end
            T* ys = s_stage[0];
            const volatile T* yh = sP.y;
            for (int r = rank * kThreads + threadIdx.x; r < sP.N; r += A.team_size * kThreads) ys[r] = yh[r];
            host_x = sP.x_out;
            host_res = sP.res;
            __syncthreads();
            if (threadIdx.x == 0) {
                sP.y = ys;
                sP.x_out = s_stage[1];
                sP.ldx = sP.K;
                sP.res = s_res_dev;
            }
            if (!grid_sync(bar, A.team_size, gen)) {
                if (threadIdx.x == 0) atomicExch(A.error, 1);
                return;
            }
        }
        if (!solve_body<T, ADAPT>(sP, rank, A.team_size, bar, gen)) {
            if (threadIdx.x == 0) atomicExch(A.error, 1);
            if (threadIdx.x == 0 && rank == 0) sP.res[0].status = kDevTimeout;
            return;
        }
        if (A.server) {
            // copy x and the result to the caller's host buffers, then flag completion; every CTA wrote its
            // own slice of x, so the team barrier comes before any CTA copies another's entries
            if (!grid_sync(bar, A.team_size, gen)) {
                if (threadIdx.x == 0) atomicExch(A.error, 1);
                return;
            }
            const T* xs = sP.x_out;
            for (int i = rank * kThreads + threadIdx.x; i < sP.K; i += A.team_size * kThreads) host_x[i] = __ldcg(xs + i);
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

template <typename T>
static const void* team_fn(bool adapt)
{
    return adapt ? (const void*)team_kernel<T, true> : (const void*)team_kernel<T, false>;
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
    bool adapt = false;  // the problems use an adaptive-step row (the team kernel with that code)
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
    ds::MrhsPlan* mplan;  // right-hand sides solved together (FP32 Lasso instances)
    double* mfista;       // the multi-rhs plan's copy of the FISTA table
    // schedule of the multi-rhs blocks (chosen by ds_batch_autotune) and the creation
    // arguments, kept so that the autotuner can build the other candidates
    struct Cfg {
        int allow_tc = 1;       // tensor-core bulk phase on BF16 copies
        int block_r = 64;       // right-hand sides per block
        int sort_lambda = 0;    // group right-hand sides of similar lambda into a block
        double lo_switch = 0;   // > 0: bulk-to-FP32 switch level
    } cfg;
    std::vector<const ds_dict*> c_dicts;
    std::vector<const void*> c_Y;
    std::vector<void*> c_X;
    ds_options c_opt;
};

namespace ds {

template <typename T>
static ds_status batch_create_t(ds_ctx* ctx, int n, const ds_dict* const* dicts, const void* const* Y,
                                const int* n_rhs, const double* const* lambdas, const ds_options* opt,
                                void* const* X_out, ds_batch* B)
{
    const ds_batch::Cfg& cfg = B->cfg;
    if (opt->alg == DS_FISTA) {
        ds_status fs = ctx_fista_table(ctx, opt->max_iter);
        if (fs != DS_OK) return fs;
    }
    // instances whose right-hand sides are solved together (FP32 Lasso, tests of Lemmas 2-4)
    std::vector<char> multi(n, 0);
    std::vector<MrhsBlock> blocks;
    for (int i = 0; i < n; i++) {
        multi[i] = sizeof(T) == 4 && opt->batch_multi_rhs && !dicts[i]->is_group && opt->test <= DS_DOME &&
                   (opt->alg == DS_ISTA || opt->alg == DS_FISTA) && !opt->step_backtracking && n_rhs[i] >= 2;
        if (!multi[i]) continue;
        // right-hand sides in order, or sorted by lambda (similar iteration counts and
        // screened sets in a block: a tighter union list and fewer idle slots)
        std::vector<int> ord(n_rhs[i]);
        std::iota(ord.begin(), ord.end(), 0);
        if (cfg.sort_lambda)
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return lambdas[i][a] < lambdas[i][b]; });
        const int br = std::max(2, std::min(kMrhsMaxR, cfg.block_r));
        for (int r0 = 0; r0 < n_rhs[i]; r0 += br) {
            MrhsBlock blk;
            std::memset(&blk, 0, sizeof(blk));
            blk.dict = dicts[i];
            blk.R = std::min(br, n_rhs[i] - r0);
            blk.Y = Y[i];
            blk.X = X_out[i];
            blk.inst = i;
            for (int r = 0; r < blk.R; r++) blk.ridx[r] = ord[r0 + r];
            blocks.push_back(blk);
        }
    }
    // problems (instance, rhs) of the other instances, instances ordered largest first
    std::vector<int> inst;
    for (int i = 0; i < n; i++)
        if (!multi[i]) inst.push_back(i);
    std::stable_sort(inst.begin(), inst.end(), [&](int a, int b) {
        return (double)dicts[a]->N * dicts[a]->K > (double)dicts[b]->N * dicts[b]->K;
    });
    std::vector<int> res_base(n, 0);
    for (int i = 1; i < n; i++) res_base[i] = res_base[i - 1] + n_rhs[i - 1];
    B->lam_src.assign(lambdas, lambdas + n);
    B->n_inst = n;
    B->n_rhs.assign(n_rhs, n_rhs + n);
    if (!blocks.empty()) {
        // the plan copies the FISTA table pointer: the context's table stays valid while the plan
        // lives (it only grows on later calls), so take a private copy below as for the teams
        ds_status ms = DS_OK;
        double* mf = nullptr;
        if (ctx->fista_n > 0) {
            if (cudaMalloc(&mf, sizeof(double) * 2 * (size_t)ctx->fista_n) != cudaSuccess) {
                cudaGetLastError();
                return DS_ERR_OOM;
            }
            B->mfista = mf;
            if (cudaMemcpy(mf, ctx->fista, sizeof(double) * 2 * (size_t)ctx->fista_n, cudaMemcpyDeviceToDevice) !=
                cudaSuccess)
                return DS_ERR_CUDA;
        }
        MrhsCfg mc;
        mc.allow_tc = cfg.allow_tc;
        mc.lo_switch = cfg.lo_switch;
        mc.team_size = opt->team_size;
        ms = mrhs_plan_create(ctx, (int)blocks.size(), blocks.data(), opt, mf, ctx->fista_n, mc, &B->mplan);
        if (ms != DS_OK) return ms;
    }
    int n_jobs = 0, maxN = 1, maxK = 1, maxG = 1, maxgs = 1;
    for (int i : inst) {
        n_jobs += n_rhs[i];
        maxN = std::max(maxN, (int)dicts[i]->N);
        maxK = std::max(maxK, (int)dicts[i]->K);
        maxG = std::max(maxG, dicts[i]->nG);
        maxgs = std::max(maxgs, dicts[i]->max_gsize);
    }
    B->n_jobs = n_jobs;
    if (n_jobs == 0) return DS_OK;
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
    for (int ii = 0; ii < (int)inst.size(); ii++) {
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
    B->adapt = opt->alg == DS_SPARSA || opt->alg == DS_TWIST || opt->step_backtracking;
    const void* kfn = team_fn<T>(B->adapt);
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(ctx->smem_optin - 40 * 1024)) != cudaSuccess)
        return DS_ERR_CUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kThreads, B->smem) != cudaSuccess || occ < 1)
        return DS_ERR_UNSUPPORTED;
    return DS_OK;
}

// Device work of one run, in stream order (captured into the graph).
template <typename T>
static ds_status batch_enqueue_t(ds_batch* B, cudaStream_t s)
{
    if (B->mplan) {
        ds_status ms = mrhs_plan_enqueue(B->mplan, s);
        if (ms != DS_OK) return ms;
    }
    if (B->n_jobs == 0) return DS_OK;
    TeamArgs<T>* A = reinterpret_cast<TeamArgs<T>*>(B->args);
    if (cudaMemcpyAsync(B->djobs, B->hjobs, sizeof(SolveP<T>) * B->n_jobs, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaMemcpyAsync(B->dlam, B->hlam, sizeof(double) * B->n_jobs, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaMemsetAsync(B->dctl, 0, B->ctl_bytes, s) != cudaSuccess) return DS_ERR_CUDA;
    if (cudaMemsetAsync(B->dres, 0, sizeof(DevResult) * B->n_jobs, s) != cudaSuccess) return DS_ERR_CUDA;
    void* args[] = {(void*)A};
    if (cudaLaunchCooperativeKernel(team_fn<T>(B->adapt), dim3(B->grid), dim3(kThreads), args, B->smem, s) !=
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
    if (B->mplan) ds::mrhs_plan_destroy(B->mplan);
    if (B->mfista) cudaFree(B->mfista);
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

static ds_status batch_create_cfg(ds_ctx* ctx, int n, const ds_dict* const* dicts, const void* const* Y,
                                  const int* n_rhs, const double* const* lambdas, const ds_options* opt,
                                  void* const* X_out, const ds_batch::Cfg& cfg, ds_batch** out)
{
    if (!ctx || n < 1 || !dicts || !Y || !n_rhs || !lambdas || !opt || !X_out || !out) return DS_ERR_INVALID;
    *out = nullptr;
    if (opt->max_iter < 1 || !(opt->tol_gap_rel >= 0.0) || opt->test < DS_TEST_NONE || opt->test > DS_DGST3 ||
        opt->alg < DS_ISTA || opt->alg > DS_TWIST || opt->L < 0.0 || opt->team_size < 0)
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
    B->cfg = cfg;
    B->c_dicts.assign(dicts, dicts + n);
    B->c_Y.assign(Y, Y + n);
    B->c_X.assign(X_out, X_out + n);
    B->c_opt = *opt;
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

ds_status ds_batch_create(ds_ctx* ctx, int n, const ds_dict* const* dicts, const void* const* Y, const int* n_rhs,
                          const double* const* lambdas, const ds_options* opt, void* const* X_out, ds_batch** out)
{
    return batch_create_cfg(ctx, n, dicts, Y, n_rhs, lambdas, opt, X_out, ds_batch::Cfg(), out);
}

ds_status ds_batch_run(ds_batch* B, ds_result* res)
{
    if (!B || !res) return DS_ERR_INVALID;
    if (cudaSetDevice(B->ctx->device) != cudaSuccess) return DS_ERR_CUDA;
    for (int j = 0; j < B->n_jobs; j++) B->hlam[j] = B->lam_src[B->job_inst[j]][B->job_rhs[j]];
    int nb = 0;
    const ds::MrhsBlock* blks = B->mplan ? ds::mrhs_plan_blocks(B->mplan, &nb) : nullptr;
    if (B->mplan) {
        double* ml = ds::mrhs_plan_lambdas(B->mplan);
        for (int j = 0; j < nb; j++)
            for (int r = 0; r < blks[j].R; r++) ml[(size_t)j * ds::kMrhsMaxR + r] = B->lam_src[blks[j].inst][blks[j].ridx[r]];
    }
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
    if (B->n_jobs > 0 && cudaMemcpy(&err, B->derr, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return DS_ERR_CUDA;
    if (B->mplan) {
        int merr = 0;
        if (cudaMemcpy(&merr, ds::mrhs_plan_error_flag(B->mplan), sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return DS_ERR_CUDA;
        err |= merr;
        const ds::DevResult* mr = ds::mrhs_plan_results(B->mplan);
        std::vector<int> base(B->n_inst, 0);
        for (int i = 1; i < B->n_inst; i++) base[i] = base[i - 1] + B->n_rhs[i - 1];
        for (int j = 0; j < nb; j++)
            for (int r = 0; r < blks[j].R; r++) {
                const ds::DevResult& q = mr[(size_t)j * ds::kMrhsMaxR + r];
                ds_result& o = res[base[blks[j].inst] + blks[j].ridx[r]];
                o.iters = q.iters;
                o.status = q.status;
                o.n_active = q.n_active;
                o.nnz = q.nnz;
                o.gap = q.gap;
                o.primal = q.primal;
                o.dual = q.dual;
                o.lambda = q.lambda;
                o.lambda_max = q.lambda_max;
                o.ms = B->ms_last;
                o.cols_corr = q.cols_corr;
                o.cols_synth = q.cols_synth;
                o.cols_lowp = q.cols_lowp;
            }
    }
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
    if (uses_graph) *uses_graph = B->use_graph ? 1 : 0;
    if (B->n_jobs == 0) {  // every instance runs in the multi-rhs kernel
        ds::mrhs_plan_info(B->mplan, teams, team_size);
        return DS_OK;
    }
    const int ts = B->dtype == DS_FP32 ? reinterpret_cast<ds::TeamArgs<float>*>(B->args)->team_size
                                       : reinterpret_cast<ds::TeamArgs<double>*>(B->args)->team_size;
    if (team_size) *team_size = ts;
    if (teams) *teams = B->grid / ts;
    return DS_OK;
}

ds_status ds_batch_schedule(const ds_batch* B, int* tensor_bulk, int* block_rhs, int* sort_lambda, double* lowp_switch)
{
    if (!B) return DS_ERR_INVALID;
    if (tensor_bulk) *tensor_bulk = B->cfg.allow_tc;
    if (block_rhs) *block_rhs = B->cfg.block_r;
    if (sort_lambda) *sort_lambda = B->cfg.sort_lambda;
    if (lowp_switch) *lowp_switch = B->cfg.lo_switch;
    return DS_OK;
}

ds_status ds_batch_autotune(ds_batch* B, int max_candidates, int* chosen, int* n_tried, float* ms_tried)
{
    if (!B || max_candidates < 1) return DS_ERR_INVALID;
    const int n = (int)B->c_dicts.size();
    bool bf16 = false, multi = false;
    int total = 0;
    for (int i = 0; i < n; i++) {
        total += B->n_rhs[i];
        bf16 |= B->c_dicts[i]->lo_kind == 1;
        multi |= B->n_rhs[i] >= 2;
    }
    // candidate schedules of the multi-rhs blocks; the plan's own schedule first
    std::vector<ds_batch::Cfg> cands;
    auto add = [&](int tc, int br, int sorted, double sw) {
        ds_batch::Cfg c;
        c.allow_tc = tc;
        c.block_r = br;
        c.sort_lambda = sorted;
        c.lo_switch = sw;
        for (const auto& d : cands)
            if (d.allow_tc == c.allow_tc && d.block_r == c.block_r && d.sort_lambda == c.sort_lambda &&
                d.lo_switch == c.lo_switch)
                return;
        cands.push_back(c);
    };
    cands.push_back(B->cfg);
    if (multi) {
        add(B->cfg.allow_tc, 32, 1, B->cfg.lo_switch);
        if (bf16) {
            add(1 - B->cfg.allow_tc, B->cfg.block_r, B->cfg.sort_lambda, B->cfg.lo_switch);
            add(1 - B->cfg.allow_tc, 32, 1, B->cfg.lo_switch);
            add(1, 64, 0, 1e-2);
        }
    }
    if ((int)cands.size() > max_candidates) cands.resize(max_candidates);
    std::vector<ds_result> res(total);
    int best = 0;
    float best_ms = 0.f;
    ds_batch* best_plan = nullptr;  // a candidate that beats the plan's own schedule
    for (int k = 0; k < (int)cands.size(); k++) {
        ds_batch* P = B;
        if (k > 0) {
            ds_status st = batch_create_cfg(B->ctx, n, B->c_dicts.data(), B->c_Y.data(), B->n_rhs.data(),
                                            B->lam_src.data(), &B->c_opt, B->c_X.data(), cands[k], &P);
            if (st != DS_OK) {
                if (ms_tried) ms_tried[k] = -1.f;
                continue;
            }
        }
        ds_status st = ds_batch_run(P, res.data());
        const float ms = st == DS_OK ? P->ms_last : -1.f;
        if (ms_tried) ms_tried[k] = ms;
        const bool better = st == DS_OK && (k == 0 || (ms > 0.f && ms < best_ms));
        if (better) {
            best = k;
            best_ms = ms;
            if (k > 0) {
                if (best_plan) ds_batch_destroy(best_plan);
                best_plan = P;
                P = nullptr;
            }
        }
        if (k > 0 && P) ds_batch_destroy(P);
        if (k == 0 && st != DS_OK) return st;
    }
    if (best_plan) {
        // the batch takes over the faster plan; its old internals go with the candidate
        std::swap(*B, *best_plan);
        ds_batch_destroy(best_plan);
    }
    if (chosen) *chosen = best;
    if (n_tried) *n_tried = (int)cands.size();
    return DS_OK;
}

ds_status ds_batch_layout(const ds_batch* B, int* multi_rhs_blocks, int* multi_rhs_teams, int* multi_rhs_team_size,
                          int* single_problems)
{
    if (!B) return DS_ERR_INVALID;
    int nb = 0, t = 0, ts = 0;
    if (B->mplan) {
        ds::mrhs_plan_blocks(B->mplan, &nb);
        ds::mrhs_plan_info(B->mplan, &t, &ts);
    }
    if (multi_rhs_blocks) *multi_rhs_blocks = nb;
    if (multi_rhs_teams) *multi_rhs_teams = t;
    if (multi_rhs_team_size) *multi_rhs_team_size = ts;
    if (single_problems) *single_problems = B->n_jobs;
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

// =================================================================== server

namespace ds {

// First-fit allocator of 256-byte aligned blocks in the server's device pool.
class PoolAlloc {
  public:
    void init(size_t size)
    {
        free_.clear();
        free_[0] = size;
    }
    bool alloc(size_t n, size_t* off)
    {
        n = align_up(n, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, o2 = it->first + n;
            free_.erase(it);
            if (rest) free_[o2] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = align_up(n, 256);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<size_t, size_t> free_;
};

static double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace ds

struct ds_server {
    struct Ticket {
        int64_t seq = -1;   // publication order (-1: pending)
        int slot = -1;
        size_t off = 0, bytes = 0;
        void* x_out = nullptr;
        std::vector<float> y;  // copy of y while pending
        const ds_dict* dict = nullptr;
        double lambda = 0.0;
        ds_options opt;
        double t_submit = 0.0;
        int state = 0;  // 0 pending, 1 published, 2 done
        ds_result res;
    };
    ds_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    int team_size = 0, n_teams = 0, ring = 0;
    int64_t max_N = 0, max_K = 0;
    size_t budget = 0, in_use = 0;
    void* pool = nullptr;
    ds::PoolAlloc alloc;
    ds::ServerJob<float>* ring_h = nullptr;
    ds::ServerJob<float>* ring_d = nullptr;
    double* lam_h = nullptr;
    double* lam_d = nullptr;
    float* y_h = nullptr;
    float* y_d = nullptr;
    float* x_h = nullptr;
    float* x_d = nullptr;
    ds::DevResult* res_h = nullptr;
    ds::DevResult* res_d = nullptr;
    int* done_h = nullptr;
    int* done_d = nullptr;
    int* ctl_h = nullptr;  // [0] published, [1] stop
    int* ctl_d = nullptr;
    void* dctl = nullptr;  // bars, team_job, next_job, error
    size_t dctl_bytes = 0, bars_bytes = 0;
    int* derr = nullptr;
    double* fista = nullptr;
    int fista_n = 0;
    ds::TeamArgs<float> args;
    int smem = 0;
    std::unordered_map<uint64_t, Ticket> tickets;
    std::deque<uint64_t> pending;
    bool adapt_launch = false;  // the running (or next) launch is the instance with the adaptive-step code
    std::vector<int64_t> slot_seq;
    std::vector<uint64_t> slot_ticket;
    uint64_t next_ticket = 1;
    int64_t published = 0;
    int64_t completed = 0;
    long long launches = 0;
    std::mutex mu;
};

namespace ds {

static size_t request_bytes(ds_server* S, const ds_dict* d, const ds_options* opt, Geometry* g_out, DictDesc* dd_out)
{
    DictDesc dd = dict_desc(d);
    Geometry g;
    if (geometry<float>(dd, S->team_size, S->ctx->smem_optin, &g) != DS_OK) return 0;
    Ws<float> w;
    double* l;
    DevResult* r;
    double* c;
    size_t b = align_up(layout<float>(nullptr, dd, g, 1, &w, &l, &r, &c), 256);
    b += align_up(sizeof(float) * d->N, 256) + align_up(sizeof(float) * d->K, 256) + align_up(sizeof(DevResult), 256);
    (void)opt;
    *g_out = g;
    *dd_out = dd;
    return b;
}

// Publish a pending request if its ring slot is free and the pool has room.
static bool server_publish(ds_server* S, uint64_t tid, ds_server::Ticket& t, const float* y_src)
{
    const int64_t seq = S->published;
    const int slot = (int)(seq % S->ring);
    if (S->slot_seq[slot] >= 0) return false;  // previous occupant not harvested yet
    Geometry g;
    DictDesc dd;
    const size_t bytes = request_bytes(S, t.dict, &t.opt, &g, &dd);
    size_t off = 0;
    if (!bytes || !S->alloc.alloc(bytes, &off)) return false;  // admission by HBM footprint
    char* blk = reinterpret_cast<char*>(S->pool) + off;
    Ws<float> w;
    double* l;
    DevResult* r;
    double* c;
    const size_t wsb = align_up(layout<float>(blk, dd, g, 1, &w, &l, &r, &c), 256);
    ServerJob<float> job;
    std::memset(&job, 0, sizeof(job));
    fill_params<float>(job.P, dd, g, &t.opt);
    job.P.fista = S->fista;
    job.P.fista_n = S->fista_n;
    job.P.n_lambda = 1;
    job.P.lambdas = S->lam_d + slot;
    job.P.y = S->y_d + (size_t)slot * S->max_N;
    job.P.x_out = S->x_d + (size_t)slot * S->max_K;
    job.P.ldx = t.dict->K;
    job.P.res = S->res_d + slot;
    job.P.ws = w;
    job.P.abort_flag = S->ctl_d + 1;  // the stop flag: destroy ends in-flight solves
    job.y_dev = reinterpret_cast<float*>(blk + wsb);
    job.x_dev = reinterpret_cast<float*>(blk + wsb + align_up(sizeof(float) * t.dict->N, 256));
    job.res_dev = reinterpret_cast<DevResult*>(blk + wsb + align_up(sizeof(float) * t.dict->N, 256) +
                                               align_up(sizeof(float) * t.dict->K, 256));
    S->lam_h[slot] = t.lambda;
    std::memcpy(S->y_h + (size_t)slot * S->max_N, y_src, sizeof(float) * t.dict->N);
    S->ring_h[slot] = job;
    reinterpret_cast<volatile int*>(S->done_h)[slot] = 0;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    reinterpret_cast<volatile int*>(S->ctl_h)[0] = (int)(seq + 1);
    std::atomic_thread_fence(std::memory_order_seq_cst);
    S->published = seq + 1;
    S->slot_seq[slot] = seq;
    S->slot_ticket[slot] = tid;
    S->in_use += bytes;
    t.seq = seq;
    t.slot = slot;
    t.off = off;
    t.bytes = bytes;
    t.state = 1;
    t.y.clear();
    t.y.shrink_to_fit();
    return true;
}

static void server_harvest(ds_server* S)
{
    std::atomic_thread_fence(std::memory_order_seq_cst);
    for (int slot = 0; slot < S->ring; slot++) {
        const int64_t seq = S->slot_seq[slot];
        if (seq < 0) continue;
        if (reinterpret_cast<volatile int*>(S->done_h)[slot] != (int)(seq + 1)) continue;
        std::atomic_thread_fence(std::memory_order_seq_cst);
        auto it = S->tickets.find(S->slot_ticket[slot]);
        if (it != S->tickets.end()) {
            ds_server::Ticket& t = it->second;
            std::memcpy(t.x_out, S->x_h + (size_t)slot * S->max_K, sizeof(float) * t.dict->K);
            const DevResult& r = S->res_h[slot];
            t.res.iters = r.iters;
            t.res.status = r.status;
            t.res.n_active = r.n_active;
            t.res.nnz = r.nnz;
            t.res.gap = r.gap;
            t.res.primal = r.primal;
            t.res.dual = r.dual;
            t.res.lambda = r.lambda;
            t.res.lambda_max = r.lambda_max;
            t.res.cols_corr = r.cols_corr;
            t.res.cols_synth = r.cols_synth;
            t.res.cols_lowp = r.cols_lowp;
            t.res.ms = now_ms() - t.t_submit;  // latency: submission to completion observed by the host
            t.state = 2;
            S->alloc.release(t.off, t.bytes);
            S->in_use -= t.bytes;
        }
        S->slot_seq[slot] = -1;
        S->completed++;
    }
}

static ds_status server_launch(ds_server* S)
{
    // counters of the previous launch: barriers restart, the queue head persists
    if (cudaMemsetAsync(S->dctl, 0, S->bars_bytes, S->stream) != cudaSuccess) return DS_ERR_CUDA;
    void* a[] = {(void*)&S->args};
    const int grid = S->n_teams * S->team_size;
    if (cudaLaunchCooperativeKernel(team_fn<float>(S->adapt_launch), dim3(grid), dim3(kThreads), a, S->smem,
                                    S->stream) != cudaSuccess)
        return DS_ERR_CUDA;
    S->launches++;
    S->ctx->launches++;
    return DS_OK;
}

static bool adaptive_request(const ds_options& o)
{
    return o.alg == DS_SPARSA || o.alg == DS_TWIST || o.step_backtracking;
}

static ds_status server_pump(ds_server* S)
{
    server_harvest(S);
    // fixed-step requests run on the kernel instance without the adaptive-step code; when no launch is
    // running and nothing published is outstanding, the request at the head of the queue picks the
    // instance of the next launch, and an adaptive request waits for a launch of the other instance
    const cudaError_t q0 = cudaStreamQuery(S->stream);
    if (q0 != cudaSuccess && q0 != cudaErrorNotReady) return DS_ERR_CUDA;
    if (q0 == cudaSuccess && S->published == S->completed) {
        while (!S->pending.empty() && S->tickets.find(S->pending.front()) == S->tickets.end()) S->pending.pop_front();
        if (!S->pending.empty()) S->adapt_launch = adaptive_request(S->tickets.find(S->pending.front())->second.opt);
    }
    while (!S->pending.empty()) {
        auto it = S->tickets.find(S->pending.front());
        if (it == S->tickets.end()) {
            S->pending.pop_front();
            continue;
        }
        if (adaptive_request(it->second.opt) && !S->adapt_launch) break;
        if (!server_publish(S, it->first, it->second, it->second.y.data())) break;
        S->pending.pop_front();
    }
    // a kernel that went idle exits; relaunch it while published work is outstanding
    if (S->published > S->completed) {
        const cudaError_t q = cudaStreamQuery(S->stream);
        if (q == cudaSuccess) return server_launch(S);
        if (q != cudaErrorNotReady) return DS_ERR_CUDA;
    }
    int err = 0;
    cudaMemcpy(&err, S->derr, sizeof(int), cudaMemcpyDeviceToHost);
    return err ? DS_ERR_TIMEOUT : DS_OK;
}

}  // namespace ds

extern "C" {

ds_status ds_server_destroy(ds_server* S)
{
    if (!S) return DS_OK;
    if (S->ctx) cudaSetDevice(S->ctx->device);
    if (S->ctl_h) {
        reinterpret_cast<volatile int*>(S->ctl_h)[1] = 1;  // stop
        std::atomic_thread_fence(std::memory_order_seq_cst);
    }
    if (S->stream) {
        cudaStreamSynchronize(S->stream);
        cudaStreamDestroy(S->stream);
    }
    if (S->pool) cudaFree(S->pool);
    if (S->dctl) cudaFree(S->dctl);
    if (S->ring_h) cudaFreeHost(S->ring_h);
    if (S->lam_h) cudaFreeHost(S->lam_h);
    if (S->y_h) cudaFreeHost(S->y_h);
    if (S->x_h) cudaFreeHost(S->x_h);
    if (S->res_h) cudaFreeHost(S->res_h);
    if (S->done_h) cudaFreeHost(S->done_h);
    if (S->ctl_h) cudaFreeHost(S->ctl_h);
    delete S;
    return DS_OK;
}

ds_status ds_server_create(ds_ctx* ctx, size_t hbm_budget_bytes, int64_t max_N, int64_t max_K, int team_size,
                           ds_server** out)
{
    if (!ctx || !out || max_N < 1 || max_K < 1 || hbm_budget_bytes < (1u << 20) || team_size < 0 ||
        team_size > std::min(ctx->num_sms, ds::kMaxG))
        return DS_ERR_INVALID;
    *out = nullptr;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return DS_ERR_CUDA;
    ds_server* S = new (std::nothrow) ds_server();
    if (!S) return DS_ERR_OOM;
    S->ctx = ctx;
    S->team_size = team_size ? team_size : 4;
    S->n_teams = std::max(1, ctx->num_sms / S->team_size);
    S->ring = std::max(16, 4 * S->n_teams);
    S->max_N = max_N;
    S->max_K = max_K;
    S->budget = hbm_budget_bytes;
    auto fail = [&](ds_status st) {
        ds_server_destroy(S);
        return st;
    };
    // the largest request must fit the pool at least once
    ds::DictDesc dmax;
    std::memset(&dmax, 0, sizeof(dmax));
    dmax.dtype = DS_FP32;
    dmax.N = (int)max_N;
    dmax.K = (int)max_K;
    dmax.ld = (int)max_N;
    dmax.nG = (int)max_K;
    dmax.max_gsize = ds::kMaxGroup;
    dmax.is_group = 1;
    ds::Geometry gmax;
    if (ds::geometry<float>(dmax, S->team_size, ctx->smem_optin, &gmax) != DS_OK) return fail(DS_ERR_UNSUPPORTED);
    S->smem = (int)gmax.smem;
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(DS_ERR_CUDA);
    if (cudaMalloc(&S->pool, hbm_budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        S->pool = nullptr;
        return fail(DS_ERR_OOM);
    }
    S->alloc.init(hbm_budget_bytes);
    const unsigned fl = cudaHostAllocMapped;
    if (cudaHostAlloc((void**)&S->ring_h, sizeof(ds::ServerJob<float>) * S->ring, fl) != cudaSuccess ||
        cudaHostAlloc((void**)&S->lam_h, sizeof(double) * S->ring, fl) != cudaSuccess ||
        cudaHostAlloc((void**)&S->y_h, sizeof(float) * max_N * S->ring, fl) != cudaSuccess ||
        cudaHostAlloc((void**)&S->x_h, sizeof(float) * max_K * S->ring, fl) != cudaSuccess ||
        cudaHostAlloc((void**)&S->res_h, sizeof(ds::DevResult) * S->ring, fl) != cudaSuccess ||
        cudaHostAlloc((void**)&S->done_h, sizeof(int) * S->ring, fl) != cudaSuccess ||
        cudaHostAlloc((void**)&S->ctl_h, sizeof(int) * 2, fl) != cudaSuccess)
        return fail(DS_ERR_OOM);
    std::memset(S->done_h, 0, sizeof(int) * S->ring);
    std::memset(S->ctl_h, 0, sizeof(int) * 2);
    if (cudaHostGetDevicePointer((void**)&S->ring_d, S->ring_h, 0) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&S->lam_d, S->lam_h, 0) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&S->y_d, S->y_h, 0) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&S->x_d, S->x_h, 0) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&S->res_d, S->res_h, 0) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&S->done_d, S->done_h, 0) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&S->ctl_d, S->ctl_h, 0) != cudaSuccess)
        return fail(DS_ERR_CUDA);
    // device control: barriers + team_job (reset per launch), queue head + error (persistent), FISTA table
    S->bars_bytes = ds::align_up(sizeof(ds::GridBarrier) * S->n_teams + sizeof(int) * (S->n_teams + 2), 256);
    ds_status st = ds::ctx_fista_table(ctx, 1 << 16);
    if (st != DS_OK) return fail(st);
    S->fista_n = ctx->fista_n;
    S->dctl_bytes = S->bars_bytes + 256 + ds::align_up(sizeof(double) * 2 * S->fista_n, 256);
    if (cudaMalloc(&S->dctl, S->dctl_bytes) != cudaSuccess) return fail(DS_ERR_OOM);
    if (cudaMemset(S->dctl, 0, S->dctl_bytes) != cudaSuccess) return fail(DS_ERR_CUDA);
    char* c = reinterpret_cast<char*>(S->dctl);
    int* next_job = reinterpret_cast<int*>(c + S->bars_bytes);
    S->derr = next_job + 1;
    S->fista = reinterpret_cast<double*>(c + S->bars_bytes + 256);
    if (cudaMemcpy(S->fista, ctx->fista, sizeof(double) * 2 * S->fista_n, cudaMemcpyDeviceToDevice) != cudaSuccess)
        return fail(DS_ERR_CUDA);
    ds::TeamArgs<float>& A = S->args;
    std::memset(&A, 0, sizeof(A));
    A.n_jobs = S->ring;
    A.bars = reinterpret_cast<ds::GridBarrier*>(c);
    A.team_job = reinterpret_cast<int*>(c + sizeof(ds::GridBarrier) * S->n_teams);
    A.idle_teams = A.team_job + S->n_teams;
    A.exiting = A.idle_teams + 1;
    A.n_teams = S->n_teams;
    A.next_job = next_job;
    A.error = S->derr;
    A.team_size = S->team_size;
    A.server = 1;
    A.published = S->ctl_d;
    A.stop = S->ctl_d + 1;
    A.done = S->done_d;
    A.ring = S->ring_d;
    A.idle_polls = 20000;
    if (cudaFuncSetAttribute(ds::team_fn<float>(false), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(ctx->smem_optin - 40 * 1024)) != cudaSuccess ||
        cudaFuncSetAttribute(ds::team_fn<float>(true), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(ctx->smem_optin - 40 * 1024)) != cudaSuccess)
        return fail(DS_ERR_CUDA);
    S->slot_seq.assign(S->ring, -1);
    S->slot_ticket.assign(S->ring, 0);
    *out = S;
    return DS_OK;
}

ds_status ds_server_submit(ds_server* S, const ds_dict* dict, const void* y, double lambda, const ds_options* opt,
                           void* x_out, uint64_t* ticket)
{
    if (!S || !dict || !y || !opt || !x_out || !ticket || dict->ctx != S->ctx) return DS_ERR_INVALID;
    if (dict->dtype != DS_FP32) return DS_ERR_UNSUPPORTED;
    if (dict->N > S->max_N || dict->K > S->max_K) return DS_ERR_UNSUPPORTED;
    if (!(lambda > 0.0) || opt->max_iter < 1 || !(opt->tol_gap_rel >= 0.0) || opt->test < DS_TEST_NONE ||
        opt->test > DS_DGST3 || opt->alg < DS_ISTA || opt->alg > DS_TWIST || opt->L < 0.0)
        return DS_ERR_INVALID;
    if (dict->is_group && (opt->test == DS_SAFE || opt->test == DS_DST3 || opt->test == DS_DOME)) return DS_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (cudaSetDevice(S->ctx->device) != cudaSuccess) return DS_ERR_CUDA;
    const uint64_t tid = S->next_ticket++;
    ds_server::Ticket& t = S->tickets[tid];
    t.dict = dict;
    t.lambda = lambda;
    t.opt = *opt;
    t.x_out = x_out;
    t.t_submit = ds::now_ms();
    bool done = false;
    if (S->pending.empty()) done = ds::server_publish(S, tid, t, reinterpret_cast<const float*>(y));
    if (!done) {
        t.y.assign(reinterpret_cast<const float*>(y), reinterpret_cast<const float*>(y) + dict->N);
        S->pending.push_back(tid);
    }
    *ticket = tid;
    return ds::server_pump(S);
}

ds_status ds_server_poll(ds_server* S, uint64_t ticket, ds_result* res)
{
    if (!S || !res) return DS_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (cudaSetDevice(S->ctx->device) != cudaSuccess) return DS_ERR_CUDA;
    ds_status st = ds::server_pump(S);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return DS_ERR_INVALID;
    if (it->second.state != 2) return st == DS_OK ? DS_PENDING : st;
    *res = it->second.res;
    S->tickets.erase(it);
    return DS_OK;
}

ds_status ds_server_stats(ds_server* S, int64_t* completed, int64_t* in_flight, int64_t* pending, int64_t* launches,
                          size_t* pool_in_use)
{
    if (!S) return DS_ERR_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (completed) *completed = S->completed;
    if (in_flight) *in_flight = S->published - S->completed;
    if (pending) *pending = (int64_t)S->pending.size();
    if (launches) *launches = S->launches;
    if (pool_in_use) *pool_in_use = S->in_use;
    return DS_OK;
}

}  // extern "C"
