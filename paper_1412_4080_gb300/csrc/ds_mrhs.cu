// ds_mrhs.cu -- right-hand sides that share a dictionary, solved together.
//
// A block of up to 64 Lasso problems on one FP32 dictionary (each with its own
// y and lambda) runs Algorithm 3 in lockstep on a team of CTAs.  What the
// problems share is the dominant cost: every iteration correlates the union of
// their active sets with all their dual points at once,
//
//     Z = D_A^T [theta_1 ... theta_R]       (A = union of the active sets),
//
// a dense contraction in which each dictionary entry loaded from HBM (or L2)
// is used R times from shared memory, instead of once per problem.  Everything
// that differs between the problems stays per problem: y, lambda, lambda_*,
// d_*, the screening radius (Lemmas 2-4, 8), the screened set (a 64-bit mask
// per atom), the iterates, the nonzero lists of the syntheses and the stopping
// rule.  A problem that meets its gap tolerance is written out and leaves the
// block; the contraction then runs over the remaining ones only.
//
// Per iteration, three team phases separated by the bounded barrier:
//   (A) compaction of the union list; syntheses theta_r = D u_r - y_r and
//       D x_r over each problem's nonzeros (compensated, row tiles of 64);
//   (B) gaps and stopping per problem; Z over tiles of 128 atoms x 64 problems
//       (register-tiled FP32 FMA on operands staged by cp.async, split over
//       rows when the list is short, the last CTA of a tile summing the row
//       splits in a fixed order), fused with the proximal step;
//   (C) per problem: dual scaling, radius, test; FISTA extrapolation; the next
//       nonzero lists (lanes run over problems, so per-problem arrays are
//       contiguous).
// Reductions run in a fixed order, so results do not depend on timing.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ds_solve_body.cuh"
#include "ds_tc.cuh"

#include <cuda_bf16.h>

namespace ds {

constexpr int kMR = kMrhsMaxR;     // problems per block
constexpr int kMTA = 128;          // atoms per correlation tile
constexpr int kMKC = 32;           // rows per staged chunk
constexpr int kMST = kMKC + 4;     // shared row stride (floats): conflict-free 16-byte reads
constexpr int kMSynRows = 128;     // rows per synthesis item (four per lane)
constexpr int kMW = kThreads / 32; // warps per CTA
constexpr int kMStages = 3;        // cp.async pipeline depth of the FP32 contraction
constexpr int kCB = 4;             // atoms per step of the screening pass (loads in flight)
// tensor-core contraction on the BF16 copy: stages of a 128 x 64 A tile (16 KB)
// and a B tile of up to 128 rows (theta hi | lo, 16 KB), 128-byte swizzled
constexpr int kTcRows = 64;        // rows (K) per stage
constexpr int kTcStages = 5;       // ring depth
constexpr int kTcAhead = 3;        // stages in flight ahead of the MMA
constexpr int kTcStageBytes = 32768;
constexpr int kTcCols = 128;       // tensor-memory columns (FP32 accumulators)
constexpr int kZst = kMR + 1;      // row stride of the transposed accumulator tile
// staging of the contractions, also the scratch of the block reductions
constexpr int kStage32Bytes = kMStages * (kMTA + kMR) * kMST * 4;
constexpr int kStageBytes = kTcStages * kTcStageBytes > kStage32Bytes ? kTcStages * kTcStageBytes : kStage32Bytes;
static_assert(kMTA * kZst * 4 <= kStageBytes, "accumulator tile exceeds the staging area");

struct MrhsWs {
    float* Yt;   // [kMR][npad] y, zero padded
    float* Th;   // [kMR][npad] theta
    float* Dst;  // [kMR][npad] d_* of each problem (precompute)
    uint16_t* Thi;  // [kMR][npad] BF16 theta, rounded to nearest
    uint16_t* Tlo;  // [kMR][npad] BF16 of theta - Thi
    double* Q0;  // [K][kMR] D^T y; then SAFE/DST3 thresholds, or (Dome) d_i^T y / ||d_i||
    double* Q1;  // [K][kMR] D^T d_*; then (Dome) t_i = d_i^T d_* / (||d_i|| ||d_*||)
    double* Q2;  // [K][kMR] (Dome) sqrt(1 - t_i^2)
    double* invn;  // [K] 1 / ||d_i||
    FF* xb[2];   // [K][kMR] iterates x (two generations)
    FF* u;       // [K][kMR] extrapolated points
    unsigned long long* amask;   // [K] problems for which atom i is still active
    unsigned long long* nzmask;  // [K] problems with an entry of atom i in the next synthesis
    unsigned long long* kzmask;  // [K] of those, entries of x_{t-1} of an atom screened at t
    int* act[3][2];  // lists (union, bulk group, FP32 group), two generations each
    int* keep;       // [K] per union-list position: bit 0 stays, bit 1 in the bulk list, bit 2 in the FP32 list
    int* nz_col;  // [kMR][K] nonzero lists, per CTA segment
    FF* nz_x;
    FF* wb[2];    // [kMR][npad] D x_t of the last two iterations (float-float)
    float* part;  // row-split partial tiles
    int* tilecnt; // per tile: row splits finished
    int* ctr;     // 3 work counters (dynamic claiming), used in turn
    // per-unit partials, [unit][kMR] (problem index contiguous)
    float* p_m;   // [G] max |z| per CTA
    FF* p_l1;     // [G]
    int* c_na;    // [G]
    int* c_nnzx;  // [G]
    int* c_nz;    // [G] nonzero-list lengths
    int* c_keep;  // [3][G] atoms kept per list (no problem index)
    int* s_alo;   // [G] start of each CTA's list segment (no problem index)
    double* p_v;  // [G] max |d_i^T y| per CTA
    int* p_i;     // [G] its lowest index
    FF* p_a;      // [ntile] theta^T y per row tile
    FF* p_b;      // [ntile] ||theta||^2
    FF* p_r;      // [ntile] ||D x - y||^2
};

struct MrhsP {
    const float* D;
    int N, K, ld, npad, ntile;
    const double* colnorm;
    double fmax, L, gamma, eps_test, tol;
    int alg, test, dynamic, max_iter, lambda_rel;
    const float* Y;          // problem r: y at Y + ridx[r] * N
    int R;                   // problems in the block (<= kMR)
    int ridx[kMR];           // the instance's right-hand side of each problem
    const double* lambdas;   // R entries (device)
    float* X;                // problem r: x at X + ridx[r] * K
    DevResult* res;          // R entries
    const double* fista;
    int fista_n;
    // bulk phase on the tensor cores (dictionaries with a BF16 copy), then FP32
    const uint16_t* Dlo;   // BF16 copy, column i at Dlo + i * ld_lo, zero rows N..ld_lo-1
    int ld_lo;
    int use_tc;
    double emax;           // max_i ||d_i - copy_i||
    double gamma_tc;       // accumulation bound of the tensor-core sums
    double lo_switch;      // relative nominal gap at which the block leaves the copy
    MrhsWs ws;
};

// Tensor-core state of a CTA (kernel lifetime): accumulator columns, the
// mbarriers of the ring, and the running stage counter.
struct TcState {
    uint32_t tmem;
    uint64_t* mbar;  // kTcStages
    unsigned q;      // stages consumed so far (selects slot and phase)
    unsigned issued; // stages whose MMAs were committed
};

struct MrhsStage32 {
    float Ds[kMStages][kMTA][kMST];
    float Ts[kMStages][kMR][kMST];
};

struct MrhsShared {
    alignas(1024) unsigned char stage[kStageBytes];  // MrhsStage32, or reduction scratch
    int cols[kMTA];
    int slot_r[kMR];       // live slot -> problem (-1 past the live ones)
    int dir[kMW][kMaxG + 1];
    int alo[kMaxG];
    int cnt[kMW][kMR];
    unsigned int zmax[kMR];
    double lam[kMR], yy[kMR], lstar[kMR], psi_d[kMR], coef[kMR], delta[kMR], nstar[kMR];
    double alpha[kMR], beta[kMR], s_unc[kMR], sqrt_beta[kMR], R2n[kMR], rad[kMR], Rs[kMR], rho[kMR];
    double gap[kMR], primal[kMR];
    FF thrX[kMR];
    int istar[kMR], iters[kMR], na[kMR], nnzx[kMR], stopnow[kMR];
    long long csyn[kMR];
    unsigned long long live;
    int n_slots, last, claim;
    int nA[3], kbase[3], ktot[3];  // lists: union, bulk group, FP32 group
    unsigned long long dm;
    // precision phase per problem: bulk on the BF16 copy (tensor cores), then FP32
    unsigned long long gprev, gcur, gnext;  // bulk group of iterations t-1, t, t+1
    int since[kMR], swnow[kMR], t0r[kMR];
    double best_gap[kMR], R2s[kMR], lfr[kMR], btr[kMR];
    long long ccr[kMR], clr[kMR];
    int ired1[kMW], ired2[kMW];
    int ired[kMW];
    int scan_tmp[32];
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 16-byte shared-memory load by shared address (the contraction runs out of
// line, where a generic pointer would not be known to point to shared memory).
__device__ __forceinline__ float4 lds128(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

// One compensated product-accumulation (TwoProduct by FMA, Knuth's TwoSum);
// the explicitly rounded operations keep the compiler from contracting them.
__device__ __forceinline__ void d2_add(float& s, float& c, float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float pe = fmaf(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pe));
}
__device__ __forceinline__ void d2_merge(float& s, float& c, float s2, float c2)
{
    const float t = __fadd_rn(s, s2);
    const float bb = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(s2, bb));
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, c2));
}

// Z tile = D[:, cols]^T Theta[:, slots] over row chunks [c_lo, c_hi) of 32 rows,
// staged through a kMStages-deep cp.async ring.  Thread (ta, tr) owns atoms
// ta + 32j (j < 4) and slots tr + 16q (q < JJ).  COMP: compensated sums (s in
// acc, error in cmp); otherwise cmp holds the chunk's partial sum, added to acc
// once per chunk (two-level summation keeps the rounding bound at 32 + chunks
// terms).
template <int JJ, bool COMP>
__device__ __noinline__ void mr_gemm(MrhsShared& S, const float* __restrict__ D, int ld,
                                        const float* __restrict__ Th, int ldt, int c_lo, int c_hi, float (&acc_out)[4][4],
                                        float (&cmp_out)[4][4])
{
    // accumulators in registers of this function; the caller's arrays are written once at the end
    float acc[4][4], cmp[4][4];
    MrhsStage32& St = *reinterpret_cast<MrhsStage32*>(S.stage);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ta = warp * 2 + (lane >> 4), tr = lane & 15;
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            acc[j][q] = 0.f;
            cmp[j][q] = 0.f;
        }
    auto store = [&]() {
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int q = 0; q < 4; q++) {
                acc_out[j][q] = acc[j][q];
                cmp_out[j][q] = cmp[j][q];
            }
    };
    if (c_lo >= c_hi) {
        store();
        return;
    }
    auto issue = [&](int c, int buf) {
        const int n0 = c * kMKC;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int qd = tid + h * kThreads;
            const int a = qd >> 3, v = qd & 7;
            const int col = S.cols[a];
            const int n = n0 + 4 * v;
            const bool ok = col >= 0 && n < ld;  // rows N..ld-1 of the owned copy are zero
            const float* src = ok ? D + (size_t)col * ld + n : D;
            cp_async16(&St.Ds[buf][a][4 * v], src, ok ? 16 : 0);
        }
        if (tid < JJ * 16 * 8) {
            const int sl = tid >> 3, v = tid & 7;
            const int r = S.slot_r[sl];
            const bool ok = r >= 0;
            const float* src = ok ? Th + (size_t)r * ldt + n0 + 4 * v : Th;
            cp_async16(&St.Ts[buf][sl][4 * v], src, ok ? 16 : 0);
        }
    };
    // prologue: kMStages - 1 chunks in flight (empty groups keep the counting uniform)
#pragma unroll
    for (int k = 0; k < kMStages - 1; k++) {
        if (c_lo + k < c_hi) issue(c_lo + k, k);
        cp_async_commit();
    }
    int buf = 0;
    for (int c = c_lo; c < c_hi; c++) {
        cp_async_wait<kMStages - 2>();
        __syncthreads();  // chunk c landed for every thread; chunk c-1's buffer is free
        {
            const int cn = c + kMStages - 1;
            if (cn < c_hi) issue(cn, (buf + kMStages - 1) % kMStages);
            cp_async_commit();
        }
        const uint32_t dsb = smem_u32(&St.Ds[buf][ta][0]), tsb = smem_u32(&St.Ts[buf][tr][0]);
#pragma unroll
        for (int k4 = 0; k4 < kMKC / 4; k4++) {
            float4 a4[4], t4[JJ];
#pragma unroll
            for (int j = 0; j < 4; j++) a4[j] = lds128(dsb + (32 * j * kMST + 4 * k4) * 4);
#pragma unroll
            for (int q = 0; q < JJ; q++) t4[q] = lds128(tsb + (16 * q * kMST + 4 * k4) * 4);
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int q = 0; q < JJ; q++) {
                    if (COMP) {
                        d2_add(acc[j][q], cmp[j][q], a4[j].x, t4[q].x);
                        d2_add(acc[j][q], cmp[j][q], a4[j].y, t4[q].y);
                        d2_add(acc[j][q], cmp[j][q], a4[j].z, t4[q].z);
                        d2_add(acc[j][q], cmp[j][q], a4[j].w, t4[q].w);
                    } else {
                        cmp[j][q] = fmaf(a4[j].x, t4[q].x, cmp[j][q]);
                        cmp[j][q] = fmaf(a4[j].y, t4[q].y, cmp[j][q]);
                        cmp[j][q] = fmaf(a4[j].z, t4[q].z, cmp[j][q]);
                        cmp[j][q] = fmaf(a4[j].w, t4[q].w, cmp[j][q]);
                    }
                }
        }
        if (!COMP) {
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int q = 0; q < JJ; q++) {
                    acc[j][q] += cmp[j][q];
                    cmp[j][q] = 0.f;
                }
        }
        buf = (buf + 1) % kMStages;
    }
    cp_async_wait<0>();
    __syncthreads();  // the staging is free for the caller
    store();
}

// Z tile on the tensor cores: the BF16 copy of the tile's atoms times theta
// split in BF16 (hi | lo), over row chunks [c_lo, c_hi) of 64 rows, through a
// kTcStages-deep ring of 128-byte-swizzled stages (cp.async into the swizzled
// positions, then one thread issues 4 MMAs of K = 16 per stage and commits them
// to the stage's mbarrier, which frees the stage for reuse).  The FP32
// accumulators (hi columns, then lo columns) go through a transposed shared
// tile so that acc[j][q] has the thread mapping of the FP32 path.
__device__ __noinline__ bool mr_gemm_tc(MrhsShared& S, const MrhsP& P, int c_lo, int c_hi, int JJ, TcState& tc,
                                           float (&acc)[4][4])
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ta = warp * 2 + (lane >> 4), tr = lane & 15;
    const MrhsWs& W = P.ws;
    const int nb = 16 * JJ;  // B rows per half
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[j][q] = 0.f;
    if (c_lo >= c_hi) return true;
    const int n = c_hi - c_lo;
    const unsigned q0 = tc.q;
    const uint32_t st0 = smem_u32(S.stage);
    auto issue = [&](int i) {
        const unsigned g = q0 + i;
        unsigned char* A = S.stage + (g % kTcStages) * kTcStageBytes;
        unsigned char* B = A + 16384;
        const int n0 = (c_lo + i) * kTcRows;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int qd = tid + h * kThreads;
            const int a = qd >> 3, cc = qd & 7;
            const int col = S.cols[a];
            const int nn = n0 + cc * 8;
            const bool ok = col >= 0 && nn < P.ld_lo;  // rows N..ld_lo-1 of the copy are zero
            const uint16_t* src = ok ? P.Dlo + (size_t)col * P.ld_lo + nn : P.Dlo;
            cp_async16(A + sw128_offset(a, cc), src, ok ? 16 : 0);
        }
        for (int qd = tid; qd < 2 * nb * 8; qd += kThreads) {
            const int row = qd >> 3, cc = qd & 7;
            const int r = S.slot_r[row < nb ? row : row - nb];
            const uint16_t* base = row < nb ? W.Thi : W.Tlo;
            const bool ok = r >= 0;
            const uint16_t* src = ok ? base + (size_t)r * P.npad + n0 + cc * 8 : base;
            cp_async16(B + sw128_offset(row, cc), src, ok ? 16 : 0);
        }
    };
    // a slot is rewritten only after the MMAs that read its previous stage completed
    auto slot_free = [&](int i) -> bool {
        const unsigned g = q0 + i;
        if (g < (unsigned)kTcStages) return true;
        const unsigned prev = g - kTcStages;
        return mbar_wait(tc.mbar + (prev % kTcStages), (prev / kTcStages) & 1u);
    };
    bool ok = true;
#pragma unroll
    for (int i = 0; i < kTcAhead; i++) {
        if (i < n && ok) {
            if (slot_free(i)) issue(i);
            else ok = false;
        }
        cp_async_commit();
    }
    const uint32_t idesc = idesc_bf16_f32(128, 2 * nb);
    for (int i = 0; i < n; i++) {
        const int ia = i + kTcAhead;
        if (ia < n && ok) {
            if (slot_free(ia)) issue(ia);
            else ok = false;
        }
        cp_async_commit();
        cp_async_wait<kTcAhead>();  // this thread's copies of stage i landed
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && ok) {
            tc_fence_after();
            const unsigned g = q0 + i;
            const uint32_t A = st0 + (g % kTcStages) * kTcStageBytes, B = A + 16384;
#pragma unroll
            for (int k = 0; k < kTcRows / 16; k++)
                mma_bf16(tc.tmem, sw128_desc(A + 32 * k), sw128_desc(B + 32 * k), idesc, (i > 0 || k > 0) ? 1u : 0u);
            mma_commit(tc.mbar + (g % kTcStages));
        }
    }
    cp_async_wait<0>();
    if (!__syncthreads_and(ok)) return false;
    tc.q = q0 + n;
    tc.issued = tc.q;
    {
        const unsigned g = q0 + n - 1;
        if (!__syncthreads_and(mbar_wait(tc.mbar + (g % kTcStages), (g / kTcStages) & 1u))) return false;
    }
    tc_fence_after();
    float* Zs = reinterpret_cast<float*>(S.stage);  // [kMTA][kZst]; every stage has been consumed
    {
        const int qw = warp & 3, pw = warp >> 2;
        const uint32_t lane_base = (uint32_t)(32 * qw) << 16;
        for (int cc = 0; cc < JJ; cc++) {
            const int c0 = pw * 4 * JJ + 4 * cc;
            float hi[4], lo[4];
            tmem_ld4(tc.tmem + lane_base + c0, hi);
            tmem_ld4(tc.tmem + lane_base + nb + c0, lo);
#pragma unroll
            for (int k = 0; k < 4; k++) Zs[(32 * qw + lane) * kZst + c0 + k] = hi[k] + lo[k];
        }
    }
    tc_fence_before();
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int q = 0; q < 4; q++)
            if (q < JJ) acc[j][q] = Zs[(ta + 32 * j) * kZst + tr + 16 * q];
    __syncthreads();  // the staging is free again
    return true;
}

template <bool COMP>
__device__ __forceinline__ void mr_gemm_any(int JJ, MrhsShared& S, const float* D, int ld, const float* Th, int ldt,
                                            int c_lo, int c_hi, float (&acc)[4][4], float (&cmp)[4][4])
{
    switch (JJ) {
        case 1: mr_gemm<1, COMP>(S, D, ld, Th, ldt, c_lo, c_hi, acc, cmp); break;
        case 2: mr_gemm<2, COMP>(S, D, ld, Th, ldt, c_lo, c_hi, acc, cmp); break;
        case 3: mr_gemm<3, COMP>(S, D, ld, Th, ldt, c_lo, c_hi, acc, cmp); break;
        default: mr_gemm<4, COMP>(S, D, ld, Th, ldt, c_lo, c_hi, acc, cmp); break;
    }
}


// Work counter of the team's next claim loop: the loops take the three
// counters in turn, and each resets the one the next loop will use (its last
// use was two grid phases earlier).
__device__ __forceinline__ int* mr_counter(const MrhsWs& W, int& cu, int b)
{
    int* c = W.ctr + (cu % 3);
    if (b == 0 && threadIdx.x == 0) W.ctr[(cu + 1) % 3] = 0;
    cu++;
    return c;
}

// Z = D_A^T Theta over the tiles of `nA` list atoms (ids from `list`, or the
// identity when null), stream-K: the (tile, row chunk) units are cut into G
// equal contiguous runs, one per CTA, so a CTA streams about U/G chunks with
// at most one partial tile at each end.  A partial tile is parked in the CTA's
// slot (2b: first tile of its run, 2b + 1: last); the CTA that completes the
// tile's chunk count adds the parked partials in CTA order (a fixed order) and
// calls epi(acc, cmp) with S.cols holding the tile's atoms.
template <int KIND, typename Epi>
__device__ __forceinline__ bool mr_tiles(MrhsShared& S, const MrhsP& P, const int* list, int nA, const float* Th,
                                         int JJ, int b, int G, TcState& tc, int grp, Epi epi)
{
    constexpr bool COMP = KIND == 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ta = warp * 2 + (lane >> 4), tr = lane & 15;
    const MrhsWs& W = P.ws;
    const int TA = (nA + kMTA - 1) / kMTA;
    const int nc = P.npad / (KIND == 2 ? kTcRows : kMKC);
    const long long U = (long long)TA * nc;
    constexpr int TS = kMTA * kMR * (COMP ? 2 : 1);
    auto ulo = [&](int bb) -> long long { return (long long)bb * U / G; };
    const long long u0 = ulo(b), u1 = ulo(b + 1);
    const int first_tile = (int)(u0 / nc);
    // each contraction of a phase has its own parked tiles and counters: a CTA may start the
    // next one while others still add up this one's partial tiles
    float* part = W.part + (size_t)grp * 2 * G * kMTA * kMR * 2;
    int* tilecnt = W.tilecnt + (size_t)grp * ((P.K + kMTA - 1) / kMTA);
    long long u = u0;
    while (u < u1) {
        const int ti = (int)(u / nc);
        const int c_a = (int)(u - (long long)ti * nc);
        const int c_b = (int)min((long long)nc, u1 - (long long)ti * nc);
        u = (long long)ti * nc + c_b;
        if (tid < kMTA) {
            const int p = ti * kMTA + tid;
            S.cols[tid] = p < nA ? (list ? __ldcg(list + p) : p) : -1;
        }
        __syncthreads();
        float acc[4][4], cmp[4][4];
        if (KIND == 2) {
            if (!mr_gemm_tc(S, P, c_a, c_b, JJ, tc, acc)) return false;
        } else {
            mr_gemm_any<COMP>(JJ, S, P.D, P.ld, Th, P.npad, c_a, c_b, acc, cmp);
        }
        bool fin = true;
        if (c_b - c_a < nc) {
            float* pt = part + (size_t)(2 * b + (ti == first_tile ? 0 : 1)) * TS;
#pragma unroll
            for (int j = 0; j < 4; j++)
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (q < JJ) {
                        const int o = (ta + 32 * j) * kMR + tr + 16 * q;
                        pt[o] = acc[j][q];
                        if (COMP) pt[kMTA * kMR + o] = cmp[j][q];
                    }
            __threadfence();
            __syncthreads();
            if (tid == 0) S.last = (atomicAdd(tilecnt + ti, c_b - c_a) + (c_b - c_a) == nc);
            __syncthreads();
            fin = S.last != 0;
            if (fin) {
                __threadfence();
                const long long t_lo = (long long)ti * nc, t_hi = t_lo + nc;
                int b0 = (int)((t_lo * G) / U);  // the CTA whose run contains unit t_lo
                while (b0 > 0 && ulo(b0) > t_lo) b0--;
                while (b0 + 1 < G && ulo(b0 + 1) <= t_lo) b0++;
#pragma unroll
                for (int j = 0; j < 4; j++)
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        if (q < JJ) {
                            const int o = (ta + 32 * j) * kMR + tr + 16 * q;
                            float s = 0.f, c = 0.f;
                            for (int bb = b0; bb < G && ulo(bb) < t_hi; bb++) {
                                if (ulo(bb + 1) <= max(ulo(bb), t_lo)) continue;  // no units of this tile
                                const int sl = 2 * bb + (ti == (int)(ulo(bb) / nc) ? 0 : 1);
                                const float* ps = part + (size_t)sl * TS;
                                if (COMP) d2_merge(s, c, __ldcg(ps + o), __ldcg(ps + kMTA * kMR + o));
                                else s += __ldcg(ps + o);
                            }
                            acc[j][q] = s;
                            cmp[j][q] = c;
                        }
                if (tid == 0) tilecnt[ti] = 0;
            }
        }
        if (fin) epi(acc, cmp);
        __syncthreads();
    }
    return true;
}

// ----------------------------------------------------- block-wide reductions
//
// Per-problem partials are laid out [unit][kMR].  Warp w adds units w, w+16,
// ... for problems lane and lane + 32 (fixed order); thread r < kMR then adds
// the 16 warp results in warp order.  Every CTA that reduces the same
// partials gets the same bits.

struct RedScratch {
    float s[8][kMW][kMR];  // up to four float-float sums
    int n[3][kMW][kMR];    // up to three integer sums
};
static_assert(sizeof(RedScratch) <= kStageBytes, "reduction scratch exceeds the staging area");

// ------------------------------------------------------------ synthesis item
//
// Rows [128 rb, 128 rb + 128) of problem r: w_t = D x_t over its nonzero list
// (compensated), then theta_t = (1 + beta) w_t - beta (w_{t-1} - corrections) - y
// (FISTA, Table 1) and the row block's partials of theta^T y, ||theta||^2 and
// ||D x_t - y||^2.  The 16 warps split the list (8 entries in flight per warp,
// 4 rows per lane); their partial sums merge in warp order in shared memory.
__device__ __noinline__ void mr_synth_item(MrhsShared& S, const MrhsP& P, int r, int rb, int G, int t)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const MrhsWs& W = P.ws;
    const int N = P.N, K = P.K, ld = P.ld, npad = P.npad;
    int* dir = S.dir[0];
    if (warp == 0) {
        // where each CTA's segment of the list starts (exclusive prefix of the segment lengths);
        // the segment lengths are loaded together first so their L2 round trips overlap
        int cv[kMaxG / 32];
#pragma unroll
        for (int q = 0; q < kMaxG / 32; q++) {
            const int bb = 32 * q + lane;
            cv[q] = bb < G ? __ldcg(W.c_nz + bb * kMR + r) : 0;
        }
        int run = 0;
#pragma unroll
        for (int q = 0; q < kMaxG / 32; q++) {
            const int b0 = 32 * q;
            if (b0 >= G) break;
            const int bb = b0 + lane;
            const int c = cv[q];
            int x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (bb < G) dir[bb] = run + x - c;
            run += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) dir[G] = run;
    }
    __syncthreads();
    const int E = dir[G];
    const int e_lo = (int)((long long)warp * E / kMW), e_hi = (int)((long long)(warp + 1) * E / kMW);
    const int nb = rb * kMSynRows + lane;
    Dot2f ax[4], ac[4];
    const size_t rk = (size_t)r * K;
    for (int e0 = e_lo; e0 < e_hi; e0 += 32) {
        const int e = e0 + lane;
        int col = 0;
        FF xx{0.f, 0.f};
        if (e < e_hi) {
            int lo = 0, hi = G;  // largest segment start <= e
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (dir[mid] <= e) lo = mid;
                else hi = mid;
            }
            const size_t idx = rk + S.alo[lo] + (e - dir[lo]);
            col = __ldcg(W.nz_col + idx);
            xx = ldcg_x(W.nz_x + idx);
        }
        const int ne = min(32, e_hi - e0);
        for (int k0 = 0; k0 < ne; k0 += 8) {
            float d[8][4];
            FF xk[8];
            int ck[8];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const int k = min(k0 + q, 31);
                const bool in = k0 + q < ne;
                ck[q] = __shfl_sync(0xffffffffu, col, k);
                xk[q].h = __shfl_sync(0xffffffffu, xx.h, k);
                xk[q].l = __shfl_sync(0xffffffffu, xx.l, k);
                const int ci = ck[q] >= 0 ? ck[q] : -ck[q] - 1;
                const float* dc = P.D + (size_t)ci * ld;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int n = nb + 32 * j;
                    d[q][j] = (in && n < N) ? __ldg(dc + n) : 0.f;
                }
            }
#pragma unroll
            for (int q = 0; q < 8; q++) {
                if (ck[q] >= 0) {
#pragma unroll
                    for (int j = 0; j < 4; j++) syn_add(ax[j], d[q][j], xk[q]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; j++) syn_add(ac[j], d[q][j], xk[q]);
                }
            }
        }
    }
    float* red = reinterpret_cast<float*>(S.stage);  // [kMW][4][kMSynRows]
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int nl = lane + 32 * j;
        red[(warp * 4 + 0) * kMSynRows + nl] = ax[j].s;
        red[(warp * 4 + 1) * kMSynRows + nl] = ax[j].c;
        red[(warp * 4 + 2) * kMSynRows + nl] = ac[j].s;
        red[(warp * 4 + 3) * kMSynRows + nl] = ac[j].c;
    }
    __syncthreads();
    float* red2 = red + kMW * 4 * kMSynRows;  // [4 warps][6]
    if (tid < kMSynRows) {
        const int n = rb * kMSynRows + tid;
        Dot2f axm, acm;
        for (int w = 0; w < kMW; w++) {
            dot2_merge(axm, red[(w * 4 + 0) * kMSynRows + tid], red[(w * 4 + 1) * kMSynRows + tid]);
            dot2_merge(acm, red[(w * 4 + 2) * kMSynRows + tid], red[(w * 4 + 3) * kMSynRows + tid]);
        }
        Dot2f pa, pb, pr;
        if (n < N) {
            // FISTA (Table 1): D u_t = (1 + beta) D x_t - beta D x'_{t-1}, x'_{t-1} = x_{t-1} without the
            // atoms screened at t; theta = D u_t - y carried in float-float
            const double bt = S.btr[r];
            const FF w = ff_fast_two_sum(axm.s, axm.c);
            W.wb[t & 1][(size_t)r * npad + n] = w;
            const float yv = __ldcg(W.Yt + (size_t)r * npad + n);
            FF u = w;
            if (bt != 0.0) {
                const FF wp = ff_sub(ldcg_x(W.wb[(t - 1) & 1] + (size_t)r * npad + n), ff_fast_two_sum(acm.s, acm.c));
                u = ff_sub(ff_mul(w, ff_from_double(1.0 + bt)), ff_mul(wp, ff_from_double(bt)));
            }
            const FF tf = ff_sub(u, FF{yv, 0.f});
            const float th = tf.h + tf.l;
            W.Th[(size_t)r * npad + n] = th;
            if (P.use_tc) {
                // theta = hi + lo + O(2^-18 |theta|) in BF16, for the tensor cores
                const __nv_bfloat16 hb = __float2bfloat16_rn(th);
                const __nv_bfloat16 lb = __float2bfloat16_rn(th - __bfloat162float(hb));
                W.Thi[(size_t)r * npad + n] = __bfloat16_as_ushort(hb);
                W.Tlo[(size_t)r * npad + n] = __bfloat16_as_ushort(lb);
            }
            pa.add(th, yv);
            pb.add(th, th);
            acc_resid_sq(pr, axm, yv);
        }
        pa = dot2_warp_reduce(pa);
        pb = dot2_warp_reduce(pb);
        pr = dot2_warp_reduce(pr);
        if (lane == 0) {
            red2[warp * 6 + 0] = pa.s; red2[warp * 6 + 1] = pa.c;
            red2[warp * 6 + 2] = pb.s; red2[warp * 6 + 3] = pb.c;
            red2[warp * 6 + 4] = pr.s; red2[warp * 6 + 5] = pr.c;
        }
    }
    __syncthreads();
    if (tid == 0) {
        Dot2f pa, pb, pr;
        for (int w = 0; w < kMSynRows / 32; w++) {
            dot2_merge(pa, red2[w * 6 + 0], red2[w * 6 + 1]);
            dot2_merge(pb, red2[w * 6 + 2], red2[w * 6 + 3]);
            dot2_merge(pr, red2[w * 6 + 4], red2[w * 6 + 5]);
        }
        W.p_a[rb * kMR + r] = FF{pa.s, pa.c};
        W.p_b[rb * kMR + r] = FF{pb.s, pb.c};
        W.p_r[rb * kMR + r] = FF{pr.s, pr.c};
    }
    __syncthreads();
}

// --------------------------------------------------------------- the body

// One block of problems by a team of G CTAs (rank b) on barrier `bar`.
__device__ __noinline__ bool mrhs_body(const MrhsP& P, const int b, const int G, GridBarrier* bar, unsigned int& gen,
                                       TcState& tc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // the staging area starts on a 1024-byte boundary (swizzled tensor-core tiles)
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem_raw);
    MrhsShared& S = *reinterpret_cast<MrhsShared*>(smem_raw + ((1024u - (sa & 1023u)) & 1023u));
    RedScratch& RS = *reinterpret_cast<RedScratch*>(S.stage);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ta = warp * 2 + (lane >> 4), tr = lane & 15;
    const MrhsWs& W = P.ws;
    const int N = P.N, K = P.K, ld = P.ld, npad = P.npad, ntile = P.ntile, R = P.R;
    const int gwarp = b * kMW + warp, twarps = G * kMW;
    const bool dome = P.test == 3;
    const bool need_n = P.test == 2 || P.test == 3;
    const bool ista = P.alg == 0;
    const float invL = (float)(1.0 / P.L);
    int cu = 0;  // claim loops so far (same in every CTA)

    // -------------------------------------------- (C0a) staging, ||y_r||^2
    if (tid < kMR) S.slot_r[tid] = tid < R ? tid : -1;
    if (tid == 0) S.n_slots = R;
    for (size_t k = (size_t)b * kThreads + tid; k < (size_t)kMR * npad; k += (size_t)G * kThreads) {
        const int r = (int)(k / npad), n = (int)(k - (size_t)r * npad);
        W.Yt[k] = (r < R && n < N) ? P.Y[(size_t)P.ridx[r] * N + n] : 0.f;
        W.Th[k] = 0.f;
        W.Dst[k] = 0.f;
        W.wb[0][k] = FF{0.f, 0.f};
        W.wb[1][k] = FF{0.f, 0.f};
        if (P.use_tc) {
            W.Thi[k] = 0;
            W.Tlo[k] = 0;
        }
    }
    for (size_t k = (size_t)b * kThreads + tid; k < (size_t)R * K; k += (size_t)G * kThreads) {
        const int r = (int)(k / K);
        P.X[(size_t)P.ridx[r] * K + (k - (size_t)r * K)] = 0.f;
    }
    for (int k = b * kThreads + tid; k < 2 * ((K + kMTA - 1) / kMTA); k += G * kThreads) W.tilecnt[k] = 0;
    if (b == 0 && tid < 3) W.ctr[tid] = 0;
    for (int it = gwarp; it < ntile * kMR; it += twarps) {
        const int rt = it / kMR, r = it - rt * kMR;
        Dot2f acc;
        if (r < R) {
            for (int k = 0; k < kMSynRows / 32; k++) {
                const int n = rt * kMSynRows + 32 * k + lane;
                if (n < N) {
                    const float v = P.Y[(size_t)P.ridx[r] * N + n];
                    acc.add(v, v);
                }
            }
        }
        acc = dot2_warp_reduce(acc);
        if (lane == 0) W.p_a[rt * kMR + r] = FF{acc.s, acc.c};
    }
    if (!grid_sync(bar, G, gen)) return false;

    // -------------------------------------------- (C0b) B = D^T Y (compensated), lambda_*
    {
        // ||y_r||^2
        for (int h = 0; h < 2; h++) {
            const int r = lane + 32 * h;
            Dot2f a;
            for (int u = warp; u < ntile; u += kMW) {
                const FF v = ldcg_x(W.p_a + u * kMR + r);
                dot2_merge(a, v.h, v.l);
            }
            RS.s[0][warp][r] = a.s;
            RS.s[1][warp][r] = a.c;
        }
        __syncthreads();
        if (tid < kMR) {
            Dot2f a;
            for (int w = 0; w < kMW; w++) dot2_merge(a, RS.s[0][w][tid], RS.s[1][w][tid]);
            S.yy[tid] = a.value();
        }
        __syncthreads();
        const int JJ = (R + 15) / 16;
        double best[4];
        int arg[4];
#pragma unroll
        for (int q = 0; q < 4; q++) { best[q] = -1.0; arg[q] = 0x7fffffff; }
        if (!mr_tiles<1>(S, P, nullptr, K, W.Yt, JJ, b, G, tc, 0, [&](float (&acc)[4][4], float (&cmp)[4][4]) {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int i = S.cols[ta + 32 * j];
                if (i < 0) continue;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if (q >= JJ) continue;
                    const int r = S.slot_r[tr + 16 * q];
                    if (r < 0) continue;
                    const double v = (double)acc[j][q] + (double)cmp[j][q];
                    W.Q0[(size_t)i * kMR + r] = v;
                    const double a = fabs(v);
                    if (a > best[q] || (a == best[q] && i < arg[q])) { best[q] = a; arg[q] = i; }
                }
            }
        })) return false;
        // per-CTA argmax: the two halves of each warp, then the warps in order
        double* bv = reinterpret_cast<double*>(S.stage);        // [kMW][kMR]
        int* bi = reinterpret_cast<int*>(bv + kMW * kMR);        // [kMW][kMR]
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const double ob = __shfl_xor_sync(0xffffffffu, best[q], 16);
            const int oa = __shfl_xor_sync(0xffffffffu, arg[q], 16);
            if (ob > best[q] || (ob == best[q] && oa < arg[q])) { best[q] = ob; arg[q] = oa; }
            if (lane < 16 && q < JJ) { bv[warp * kMR + tr + 16 * q] = best[q]; bi[warp * kMR + tr + 16 * q] = arg[q]; }
        }
        __syncthreads();
        if (tid < R) {
            double bb = -1.0;
            int ba = 0x7fffffff;
            for (int w = 0; w < kMW; w++) {
                const double v = bv[w * kMR + tid];
                const int a = bi[w * kMR + tid];
                if (v > bb || (v == bb && a < ba)) { bb = v; ba = a; }
            }
            W.p_v[b * kMR + tid] = bb;
            W.p_i[b * kMR + tid] = ba;
        }
        __syncthreads();
    }
    if (!grid_sync(bar, G, gen)) return false;

    // -------------------------------------------- (C0c) per problem: lambda, the test centres
    {
        double* bv = reinterpret_cast<double*>(S.stage);
        int* bi = reinterpret_cast<int*>(bv + kMW * kMR);
        for (int h = 0; h < 2; h++) {
            const int r = lane + 32 * h;
            double bb = -1.0;
            int ba = 0x7fffffff;
            if (r < R)
                for (int u = warp; u < G; u += kMW) {
                    const double v = __ldcg(W.p_v + u * kMR + r);
                    const int a = __ldcg(W.p_i + u * kMR + r);
                    if (v > bb || (v == bb && a < ba)) { bb = v; ba = a; }
                }
            bv[warp * kMR + r] = bb;
            bi[warp * kMR + r] = ba;
        }
        __syncthreads();
        if (tid < R) {
            const int r = tid;
            double bb = -1.0;
            int ba = 0x7fffffff;
            for (int w = 0; w < kMW; w++) {
                const double v = bv[w * kMR + r];
                const int a = bi[w * kMR + r];
                if (v > bb || (v == bb && a < ba)) { bb = v; ba = a; }
            }
            const double lstar = bb;
            const double lam = P.lambda_rel ? P.lambdas[r] * lstar : P.lambdas[r];
            S.lstar[r] = lstar;
            S.istar[r] = ba;
            S.lam[r] = lam;
            S.thrX[r] = ff_from_double(lam / P.L);
            const double nstar = P.colnorm[ba];
            const double psi = lstar / lam - 1.0;
            // Lasso: n = d_* (Lemma 3), n^T y = lambda_*, ||n|| = ||d_*||
            const double nn = nstar * nstar;
            S.nstar[r] = nstar;
            S.psi_d[r] = psi / nstar;
            S.coef[r] = need_n ? psi / nn : 0.0;
            S.delta[r] = need_n ? fabs(psi) / nstar : 0.0;
            S.csyn[r] = 0;
            S.R2n[r] = 0.0;
            S.gap[r] = INFINITY;
            S.primal[r] = 0.0;
            S.iters[r] = 0;
        }
        __syncthreads();
    }
    if (tid == 0) {
        unsigned long long live = 0;
        for (int r = 0; r < R; r++)
            if (S.lam[r] < S.lstar[r]) live |= 1ull << r;
        S.live = live;
        S.gcur = S.gprev = S.gnext = P.use_tc ? live : 0ull;
        for (int r = 0; r < kMR; r++) {
            S.best_gap[r] = INFINITY;
            S.since[r] = 0;
            S.swnow[r] = 0;
            S.t0r[r] = 0;
            S.lfr[r] = 1.0;
            S.btr[r] = 0.0;
            S.R2s[r] = 0.0;
            S.ccr[r] = (long long)K * (need_n ? 2 : 1);  // the precompute passes
            S.clr[r] = 0;
        }
        int k = 0;
        for (int r = 0; r < kMR; r++)
            if ((live >> r) & 1) S.slot_r[k++] = r;
        S.n_slots = k;
        for (int q = k; q < kMR; q++) S.slot_r[q] = -1;
    }
    __syncthreads();
    // problems with lambda >= lambda_*: x = 0, y / lambda is dual optimal (Sec. 2.2.2)
    if (b == 0 && tid < R && !((S.live >> tid) & 1)) {
        DevResult& o = P.res[tid];
        o.iters = 0; o.status = kDevOk; o.n_active = 0; o.nnz = 0; o.gap = 0.0;
        o.primal = 0.5 * S.yy[tid]; o.dual = 0.5 * S.yy[tid]; o.lambda = S.lam[tid]; o.lambda_max = S.lstar[tid];
        o.cols_corr = S.ccr[tid]; o.cols_synth = 0; o.cols_lowp = 0;
    }
    if (need_n && S.live) {
        // d_* = sign(b_{i*}) d_{i*} of every problem (Lemma 3)
        for (size_t k = (size_t)b * kThreads + tid; k < (size_t)R * npad; k += (size_t)G * kThreads) {
            const int r = (int)(k / npad), n = (int)(k - (size_t)r * npad);
            float v = 0.f;
            if (((S.live >> r) & 1) && n < N) {
                const int is = S.istar[r];
                const float d = P.D[(size_t)is * ld + n];
                v = __ldcg(W.Q0 + (size_t)is * kMR + r) < 0.0 ? -d : d;
            }
            W.Dst[k] = v;
        }
        if (!grid_sync(bar, G, gen)) return false;
        const int JJ = (S.n_slots + 15) / 16;
        if (!mr_tiles<1>(S, P, nullptr, K, W.Dst, JJ, b, G, tc, 0, [&](float (&acc)[4][4], float (&cmp)[4][4]) {
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int i = S.cols[ta + 32 * j];
                if (i < 0) continue;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if (q >= JJ) continue;
                    const int r = S.slot_r[tr + 16 * q];
                    if (r < 0) continue;
                    W.Q1[(size_t)i * kMR + r] = (double)acc[j][q] + (double)cmp[j][q];
                }
            }
        })) return false;
        if (!grid_sync(bar, G, gen)) return false;
    }

    // -------------------------------------------- (C0d) thresholds, static test, initial state
    {
        const int p_lo = (int)((long long)b * K / G), p_hi = (int)((long long)(b + 1) * K / G);
        const int w_lo = p_lo + (int)((long long)warp * (p_hi - p_lo) / kMW);
        const int w_hi = p_lo + (int)((long long)(warp + 1) * (p_hi - p_lo) / kMW);
        const bool stat = !P.dynamic && P.test != 0;
        const unsigned long long live = S.live, gcur = S.gcur;
        double rad0[2] = {0.0, 0.0}, R0[2] = {0.0, 0.0};
        for (int h = 0; h < 2; h++) {
            const int r = lane + 32 * h;
            if (stat && ((live >> r) & 1)) {
                // Algorithm 1: the test at theta = -y, with m = lambda_*
                const double lam = S.lam[r], yy = S.yy[r];
                const double mu = dual_scale(-yy, yy, lam, S.lstar[r] * (1.0 + 1e-12));
                const double R2 = fmax(yy / (lam * lam) + 2.0 * mu * yy / lam + mu * mu * yy, 0.0);
                R0[h] = sqrt(R2);
                rad0[h] = P.test == 2 ? sqrt(fmax(R2 - S.delta[r] * S.delta[r], 0.0)) : R0[h];
            }
        }
        int kept0 = 0, kept1 = 0, kept2 = 0;
        for (int i = w_lo; i < w_hi; i++) {
            const double inv = 1.0 / P.colnorm[i];
            if (lane == 0) W.invn[i] = inv;
            bool on[2];
            for (int h = 0; h < 2; h++) {
                const int r = lane + 32 * h;
                const size_t idx = (size_t)i * kMR + r;
                on[h] = (live >> r) & 1;
                if (on[h] && P.test != 0) {
                    const double bi = __ldcg(W.Q0 + idx), lam = S.lam[r];
                    bool kill = false;
                    if (!dome) {
                        // sphere tests (Lemmas 2, 3): (1 - |d_i^T c|) / ||d_i||
                        const double dtc = bi / lam - (P.test == 2 ? S.coef[r] * __ldcg(W.Q1 + idx) : 0.0);
                        const double th = (1.0 - fabs(dtc)) * inv;
                        W.Q0[idx] = th;
                        kill = stat && th - rad0[h] > P.eps_test;
                    } else {
                        const double dc = bi * inv;
                        const double tt = __ldcg(W.Q1 + idx) * inv / S.nstar[r];
                        const double sq = sqrt(fmax(1.0 - tt * tt, 0.0));
                        W.Q0[idx] = dc;
                        W.Q1[idx] = tt;
                        W.Q2[idx] = sq;
                        if (stat) {
                            const double dc0 = dc / lam, psi = S.psi_d[r], Rr = R0[h];
                            const double rho = sqrt(fmax(Rr * Rr - psi * psi, 0.0));
                            const double up = (tt * Rr <= -psi) ? dc0 + Rr : dc0 - psi * tt + rho * sq;
                            const double dn = (-tt * Rr <= -psi) ? -dc0 + Rr : -dc0 + psi * tt + rho * sq;
                            kill = (inv - up > P.eps_test) && (inv - dn > P.eps_test);
                        }
                    }
                    if (kill) on[h] = false;
                }
                W.xb[0][idx] = FF{0.f, 0.f};
                W.xb[1][idx] = FF{0.f, 0.f};
                W.u[idx] = FF{0.f, 0.f};
            }
            const unsigned lo = __ballot_sync(0xffffffffu, on[0]), hi = __ballot_sync(0xffffffffu, on[1]);
            const unsigned long long m = ((unsigned long long)hi << 32) | lo;
            const int kf = (m != 0ull) | (((m & gcur) != 0ull) << 1) | (((m & ~gcur) != 0ull) << 2);
            if (lane == 0) {
                W.amask[i] = m;
                W.nzmask[i] = 0ull;
                W.kzmask[i] = 0ull;
                W.act[0][0][i] = i;
                W.keep[i] = kf;
            }
            kept0 += kf & 1;
            kept1 += (kf >> 1) & 1;
            kept2 += (kf >> 2) & 1;
        }
        if (lane == 0) {
            S.ired[warp] = kept0;
            S.ired1[warp] = kept1;
            S.ired2[warp] = kept2;
        }
        if (tid < kMR) {
            W.c_nz[b * kMR + tid] = 0;
            W.p_l1[b * kMR + tid] = FF{0.f, 0.f};
            W.c_na[b * kMR + tid] = 0;
            W.c_nnzx[b * kMR + tid] = 0;
        }
        __syncthreads();
        if (tid == 0) {
            int k0 = 0, k1 = 0, k2 = 0;
            for (int w = 0; w < kMW; w++) {
                k0 += S.ired[w];
                k1 += S.ired1[w];
                k2 += S.ired2[w];
            }
            W.c_keep[b] = k0;
            W.c_keep[G + b] = k1;
            W.c_keep[2 * G + b] = k2;
            W.s_alo[b] = p_lo;
            S.nA[0] = K;
            S.nA[1] = S.nA[2] = 0;
        }
    }
    if (!grid_sync(bar, G, gen)) return false;

    // ================================================================ iterations
    //
    // Lists (each compacted in order, double-buffered): 0 the union of the
    // active sets of the live problems, 1 of the problems in their bulk phase
    // (tensor cores on the BF16 copy), 2 of the problems in FP32.  A problem
    // leaves the bulk phase on its own, with a fresh FISTA sequence.
    int cur = 0;  // list generation
    int xi = 0;   // xb[xi] holds the current x
    for (int t = 1;; t++) {
        // ======================================== (A) compaction + syntheses
        {
            const int nA = S.nA[0];
            const int nxt = cur ^ 1;
            const int p_lo = (int)((long long)b * nA / G), p_hi = (int)((long long)(b + 1) * nA / G);
            if (warp < 3) {
                int base = 0, tot = 0;
                for (int k = lane; k < G; k += 32) {
                    const int c = __ldcg(W.c_keep + warp * G + k);
                    if (k < b) base += c;
                    tot += c;
                }
                base = warp_sum(base);
                tot = warp_sum(tot);
                if (lane == 0) { S.kbase[warp] = base; S.ktot[warp] = tot; }
            }
            for (int k = tid; k < G; k += kThreads) S.alo[k] = __ldcg(W.s_alo + k);
            __syncthreads();
            int gb0 = S.kbase[0], gb1 = S.kbase[1], gb2 = S.kbase[2];
            for (int base = p_lo; base < p_hi; base += kThreads) {
                const int p = base + tid;
                int a = 0, kf = 0;
                if (p < p_hi) {
                    a = __ldcg(W.act[0][cur] + p);
                    kf = __ldcg(W.keep + p);
                }
                // one packed scan of the three keep bits (at most 512 per field)
                const int v = (kf & 1) | (((kf >> 1) & 1) << 10) | (((kf >> 2) & 1) << 20);
                int tot;
                const int pre = block_exclusive_scan(v, S.scan_tmp, &tot);
                if (kf & 1) W.act[0][nxt][gb0 + (pre & 1023)] = a;
                if (kf & 2) W.act[1][nxt][gb1 + ((pre >> 10) & 1023)] = a;
                if (kf & 4) W.act[2][nxt][gb2 + ((pre >> 20) & 1023)] = a;
                gb0 += tot & 1023;
                gb1 += (tot >> 10) & 1023;
                gb2 += (tot >> 20) & 1023;
            }
            // syntheses: items (live problem, block of 128 rows), claimed by the team's CTAs
            const int ns = S.n_slots;
            int* ctr = mr_counter(W, cu, b);
            for (;;) {
                if (tid == 0) S.claim = atomicAdd(ctr, 1);
                __syncthreads();
                const int it = S.claim;
                if (it >= ntile * ns) break;
                const int s = it / ntile, rb = it - s * ntile;
                mr_synth_item(S, P, S.slot_r[s], rb, G, t);
            }
            __syncthreads();
            if (tid == 0) {
                S.nA[0] = S.ktot[0];
                S.nA[1] = S.ktot[1];
                S.nA[2] = S.ktot[2];
            }
            cur = nxt;
        }
        if (!grid_sync(bar, G, gen)) return false;

        // ======================================== (B) gaps, stop, correlation + prox
        {
            const int nA = S.nA[0];
            const int ns = S.n_slots;
            const unsigned long long live = S.live;
            // per-problem sums of the row-tile partials and of the CTA partials of (C)
            for (int h = 0; h < 2; h++) {
                const int r = lane + 32 * h;
                Dot2f a, bq, rq, l1;
                int na = 0, nx = 0, ne = 0;
                if ((live >> r) & 1) {
#pragma unroll 2
                    for (int u = warp; u < ntile; u += kMW) {
                        const FF va = ldcg_x(W.p_a + u * kMR + r), vb = ldcg_x(W.p_b + u * kMR + r);
                        const FF vr = ldcg_x(W.p_r + u * kMR + r);
                        dot2_merge(a, va.h, va.l);
                        dot2_merge(bq, vb.h, vb.l);
                        dot2_merge(rq, vr.h, vr.l);
                    }
#pragma unroll 4
                    for (int u = warp; u < G; u += kMW) {
                        const FF vl = ldcg_x(W.p_l1 + u * kMR + r);
                        const int c0 = __ldcg(W.c_na + u * kMR + r), c1 = __ldcg(W.c_nnzx + u * kMR + r);
                        const int c2 = __ldcg(W.c_nz + u * kMR + r);
                        dot2_merge(l1, vl.h, vl.l);
                        na += c0;
                        nx += c1;
                        ne += c2;
                    }
                }
                RS.s[0][warp][r] = a.s;  RS.s[1][warp][r] = a.c;
                RS.s[2][warp][r] = bq.s; RS.s[3][warp][r] = bq.c;
                RS.s[4][warp][r] = rq.s; RS.s[5][warp][r] = rq.c;
                RS.s[6][warp][r] = l1.s; RS.s[7][warp][r] = l1.c;
                RS.n[0][warp][r] = na;   RS.n[1][warp][r] = nx;   RS.n[2][warp][r] = ne;
            }
            __syncthreads();
            if (tid < kMR && ((live >> tid) & 1)) {
                const int r = tid;
                Dot2f a, bq, rq, l1;
                int na = 0, nx = 0, ne = 0;
                for (int w = 0; w < kMW; w++) {
                    dot2_merge(a, RS.s[0][w][r], RS.s[1][w][r]);
                    dot2_merge(bq, RS.s[2][w][r], RS.s[3][w][r]);
                    dot2_merge(rq, RS.s[4][w][r], RS.s[5][w][r]);
                    dot2_merge(l1, RS.s[6][w][r], RS.s[7][w][r]);
                    na += RS.n[0][w][r];
                    nx += RS.n[1][w][r];
                    ne += RS.n[2][w][r];
                }
                const double a_ = a.value(), b_ = bq.value(), r_ = rq.value(), l1_ = l1.value();
                const double lam = S.lam[r], yy = S.yy[r];
                const bool low_prev = (S.gprev >> r) & 1;  // the correlations of iteration t-1 came from the copy
                int stop = 0, sw = 0;
                if (t > 1) {
                    // P(xbar) - Dual(mu theta), Dual(v) = 1/2||y||^2 - lambda^2/2 ||v - y/lambda||^2
                    const double primal = 0.5 * r_ + lam * l1_;
                    double gap = primal - 0.5 * yy + 0.5 * lam * lam * S.R2n[r];
                    bool swok = false;
                    if (low_prev) {
                        // the nominal gap rests on the copy's correlations: stop only on the rigorous one
                        // (dual point scaled with the bounded max); leave the copy once the nominal gap
                        // reached the switch level or stopped improving
                        if (gap < 0.99 * S.best_gap[r]) {
                            S.best_gap[r] = gap;
                            S.since[r] = 0;
                        } else {
                            S.since[r]++;
                        }
                        swok = (gap <= P.lo_switch * 0.5 * yy) || S.since[r] >= 25;
                        gap = primal - 0.5 * yy + 0.5 * lam * lam * S.R2s[r];
                    }
                    S.primal[r] = primal;
                    S.gap[r] = gap;
                    S.iters[r] = t - 1;
                    S.na[r] = na;
                    S.nnzx[r] = nx;
                    stop = (P.tol > 0.0 && gap <= P.tol * 0.5 * yy) || (t - 1 >= P.max_iter);
                    sw = !stop && swok && ((S.gcur >> r) & 1);
                }
                if (sw) {
                    // FP32 polish: a fresh FISTA sequence from the bulk iterate
                    S.t0r[r] = t - 1;
                    S.lfr[r] = 1.0;
                }
                double bt = 0.0;
                if (!ista) {
                    // FISTA (Table 1): l_t = (1 + sqrt(1 + 4 l_{t-1}^2)) / 2, coefficient (l_{t-1} - 1) / l_t
                    const int tf = t - S.t0r[r];
                    if (tf <= P.fista_n) {
                        bt = P.fista[2 * (tf - 1)];
                        S.lfr[r] = P.fista[2 * (tf - 1) + 1];
                    } else {
                        const double lf = S.lfr[r];
                        const double ln = 0.5 * (1.0 + sqrt(1.0 + 4.0 * lf * lf));
                        bt = (lf - 1.0) / ln;
                        S.lfr[r] = ln;
                    }
                }
                S.btr[r] = bt;
                S.csyn[r] += ne;
                S.alpha[r] = a_;
                S.beta[r] = b_;
                S.s_unc[r] = b_ > 0.0 ? a_ / lam * fast_rcp(b_) : 0.0;
                S.sqrt_beta[r] = (double)sqrtf((float)b_) * (1.0 + 1e-6);
                S.stopnow[r] = stop;
                S.swnow[r] = sw;
            }
            __syncthreads();
            if (tid == 0) {
                unsigned long long dm = 0, sw = 0;
                for (int s = 0; s < ns; s++) {
                    const int r = S.slot_r[s];
                    if (S.stopnow[r]) dm |= 1ull << r;
                    if (S.swnow[r]) sw |= 1ull << r;
                }
                S.dm = dm;
                S.gnext = S.gcur & ~sw;
            }
            __syncthreads();
            const unsigned long long dm = S.dm;
            if (dm) {
                // problems that met their tolerance leave the block: x of iteration t-1 out
                const int p_lo = (int)((long long)b * nA / G), p_hi = (int)((long long)(b + 1) * nA / G);
                for (int p = p_lo + warp; p < p_hi; p += kMW) {
                    const int i = __ldcg(W.act[0][cur] + p);
                    const unsigned long long m = __ldcg(W.amask + i);
                    for (int h = 0; h < 2; h++) {
                        const int r = lane + 32 * h;
                        if ((dm >> r) & 1) {
                            const FF x = ((m >> r) & 1) ? ldcg_x(W.xb[xi] + (size_t)i * kMR + r) : FF{0.f, 0.f};
                            P.X[(size_t)P.ridx[r] * K + i] = it_round(x);
                        }
                    }
                }
                if (b == 0 && tid < kMR && ((dm >> tid) & 1)) {
                    const int r = tid;
                    DevResult& o = P.res[r];
                    o.iters = S.iters[r];
                    o.status = (P.tol > 0.0 && !(S.gap[r] <= P.tol * 0.5 * S.yy[r])) ? kDevNotConverged : kDevOk;
                    o.n_active = S.na[r];
                    o.nnz = S.nnzx[r];
                    o.gap = S.gap[r];
                    o.primal = S.primal[r];
                    o.dual = S.primal[r] - S.gap[r];
                    o.lambda = S.lam[r];
                    o.lambda_max = S.lstar[r];
                    o.cols_corr = S.ccr[r];
                    o.cols_synth = S.csyn[r];
                    o.cols_lowp = S.clr[r];
                }
                __syncthreads();
                if (tid == 0) S.live &= ~dm;
                __syncthreads();
            }
            if (S.live == 0ull) break;
            const unsigned long long live2 = S.live;
            if (tid < kMR && ((live2 >> tid) & 1)) {
                const bool lo = (S.gcur >> tid) & 1;
                S.ccr[tid] += lo ? S.nA[1] : S.nA[2];
                if (lo) S.clr[tid] += S.nA[1];
            }
            // the correlations of each group over its own list: bulk problems on the tensor cores
            // (BF16 copy), the others on the FP32 master
            for (int grp = 0; grp < 2; grp++) {
                const unsigned long long gm = grp == 0 ? (live2 & S.gcur) : (live2 & ~S.gcur);
                if (gm == 0ull) continue;
                if (tid == 0) {
                    int k = 0;
                    for (int r = 0; r < kMR; r++)
                        if ((gm >> r) & 1) S.slot_r[k++] = r;
                    S.n_slots = k;
                    for (int s = k; s < kMR; s++) S.slot_r[s] = -1;
                }
                if (tid < kMR) S.zmax[tid] = 0u;
                __syncthreads();
                const int JJ = (S.n_slots + 15) / 16;
                float zm[4] = {0.f, 0.f, 0.f, 0.f};
                FF* xo = W.xb[xi ^ 1];
                auto prox = [&](float (&acc)[4][4], float (&)[4][4]) {
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        const int i = S.cols[ta + 32 * j];
                        if (i < 0) continue;
                        const unsigned long long m = __ldcg(W.amask + i);
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            if (q >= JJ) continue;
                            const int r = S.slot_r[tr + 16 * q];
                            if (r < 0) continue;
                            const size_t idx = (size_t)i * kMR + r;
                            FF xn{0.f, 0.f};
                            if ((m >> r) & 1) {
                                // proximal step (Table 1): x = soft(u - z / L, lambda / L)
                                const float z = acc[j][q];
                                xn = it_soft(it_grad_step(ldcg_x(W.u + idx), z, invL), S.thrX[r]);
                                zm[q] = fmaxf(zm[q], fabsf(z));
                            }
                            xo[idx] = xn;
                        }
                    }
                };
                const bool okt = grp == 0 ? mr_tiles<2>(S, P, W.act[1][cur], S.nA[1], W.Th, JJ, b, G, tc, 0, prox)
                                          : mr_tiles<0>(S, P, W.act[2][cur], S.nA[2], W.Th, JJ, b, G, tc, 1, prox);
                if (!okt) return false;
#pragma unroll
                for (int q = 0; q < 4; q++)
                    if (q < JJ) atomicMax(&S.zmax[tr + 16 * q], __float_as_uint(zm[q]));
                __syncthreads();
                if (tid < S.n_slots) W.p_m[b * kMR + S.slot_r[tid]] = __uint_as_float(S.zmax[tid]);
                __syncthreads();
            }
            // the live list again (syntheses, stop tests)
            if (tid == 0) {
                int k = 0;
                for (int r = 0; r < kMR; r++)
                    if ((live2 >> r) & 1) S.slot_r[k++] = r;
                S.n_slots = k;
                for (int s = k; s < kMR; s++) S.slot_r[s] = -1;
            }
            __syncthreads();
        }
        if (!grid_sync(bar, G, gen)) return false;

        // ======================================== (C) screening + momentum
        {
            const int nA = S.nA[0];
            const unsigned long long live = S.live, gcur = S.gcur, gnext = S.gnext;
            {
                // m_r = max_i |z_i| over the CTA partials, then Lemma 8 and the radius per problem
                float* mx = reinterpret_cast<float*>(S.stage);  // [kMW][kMR]
                for (int h = 0; h < 2; h++) {
                    const int r = lane + 32 * h;
                    float m = 0.f;
                    if ((live >> r) & 1) {
#pragma unroll 4
                        for (int u = warp; u < G; u += kMW) m = fmaxf(m, __ldcg(W.p_m + u * kMR + r));
                    }
                    mx[warp * kMR + r] = m;
                }
                __syncthreads();
                if (tid < kMR && ((live >> tid) & 1)) {
                    const int r = tid;
                    float mf = 0.f;
                    for (int w = 0; w < kMW; w++) mf = fmaxf(mf, mx[w * kMR + r]);
                    // Lemma 8 with the nominal max |z| (gap) and a rigorous upper bound of it (radius)
                    // (copy: |z_i - zc_i| <= ||d_i - copy_i|| ||theta|| + ||copy_i|| (||theta - hi - lo|| +
                    // the accumulation bound of the tensor-core sums))
                    const double m_nom = (double)mf;
                    const bool lo = (gcur >> r) & 1;
                    const double m_up =
                        m_nom + (lo ? P.emax + (P.fmax + P.emax) * (0x1p-17 + P.gamma_tc) : P.gamma * P.fmax) *
                                    S.sqrt_beta[r];
                    const double su = S.s_unc[r];
                    const double mu_nom = (m_nom > 0.0 && fabs(su) * m_nom > 1.0) ? copysign(fast_rcp(m_nom), su) : su;
                    const double mu_s = (m_up > 0.0 && fabs(su) * m_up > 1.0) ? copysign(fast_rcp(m_up), su) : su;
                    const double il = 1.0 / S.lam[r];
                    const double yyl2 = S.yy[r] * il * il;
                    S.R2n[r] = fmax(fma(mu_nom, fma(mu_nom, S.beta[r], -2.0 * S.alpha[r] * il), yyl2), 0.0);
                    const double R2s = fmax(fma(mu_s, fma(mu_s, S.beta[r], -2.0 * S.alpha[r] * il), yyl2), 0.0);
                    S.R2s[r] = R2s;
                    const double Rs = fast_sqrt(R2s) * (1.0 + 1e-13);
                    S.Rs[r] = Rs;
                    S.rad[r] = P.test == 2 ? fast_sqrt(fmax(R2s - S.delta[r] * S.delta[r], 0.0)) * (1.0 + 1e-13) : Rs;
                    const double psi = S.psi_d[r];
                    S.rho[r] = fast_sqrt(fmax(Rs * Rs - psi * psi, 0.0)) * (1.0 + 1e-13);
                }
                __syncthreads();
            }
            const bool dyn = P.dynamic && P.test != 0;
            const int p_lo = (int)((long long)b * nA / G), p_hi = (int)((long long)(b + 1) * nA / G);
            const int w_lo = p_lo + (int)((long long)warp * (p_hi - p_lo) / kMW);
            const int w_hi = p_lo + (int)((long long)(warp + 1) * (p_hi - p_lo) / kMW);
            FF* xnew = W.xb[xi ^ 1];
            const FF* xold = W.xb[xi];
            int cnt[2] = {0, 0}, na[2] = {0, 0}, nx[2] = {0, 0}, kept0 = 0, kept1 = 0, kept2 = 0;
            Dot2f l1[2];
            double radh[2], Rsh[2], rhoh[2], psih[2], ilh[2];
            FF btXh[2];
            bool lv[2];
            for (int h = 0; h < 2; h++) {
                const int r = lane + 32 * h;
                lv[h] = (live >> r) & 1;
                radh[h] = lv[h] ? S.rad[r] : 0.0;
                Rsh[h] = lv[h] ? S.Rs[r] : 0.0;
                rhoh[h] = lv[h] ? S.rho[r] : 0.0;
                psih[h] = lv[h] ? S.psi_d[r] : 0.0;
                ilh[h] = lv[h] ? 1.0 / S.lam[r] : 0.0;
                btXh[h] = ff_from_double(lv[h] ? S.btr[r] : 0.0);
            }
            for (int p0 = w_lo; p0 < w_hi; p0 += kCB) {
                // kCB atoms per step, every load of the step issued before it is used
                int iv[kCB];
                unsigned long long mv[kCB];
#pragma unroll
                for (int q = 0; q < kCB; q++) iv[q] = p0 + q < w_hi ? __ldcg(W.act[0][cur] + p0 + q) : -1;
#pragma unroll
                for (int q = 0; q < kCB; q++) mv[q] = iv[q] >= 0 ? __ldcg(W.amask + iv[q]) : 0ull;
                bool on[kCB][2];
                double tq[kCB][2];
                FF xv[kCB][2], xw[kCB][2];
#pragma unroll
                for (int q = 0; q < kCB; q++)
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int r = lane + 32 * h;
                        on[q][h] = iv[q] >= 0 && lv[h] && ((mv[q] >> r) & 1);
                        tq[q][h] = 0.0;
                        xv[q][h] = FF{0.f, 0.f};
                        xw[q][h] = FF{0.f, 0.f};
                        if (on[q][h]) {
                            const size_t idx = (size_t)iv[q] * kMR + r;
                            if (dyn) tq[q][h] = __ldcg(W.Q0 + idx);
                            xv[q][h] = ldcg_x(xnew + idx);
                            if (!ista) xw[q][h] = ldcg_x(xold + idx);
                        }
                    }
#pragma unroll
                for (int q = 0; q < kCB; q++) {
                    bool nz[2], kz[2];
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        nz[h] = false;
                        kz[h] = false;
                        if (!on[q][h]) continue;
                        const int r = lane + 32 * h;
                        const size_t idx = (size_t)iv[q] * kMR + r;
                        bool kill = false;
                        if (dyn) {
                            if (!dome) {
                                kill = tq[q][h] - radh[h] > P.eps_test;
                            } else {
                                // Lemma 4 in its dynamic form: max over the dome of |d_i^T theta| < 1
                                const double dc0 = tq[q][h] * ilh[h];
                                const double tt = __ldcg(W.Q1 + idx), sq = __ldcg(W.Q2 + idx);
                                const double inv = __ldcg(W.invn + iv[q]);
                                const double Rr = Rsh[h], psi = psih[h], rho = rhoh[h];
                                const double up = (tt * Rr <= -psi) ? dc0 + Rr : dc0 - psi * tt + rho * sq;
                                const double dn = (-tt * Rr <= -psi) ? -dc0 + Rr : -dc0 + psi * tt + rho * sq;
                                kill = (inv - up > P.eps_test) && (inv - dn > P.eps_test);
                            }
                        }
                        if (kill) {
                            on[q][h] = false;
                            xnew[idx] = FF{0.f, 0.f};
                            W.u[idx] = FF{0.f, 0.f};
                            // the next synthesis removes d_i x_{t-1,i} from D x_{t-1} (FISTA)
                            kz[h] = !ista && it_nz(xw[q][h]);
                            nz[h] = kz[h];
                            cnt[h] += nz[h];
                            continue;
                        }
                        const FF x = xv[q][h];
                        const FF uu = ista ? x : it_momentum(x, xw[q][h], btXh[h]);
                        W.u[idx] = uu;
                        nz[h] = it_nz(x);
                        nx[h] += it_nz(x);
                        acc_abs(l1[h], x);
                        na[h] += 1;
                        cnt[h] += nz[h];
                    }
                    const unsigned lo = __ballot_sync(0xffffffffu, on[q][0]), hi = __ballot_sync(0xffffffffu, on[q][1]);
                    const unsigned zlo = __ballot_sync(0xffffffffu, nz[0]), zhi = __ballot_sync(0xffffffffu, nz[1]);
                    const unsigned klo = __ballot_sync(0xffffffffu, kz[0]), khi = __ballot_sync(0xffffffffu, kz[1]);
                    const unsigned long long onm = ((unsigned long long)hi << 32) | lo;
                    // the lists of the next iteration: union, bulk group, FP32 group
                    const int kf = (onm != 0ull) | (((onm & gnext) != 0ull) << 1) | (((onm & ~gnext) != 0ull) << 2);
                    if (lane == 0 && iv[q] >= 0) {
                        W.amask[iv[q]] = (mv[q] & ~live) | onm;
                        W.nzmask[iv[q]] = ((unsigned long long)zhi << 32) | zlo;
                        W.kzmask[iv[q]] = ((unsigned long long)khi << 32) | klo;
                        W.keep[p0 + q] = kf;
                    }
                    if (iv[q] >= 0) {
                        kept0 += kf & 1;
                        kept1 += (kf >> 1) & 1;
                        kept2 += (kf >> 2) & 1;
                    }
                }
            }
            for (int h = 0; h < 2; h++) {
                const int r = lane + 32 * h;
                S.cnt[warp][r] = cnt[h];
                RS.s[0][warp][r] = l1[h].s;
                RS.s[1][warp][r] = l1[h].c;
                RS.n[0][warp][r] = na[h];
                RS.n[1][warp][r] = nx[h];
            }
            if (lane == 0) {
                S.ired[warp] = kept0;
                S.ired1[warp] = kept1;
                S.ired2[warp] = kept2;
            }
            __syncthreads();
            if (tid < kMR) {
                const int r = tid;
                int run = 0, a = 0, x = 0;
                Dot2f l;
                for (int w = 0; w < kMW; w++) {
                    const int c = S.cnt[w][r];
                    S.cnt[w][r] = run;
                    run += c;
                    dot2_merge(l, RS.s[0][w][r], RS.s[1][w][r]);
                    a += RS.n[0][w][r];
                    x += RS.n[1][w][r];
                }
                W.c_nz[b * kMR + r] = run;
                W.p_l1[b * kMR + r] = FF{l.s, l.c};
                W.c_na[b * kMR + r] = a;
                W.c_nnzx[b * kMR + r] = x;
            }
            if (tid == 0) {
                int k0 = 0, k1 = 0, k2 = 0;
                for (int w = 0; w < kMW; w++) {
                    k0 += S.ired[w];
                    k1 += S.ired1[w];
                    k2 += S.ired2[w];
                }
                W.c_keep[b] = k0;
                W.c_keep[G + b] = k1;
                W.c_keep[2 * G + b] = k2;
                W.s_alo[b] = p_lo;
            }
            __syncthreads();
            // the nonzero lists of the next syntheses, per problem, in list order
            int e[2] = {S.cnt[warp][lane], S.cnt[warp][lane + 32]};
            for (int p0 = w_lo; p0 < w_hi; p0 += kCB) {
                int iv[kCB];
                unsigned long long zv[kCB], kv[kCB];
#pragma unroll
                for (int q = 0; q < kCB; q++) iv[q] = p0 + q < w_hi ? __ldcg(W.act[0][cur] + p0 + q) : -1;
#pragma unroll
                for (int q = 0; q < kCB; q++) {
                    zv[q] = iv[q] >= 0 ? __ldcg(W.nzmask + iv[q]) : 0ull;
                    kv[q] = iv[q] >= 0 ? __ldcg(W.kzmask + iv[q]) : 0ull;
                }
#pragma unroll
                for (int q = 0; q < kCB; q++)
#pragma unroll
                    for (int h = 0; h < 2; h++) {
                        const int r = lane + 32 * h;
                        if ((zv[q] >> r) & 1) {
                            const size_t idx = (size_t)iv[q] * kMR + r;
                            const size_t o = (size_t)r * K + p_lo + e[h]++;
                            const bool k = (kv[q] >> r) & 1;
                            W.nz_col[o] = k ? -iv[q] - 1 : iv[q];
                            W.nz_x[o] = k ? ldcg_x(xold + idx) : ldcg_x(xnew + idx);
                        }
                    }
            }
            xi ^= 1;
            __syncthreads();
            if (tid == 0) {
                S.gprev = gcur;
                S.gcur = gnext;
            }
        }
        if (!grid_sync(bar, G, gen)) return false;
    }
    return true;
}

// ------------------------------------------------------------ team kernel

struct MrhsTeamArgs {
    const MrhsP* jobs;
    int n_jobs;
    const MrhsWs* team_ws;
    GridBarrier* bars;
    int* team_job;
    int* next_job;
    int* error;
    int team_size;
    int use_tc;  // some block runs its bulk phase on the tensor cores
};

// Leaves the kernel with nothing of the CTA's in flight: outstanding copies
// waited for, the last committed MMAs waited for (bounded), tensor memory freed.
__device__ __forceinline__ void mrhs_exit(TcState& tc, bool tc_on)
{
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (tc_on) {
        if (tc.issued > 0) {
            const unsigned g = tc.issued - 1;
            mbar_wait(tc.mbar + (g % kTcStages), (g / kTcStages) & 1u);
        }
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x < 32) tmem_dealloc(tc.tmem, kTcCols);
    }
}

__global__ void __launch_bounds__(kThreads, 1) mrhs_team_kernel(const MrhsTeamArgs A)
{
    __shared__ MrhsP sP;
    __shared__ int s_job;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[kTcStages];
    const int team = blockIdx.x / A.team_size, rank = blockIdx.x % A.team_size;
    GridBarrier* bar = A.bars + team;
    unsigned int gen = 0;
    // tensor-core state for the whole launch (one CTA per SM: the allocation cannot wait)
    TcState tc;
    tc.q = 0;
    tc.issued = 0;
    tc.mbar = s_mbar;
    tc.tmem = 0;
    if (A.use_tc) {
        if (threadIdx.x < kTcStages) mbar_init(&s_mbar[threadIdx.x], 1);
        if (threadIdx.x < 32) tmem_alloc(&s_tmem, kTcCols);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        tc.tmem = s_tmem;
    }
    for (;;) {
        if (threadIdx.x == 0 && rank == 0) {
            int j = atomicAdd(A.next_job, 1);
            A.team_job[team] = j < A.n_jobs ? j : -1;
        }
        if (!grid_sync(bar, A.team_size, gen)) {
            if (threadIdx.x == 0) atomicExch(A.error, 1);
            mrhs_exit(tc, A.use_tc);
            return;
        }
        if (threadIdx.x == 0) s_job = __ldcg(A.team_job + team);
        __syncthreads();
        const int j = s_job;
        if (j < 0) {
            mrhs_exit(tc, A.use_tc);
            return;
        }
        if (threadIdx.x == 0) {
            sP = A.jobs[j];
            sP.ws = A.team_ws[team];
        }
        __syncthreads();
        if (!mrhs_body(sP, rank, A.team_size, bar, gen, tc)) {
            if (threadIdx.x == 0) atomicExch(A.error, 1);
            if (threadIdx.x == 0 && rank == 0)
                for (int r = 0; r < sP.R; r++) sP.res[r].status = kDevTimeout;
            mrhs_exit(tc, A.use_tc);
            return;
        }
        // the next job reuses the team's workspace: every CTA leaves this one first
        if (!grid_sync(bar, A.team_size, gen)) {
            if (threadIdx.x == 0) atomicExch(A.error, 1);
            mrhs_exit(tc, A.use_tc);
            return;
        }
    }
}

// ------------------------------------------------------------ host side

namespace {

struct MrhsGeom {
    int npad, ntile;
    size_t ws_bytes;
};

size_t mrhs_layout(char* base, int N, int K, int G, bool dome, MrhsWs* w)
{
    const int npad = (N + kMSynRows - 1) / kMSynRows * kMSynRows;
    const int ntile = npad / kMSynRows;
    Bump bp{base, 0};
    w->Yt = bp.take<float>((size_t)kMR * npad);
    w->Th = bp.take<float>((size_t)kMR * npad);
    w->Dst = bp.take<float>((size_t)kMR * npad);
    w->Thi = bp.take<uint16_t>((size_t)kMR * npad);
    w->Tlo = bp.take<uint16_t>((size_t)kMR * npad);
    w->Q0 = bp.take<double>((size_t)K * kMR);
    w->Q1 = bp.take<double>((size_t)K * kMR);
    w->Q2 = dome ? bp.take<double>((size_t)K * kMR) : nullptr;
    w->invn = bp.take<double>(K);
    w->xb[0] = bp.take<FF>((size_t)K * kMR);
    w->xb[1] = bp.take<FF>((size_t)K * kMR);
    w->u = bp.take<FF>((size_t)K * kMR);
    w->amask = bp.take<unsigned long long>(K);
    w->nzmask = bp.take<unsigned long long>(K);
    w->kzmask = bp.take<unsigned long long>(K);
    for (int l = 0; l < 3; l++) {
        w->act[l][0] = bp.take<int>(K);
        w->act[l][1] = bp.take<int>(K);
    }
    w->keep = bp.take<int>(K);
    w->nz_col = bp.take<int>((size_t)kMR * K);
    w->nz_x = bp.take<FF>((size_t)kMR * K);
    w->wb[0] = bp.take<FF>((size_t)kMR * npad);
    w->wb[1] = bp.take<FF>((size_t)kMR * npad);
    w->part = bp.take<float>((size_t)2 * 2 * G * kMTA * kMR * 2);
    w->tilecnt = bp.take<int>((size_t)2 * ((K + kMTA - 1) / kMTA));
    w->ctr = bp.take<int>(3);
    w->p_m = bp.take<float>((size_t)kMR * G);
    w->p_l1 = bp.take<FF>((size_t)kMR * G);
    w->c_na = bp.take<int>((size_t)kMR * G);
    w->c_nnzx = bp.take<int>((size_t)kMR * G);
    w->c_nz = bp.take<int>((size_t)kMR * G);
    w->c_keep = bp.take<int>((size_t)3 * G);
    w->s_alo = bp.take<int>(G);
    w->p_v = bp.take<double>((size_t)kMR * G);
    w->p_i = bp.take<int>((size_t)kMR * G);
    w->p_a = bp.take<FF>((size_t)kMR * ntile);
    w->p_b = bp.take<FF>((size_t)kMR * ntile);
    w->p_r = bp.take<FF>((size_t)kMR * ntile);
    return bp.off + 256;
}

}  // namespace

struct MrhsPlan {
    ds_ctx* ctx;
    int n_jobs;
    std::vector<MrhsBlock> blocks;
    void* dmem;
    MrhsP* hjobs;       // pinned
    double* hlam;       // pinned, [n_jobs][kMR]
    DevResult* hres;    // pinned, [n_jobs][kMR]
    MrhsP* djobs;
    double* dlam;
    DevResult* dres;
    void* dctl;
    size_t ctl_bytes;
    int* derr;
    MrhsTeamArgs args;
    int grid;
    size_t smem;
};

ds_status mrhs_plan_create(ds_ctx* ctx, int n_blocks, const MrhsBlock* blocks, const ds_options* opt,
                           const double* fista_dev, int fista_n, const MrhsCfg& cfg, MrhsPlan** out)
{
    *out = nullptr;
    if (n_blocks < 1) return DS_ERR_INVALID;
    MrhsPlan* M = new (std::nothrow) MrhsPlan();
    if (!M) return DS_ERR_OOM;
    M->ctx = ctx;
    M->n_jobs = n_blocks;
    M->blocks.assign(blocks, blocks + n_blocks);
    // largest blocks first
    std::vector<int> ord(n_blocks);
    for (int i = 0; i < n_blocks; i++) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) {
        return (double)blocks[a].dict->N * blocks[a].dict->K * blocks[a].R >
               (double)blocks[c].dict->N * blocks[c].dict->K * blocks[c].R;
    });
    int maxN = 1, maxK = 1;
    for (int i = 0; i < n_blocks; i++) {
        maxN = std::max(maxN, (int)blocks[i].dict->N);
        maxK = std::max(maxK, (int)blocks[i].dict->K);
    }
    // CTAs per team: every SM busy when there are few blocks (SMs / blocks each), and at least 8 when
    // there are many: a block on one or two CTAs keeps its SMs busy with its own latency-bound phases
    // (measured on 256 blocks of 64 right-hand sides: 8-CTA teams 1.8x faster than 2-CTA teams)
    const int sms = std::min(ctx->num_sms, kMaxG);
    int team = std::max(std::min(8, sms), sms / n_blocks);
    if (cfg.team_size > 0) team = cfg.team_size;
    team = std::min(team, sms);
    const int n_teams = std::max(1, std::min(std::min(ctx->num_sms, kMaxG) / team, n_blocks));
    const bool dome = opt->test == DS_DOME;
    MrhsWs wtmp;
    const size_t ws_team = align_up(mrhs_layout(nullptr, maxN, maxK, team, dome, &wtmp), 256);
    const size_t jobs_bytes = align_up(sizeof(MrhsP) * n_blocks, 256);
    const size_t lam_bytes = align_up(sizeof(double) * kMR * n_blocks, 256);
    const size_t res_bytes = align_up(sizeof(DevResult) * kMR * n_blocks, 256);
    const size_t tws_bytes = align_up(sizeof(MrhsWs) * n_teams, 256);
    M->ctl_bytes = align_up(sizeof(GridBarrier) * n_teams + sizeof(int) * (n_teams + 2), 256);
    const size_t total = ws_team * n_teams + jobs_bytes + lam_bytes + res_bytes + tws_bytes + M->ctl_bytes;
    auto fail = [&](ds_status s) {
        mrhs_plan_destroy(M);
        return s;
    };
    if (cudaMalloc(&M->dmem, total) != cudaSuccess) {
        cudaGetLastError();
        M->dmem = nullptr;
        return fail(DS_ERR_OOM);
    }
    if (cudaMallocHost((void**)&M->hjobs, jobs_bytes) != cudaSuccess ||
        cudaMallocHost((void**)&M->hlam, lam_bytes) != cudaSuccess ||
        cudaMallocHost((void**)&M->hres, res_bytes) != cudaSuccess)
        return fail(DS_ERR_OOM);
    char* d = reinterpret_cast<char*>(M->dmem);
    char* wsbase = d;
    d += ws_team * n_teams;
    M->djobs = reinterpret_cast<MrhsP*>(d);
    d += jobs_bytes;
    M->dlam = reinterpret_cast<double*>(d);
    d += lam_bytes;
    M->dres = reinterpret_cast<DevResult*>(d);
    d += res_bytes;
    MrhsWs* dtws = reinterpret_cast<MrhsWs*>(d);
    d += tws_bytes;
    M->dctl = d;
    GridBarrier* bars = reinterpret_cast<GridBarrier*>(M->dctl);
    int* team_job = reinterpret_cast<int*>(bars + n_teams);
    int* next_job = team_job + n_teams;
    M->derr = next_job + 1;
    std::vector<MrhsWs> tws(n_teams);
    for (int t = 0; t < n_teams; t++) mrhs_layout(wsbase + ws_team * t, maxN, maxK, team, dome, &tws[t]);
    if (cudaMemcpy(dtws, tws.data(), sizeof(MrhsWs) * n_teams, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(DS_ERR_CUDA);
    int use_tc = 0;
    for (int jj = 0; jj < n_blocks; jj++) {
        const int j = ord[jj];
        const MrhsBlock& B = blocks[j];
        const ds_dict* dc = B.dict;
        MrhsP P;
        std::memset(&P, 0, sizeof(P));
        P.D = reinterpret_cast<const float*>(dc->D);
        P.N = (int)dc->N;
        P.K = (int)dc->K;
        P.ld = (int)dc->ld;
        P.npad = (P.N + kMSynRows - 1) / kMSynRows * kMSynRows;
        P.ntile = P.npad / kMSynRows;
        P.colnorm = dc->colnorm;
        P.fmax = dc->fmax;
        P.L = opt->L > 0.0 ? opt->L : dc->L;
        {
            // rounding of the FP32 contraction: 32 FMAs a chunk, the chunk sums, the sums of the
            // parked partial tiles (at most one per chunk)
            const double u = std::ldexp(1.0, -24);
            const double k = 32.0 + 2.0 * (P.npad / kMKC) + 2.0;
            P.gamma = 1.01 * k * u / (1.0 - k * u);
        }
        P.eps_test = 1e-9;
        P.tol = opt->tol_gap_rel;
        P.alg = opt->alg;
        P.test = opt->test;
        P.dynamic = opt->dynamic;
        P.max_iter = opt->max_iter;
        P.lambda_rel = opt->lambda_rel;
        P.Y = reinterpret_cast<const float*>(B.Y);
        P.R = B.R;
        for (int r = 0; r < kMR; r++) P.ridx[r] = r < B.R ? B.ridx[r] : 0;
        P.lambdas = M->dlam + (size_t)jj * kMR;
        P.X = reinterpret_cast<float*>(B.X);
        P.res = M->dres + (size_t)jj * kMR;
        P.fista = fista_dev;
        P.fista_n = fista_n;
        if (dc->lo_kind == 1 && cfg.allow_tc) {
            // precision variant with a BF16 copy: bulk iterations on the tensor cores
            P.Dlo = reinterpret_cast<const uint16_t*>(dc->Dlo);
            P.ld_lo = (int)dc->ld_lo;
            P.use_tc = 1;
            P.emax = dc->emax;
            {
                // tensor-core sums, bounded as if every addition of a K = 16 step (16 products and
                // the accumulator) truncated to FP32 (unit 2^-23), plus the sums of the parked
                // partial tiles (at most one per 64-row chunk) and hi + lo
                const double u = std::ldexp(1.0, -23);
                const double k = 17.0 * (P.npad / 16) + (P.npad / kTcRows) + 2.0;
                P.gamma_tc = 1.01 * k * u / (1.0 - k * u);
            }
            P.lo_switch = cfg.lo_switch > 0.0 ? cfg.lo_switch
                                              : (opt->lowp_switch > 0.0 ? opt->lowp_switch : std::max(1e-3, opt->tol_gap_rel));
            use_tc = 1;
        }
        M->hjobs[jj] = P;
    }
    // keep the job order for lambdas/results
    std::vector<MrhsBlock> sorted(n_blocks);
    for (int jj = 0; jj < n_blocks; jj++) sorted[jj] = blocks[ord[jj]];
    M->blocks = sorted;
    std::memset(&M->args, 0, sizeof(M->args));
    M->args.jobs = M->djobs;
    M->args.n_jobs = n_blocks;
    M->args.team_ws = dtws;
    M->args.bars = bars;
    M->args.team_job = team_job;
    M->args.next_job = next_job;
    M->args.error = M->derr;
    M->args.team_size = team;
    M->args.use_tc = use_tc;
    M->grid = n_teams * team;
    M->smem = sizeof(MrhsShared) + 1024;  // + alignment of the staging area
    if (cudaFuncSetAttribute(mrhs_team_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)M->smem) !=
        cudaSuccess)
        return fail(DS_ERR_CUDA);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mrhs_team_kernel, kThreads, M->smem) != cudaSuccess ||
        occ < 1)
        return fail(DS_ERR_UNSUPPORTED);
    *out = M;
    return DS_OK;
}

const MrhsBlock* mrhs_plan_blocks(const MrhsPlan* M, int* n)
{
    *n = M->n_jobs;
    return M->blocks.data();
}

double* mrhs_plan_lambdas(MrhsPlan* M) { return M->hlam; }
const DevResult* mrhs_plan_results(const MrhsPlan* M) { return M->hres; }

ds_status mrhs_plan_enqueue(MrhsPlan* M, cudaStream_t s)
{
    if (cudaMemcpyAsync(M->djobs, M->hjobs, sizeof(MrhsP) * M->n_jobs, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaMemcpyAsync(M->dlam, M->hlam, sizeof(double) * kMR * M->n_jobs, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaMemsetAsync(M->dctl, 0, M->ctl_bytes, s) != cudaSuccess) return DS_ERR_CUDA;
    if (cudaMemsetAsync(M->dres, 0, sizeof(DevResult) * kMR * M->n_jobs, s) != cudaSuccess) return DS_ERR_CUDA;
    void* args[] = {(void*)&M->args};
    if (cudaLaunchCooperativeKernel((const void*)mrhs_team_kernel, dim3(M->grid), dim3(kThreads), args, M->smem, s) !=
        cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaMemcpyAsync(M->hres, M->dres, sizeof(DevResult) * kMR * M->n_jobs, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return DS_ERR_CUDA;
    return DS_OK;
}

int* mrhs_plan_error_flag(MrhsPlan* M) { return M->derr; }

void mrhs_plan_info(const MrhsPlan* M, int* teams, int* team_size)
{
    if (team_size) *team_size = M->args.team_size;
    if (teams) *teams = M->grid / M->args.team_size;
}

void mrhs_plan_destroy(MrhsPlan* M)
{
    if (!M) return;
    if (M->dmem) cudaFree(M->dmem);
    if (M->hjobs) cudaFreeHost(M->hjobs);
    if (M->hlam) cudaFreeHost(M->hlam);
    if (M->hres) cudaFreeHost(M->hres);
    delete M;
}

}  // namespace ds
