// ds_small.cu -- a whole screened ISTA / FISTA solve (Algorithm 3 with the
// Table 1 updates) of a small FP64 Lasso problem on one thread-block cluster.
//
// On GB300 a dependent FP64 operation takes about 64 cycles and a grid-wide
// barrier microseconds, so for a problem of a few hundred atoms the persistent
// kernel's iteration is bound by both, not by the dictionary stream.  Here the
// C <= 8 CTAs of one cluster hold the dictionary in shared memory as
// float-float pairs (hi + lo, about 48 significant bits; one slice of columns
// per CTA, one atom per thread), exchange partial sums through distributed
// shared memory and meet at one cluster barrier per iteration.  Iteration t:
//
//   (1) each CTA synthesises its atoms' part of D ubar_{t-1} and D xbar_{t-1}
//       over their nonzeros (the test of iteration t-1 still pending) and
//       writes it, with its part of ||xbar_{t-1}||_1 and its max |z_{t-1}|,
//       into its own shared memory; it arrives at the cluster barrier and,
//       before it waits, computes the Lemma 8 terms of theta_{t-1} that do
//       not need the cluster's max |z_{t-1}|;
//   (2) after the barrier every CTA reads the C parts from the others' shared
//       memory (a pull) and adds them in rank order: the cluster's max
//       |z_{t-1}| completes the Lemma 8 dual scaling and the radius of the
//       test of t-1 (Lemmas 2-4), while theta_t = D ubar_{t-1} - y, the
//       residual D xbar_{t-1} - y and their sums are formed.  The test is
//       applied to the CTA's atoms; when it may have screened a nonzero atom
//       (the dome test: always) a second exchange takes those atoms' parts
//       back out of theta_t;
//   (3) the active atoms are correlated, z = d^T theta_t, with several lanes
//       per atom when few are active, while one warp takes the duality gap of
//       iteration t-1 and the stopping rule; then the proximal step and the
//       FISTA extrapolation.
//
// When warps 6 and 7 of a CTA hold neither atoms nor rows and the test is a
// sphere test, (3) does not wait for the test: warps 0..5 correlate the atoms
// that were active before it while warp 7 runs the Lemma 8 chain and the
// radius (FP64, one dependent operation at a time) and warp 6 the primal half
// of the gap; the atoms the test then screens drop their z.  After a
// correction exchange the correlation and the gap are redone on the corrected
// theta_t.
//
// Every CTA computes the scalars from the same data in the same order, and the
// loop ends on rank 0's decision, which every CTA reads: all CTAs pass the
// same barriers.  Float-float sums carry an explicit error bound into the
// dual scaling and the radius, so the test stays safe.
#include <cooperative_groups.h>

#include "ds_solve_body.cuh"

namespace cg = cooperative_groups;

namespace ds {

constexpr int kSmThreads = 256;  // one atom per thread
constexpr int kSmMaxN = 256;     // rows
constexpr int kSmMaxC = 8;       // CTAs of the cluster (portable cluster size)

struct SmScal {  // a CTA's scalars in an iteration's exchange (its vectors go to the vector slots)
    float l1s, l1c;  // its part of ||xbar||_1 (a Dot2 pair)
    float mh, ml;    // max |z| over its atoms in the last correlation (exact float-float)
    float mq;        // max over its nonzero atoms of (thr - eps)^2 rounded up (sphere tests)
    int pad;
};
struct SmPay0 {  // precompute: a CTA's max |d_i^T y|, its (lowest) atom and the sign of d_i^T y there
    double v, sg;
    int i, pad;
};

// z = d^T v for the thread's atom column `a` of the float-float slice and a float-float vector:
// the hi x hi products with their exact errors (TwoProduct) and the running sum with its exact
// errors (TwoSum) as in Dot2 (Ogita, Rump, Oishi), the cross terms hi x lo + lo x hi in FP32.
__device__ __forceinline__ double sm_col_dot(const float* Dh, const float* Dl, int pitch, int a, const FF* v, int N)
{
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;  // even and odd rows: two independent chains
    int r = 0;
    for (; r + 1 < N; r += 2) {
        const float dh0 = Dh[r * pitch + a], dl0 = Dl[r * pitch + a];
        const float dh1 = Dh[(r + 1) * pitch + a], dl1 = Dl[(r + 1) * pitch + a];
        const FF v0 = v[r], v1 = v[r + 1];
        const float p0 = dh0 * v0.h, p1 = dh1 * v1.h;
        const float e0 = fmaf(dh0, v0.h, -p0), e1 = fmaf(dh1, v1.h, -p1);
        const float t0 = s0 + p0, t1 = s1 + p1;
        const float b0 = t0 - s0, b1 = t1 - s1;
        c0 += ((s0 - (t0 - b0)) + (p0 - b0)) + e0 + fmaf(dh0, v0.l, dl0 * v0.h);
        c1 += ((s1 - (t1 - b1)) + (p1 - b1)) + e1 + fmaf(dh1, v1.l, dl1 * v1.h);
        s0 = t0;
        s1 = t1;
    }
    if (r < N) {
        const float dh0 = Dh[r * pitch + a], dl0 = Dl[r * pitch + a];
        const FF v0 = v[r];
        const float p0 = dh0 * v0.h;
        const float e0 = fmaf(dh0, v0.h, -p0);
        const float t0 = s0 + p0, b0 = t0 - s0;
        c0 += ((s0 - (t0 - b0)) + (p0 - b0)) + e0 + fmaf(dh0, v0.l, dl0 * v0.h);
        s0 = t0;
    }
    return ((double)s0 + (double)s1) + ((double)c0 + (double)c1);
}

// 1/m rounded below: the FP32 reciprocal and one Newton step, r0 (2 - m r0) = (1/m)(1 - d^2) for
// r0 = (1 + d)/m, scaled by 1 - 2^-50 so that the FP64 roundings keep it below 1/m (a feasible dual
// scaling in Lemma 8); relative error about 2^-48 for m in the FP32 range.
__device__ __forceinline__ double rcp_lo(double m)
{
    const float mf = (float)m;
    if (!(mf > 1e-30f && mf < 1e30f)) return (1.0 / m) * (1.0 - 0x1p-50);
    const double r0 = (double)__frcp_rn(mf);
    return fma(r0, fma(-m, r0, 1.0), r0) * (1.0 - 0x1p-50);
}

// The cluster barrier in two halves (release on arrival, acquire on the wait), so that a CTA can work
// between announcing its data and waiting for the others'.
// The .aligned forms need every warp converged: each half starts with a warp barrier.
__device__ __forceinline__ void cluster_arrive()
{
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait()
{
    __syncwarp();
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Named CTA barriers for a subset of the warps (id 1 and 2; __syncthreads is id 0): `n` threads in
// whole warps.  A warp that arrives does not wait; the barrier completes when n threads have arrived
// or synced, and orders their shared-memory writes before the reads of the threads that synced.
__device__ __forceinline__ void named_sync(int id, int n)
{
    __syncwarp();
    asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n)
{
    __syncwarp();
    asm volatile("barrier.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// The same dot product as a float-float pair, on four independent chains (rows r mod 4) merged exactly.
__device__ __forceinline__ void sm_dot_step(float& s, float& c, float dh, float dl, FF v)
{
    const float p = dh * v.h;
    const float e = fmaf(dh, v.h, -p);
    const float t = s + p, b = t - s;
    c += ((s - (t - b)) + (p - b)) + e + fmaf(dh, v.l, dl * v.h);
    s = t;
}
__device__ __forceinline__ FF sm_col_dot_ff(const float* Dh, const float* Dl, int pitch, int a, const FF* v, int N)
{
    float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f, s3 = 0.f, c3 = 0.f;
    int r = 0;
    for (; r + 3 < N; r += 4) {
        sm_dot_step(s0, c0, Dh[r * pitch + a], Dl[r * pitch + a], v[r]);
        sm_dot_step(s1, c1, Dh[(r + 1) * pitch + a], Dl[(r + 1) * pitch + a], v[r + 1]);
        sm_dot_step(s2, c2, Dh[(r + 2) * pitch + a], Dl[(r + 2) * pitch + a], v[r + 2]);
        sm_dot_step(s3, c3, Dh[(r + 3) * pitch + a], Dl[(r + 3) * pitch + a], v[r + 3]);
    }
    for (; r < N; r++) sm_dot_step(s0, c0, Dh[r * pitch + a], Dl[r * pitch + a], v[r]);
    Dot2f acc;
    acc.s = s0;
    acc.c = c0;
    dot2_merge(acc, s1, c1);
    dot2_merge(acc, s2, c2);
    dot2_merge(acc, s3, c3);
    return ff_two_sum(acc.s, acc.c);
}

// acc += a * b for float-float a, b (Dot2 with the cross terms), as above.
__device__ __forceinline__ void sm_acc(Dot2f& acc, FF a, FF b)
{
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p);
    const float t = acc.s + p, bb = t - acc.s;
    acc.c += ((acc.s - (t - bb)) + (p - bb)) + e + fmaf(a.h, b.l, a.l * b.h);
    acc.s = t;
}

// Block sums of up to three Dot2 accumulators (rows 0..N-1 on threads 0..N-1), merged in warp order;
// thread 0 gets the values.
__device__ __forceinline__ void sm_block_sum3(Dot2f& a, Dot2f& b, Dot2f& c, float (*red)[6], double* out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    a = dot2_warp_reduce(a);
    b = dot2_warp_reduce(b);
    c = dot2_warp_reduce(c);
    if (lane == 0) {
        red[warp][0] = a.s; red[warp][1] = a.c;
        red[warp][2] = b.s; red[warp][3] = b.c;
        red[warp][4] = c.s; red[warp][5] = c.c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Dot2f ta, tb, tc;
        for (int w = 0; w < kSmThreads / 32; w++) {
            dot2_merge(ta, red[w][0], red[w][1]);
            dot2_merge(tb, red[w][2], red[w][3]);
            dot2_merge(tc, red[w][4], red[w][5]);
        }
        out[0] = ta.value();
        out[1] = tb.value();
        out[2] = tc.value();
    }
}

__global__ void __launch_bounds__(kSmThreads, 1) small_kernel(const SolveP<double> P, int pitch)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = P.N, K = P.K;
    const int n_loc = (K + C - 1) / C;
    const int a0 = rank * n_loc;
    const int na_loc = max(0, min(n_loc, K - a0));
    const int a = tid, ai = a0 + a;
    const bool own = a < na_loc;

    extern __shared__ __align__(16) float sm_dyn[];
    float* const Dh = sm_dyn;               // [N][pitch], atom-contiguous rows
    float* const Dl = sm_dyn + (size_t)N * pitch;
    __shared__ FF s_y[kSmMaxN], s_th[kSmMaxN], s_ds[kSmMaxN];
    __shared__ SmPay0 p0;
    __shared__ int s_lc[kSmThreads];
    __shared__ FF s_lu[kSmThreads], s_lx[kSmThreads];
    __shared__ float s_red[kSmThreads / 32][6];
    __shared__ double s_dv[kSmThreads / 32];
    __shared__ int s_iv[kSmThreads / 32];
    __shared__ double s_sc[24];
    __shared__ int s_si[8];

    // ---------------------------------------- dictionary slice and y, as float-float pairs
    for (int idx = tid; idx < na_loc * N; idx += kSmThreads) {
        const int c = idx / N, r = idx - c * N;
        const float2 d = P.Dff[(size_t)a0 * N + idx];  // column a0 + c, row r
        Dh[r * pitch + c] = d.x;
        Dl[r * pitch + c] = d.y;
    }
    for (int r = tid; r < N; r += kSmThreads) s_y[r] = ff_from_double(P.y[r]);
    __syncthreads();

    // ---------------------------------------- b = D^T y, ||y||^2, lambda_* (Sec. 2.2.2)
    const double b_a = own ? sm_col_dot(Dh, Dl, pitch, a, s_y, N) : 0.0;
    {
        Dot2f yq, z1, z2;
        if (tid < N) sm_acc(yq, s_y[tid], s_y[tid]);
        sm_block_sum3(yq, z1, z2, s_red, &s_sc[0]);  // s_sc[0] = ||y||^2
        // lowest atom attaining max |b_i|, with the sign of b there (d_* = sign(b_{i*}) d_{i*}, Lemma 3)
        double best = own ? fabs(b_a) : -1.0, bsg = b_a < 0.0 ? -1.0 : 1.0;
        int arg = own ? ai : 0x7fffffff;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const double os = __shfl_xor_sync(0xffffffffu, bsg, o);
            const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
            if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; bsg = os; }
        }
        if (lane == 0) { s_dv[warp] = best; s_iv[warp] = arg; }
        __shared__ double s_sg[kSmThreads / 32];
        if (lane == 0) s_sg[warp] = bsg;
        __syncthreads();
        if (tid == 0) {
            double bb = -1.0, bs = 1.0;
            int ba = 0x7fffffff;
            for (int w = 0; w < kSmThreads / 32; w++)
                if (s_dv[w] > bb || (s_dv[w] == bb && s_iv[w] < ba)) { bb = s_dv[w]; ba = s_iv[w]; bs = s_sg[w]; }
            p0.v = bb;
            p0.i = ba;
            p0.sg = bs;
        }
    }
    cl.sync();
    if (tid == 0) {
        double bb = -1.0, bs = 1.0;
        int ba = 0x7fffffff;
        for (int c = 0; c < C; c++) {
            const SmPay0* q = cl.map_shared_rank(&p0, c);
            const double v = q->v;
            const int i = q->i;
            if (v > bb || (v == bb && i < ba)) { bb = v; ba = i; bs = q->sg; }
        }
        s_sc[1] = bb;  // lambda_*
        s_sc[2] = bs;  // sign of b_{i*}
        s_si[0] = ba;  // i_*
    }
    __syncthreads();
    const double yy = s_sc[0], lstar = s_sc[1];
    const int star = s_si[0];
    const double lam = P.lambda_rel ? P.lam0 * lstar : P.lam0;
    const int test = P.test;
    const bool need_n = test == 2 || test == 3;  // DST3, Dome: d_* (Lemma 3)
    int* const slog = (P.scr_log && P.scr_rows > 0) ? P.scr_log : nullptr;
    DevResult* const R = P.res;

    if (!(lam < lstar)) {
        // x = 0 and theta = y / lambda is dual optimal (Sec. 2.2.2)
        if (own) {
            P.x_out[ai] = 0.0;
            if (slog) slog[ai] = 0;
        }
        if (rank == 0 && tid == 0) {
            R->iters = 0; R->status = kDevOk; R->n_active = 0; R->nnz = 0;
            R->gap = 0.0; R->primal = 0.5 * yy; R->dual = 0.5 * yy; R->lambda = lam; R->lambda_max = lstar;
            R->cols_corr = K; R->cols_synth = 0; R->cols_lowp = 0;
        }
        cl.sync();
        return;
    }

    // ---------------------------------------- d_* and D^T d_* (Lemma 3; dome, Lemma 4)
    double tv_a = 0.0, nn = 0.0;
    if (need_n) {
        // d_* = sign(b_{i*}) d_{i*}, read from the CTA that holds column i_* (its slice is loaded and never
        // written again), then ||d_*||^2 and each atom's d_i^T d_*
        const int rs = star / n_loc, cs = star - rs * n_loc;
        const float* rh = cl.map_shared_rank(Dh, rs);
        const float* rl = cl.map_shared_rank(Dl, rs);
        const float sg = (float)s_sc[2];
        for (int r = tid; r < N; r += kSmThreads) s_ds[r] = FF{sg * rh[r * pitch + cs], sg * rl[r * pitch + cs]};
        __syncthreads();
        Dot2f q, z1, z2;
        if (tid < N) sm_acc(q, s_ds[tid], s_ds[tid]);
        sm_block_sum3(q, z1, z2, s_red, &s_sc[3]);  // ||d_*||^2 on thread 0
        __syncthreads();
        nn = s_sc[3];
        if (own) tv_a = sm_col_dot(Dh, Dl, pitch, a, s_ds, N);
    }

    // ---------------------------------------- constants of lambda (Lemmas 2-4, Lemma 8)
    const double inv_lam = 1.0 / lam, yy_l2 = yy * inv_lam * inv_lam;
    const double psi = lstar * inv_lam - 1.0;
    // Lasso: n = d_*, n^T y = lambda_*, ||n||^2 = ||d_*||^2 (Lemma 3): c = y/lambda - coef d_*
    const double coef = need_n && nn > 0.0 ? (lstar * inv_lam - 1.0) / nn : 0.0;
    const double delta = need_n && nn > 0.0 ? fabs(lstar * inv_lam - 1.0) / sqrt(nn) : 0.0;
    const double nstar = P.colnorm[star];
    const double psi_dome = psi / nstar;
    const double invL = 1.0 / P.L, thrL = lam / P.L;
    const double hyy = 0.5 * yy, hlam2 = 0.5 * lam * lam, tol_abs = P.tol * 0.5 * yy;
    // error bound of the float-float correlations, per unit ||d_i|| ||theta||: the dictionary's
    // representation (2^-48), the cross terms and the dropped lo x lo product, and the FP32 sum of the
    // Dot2 error terms ((N + 1) 2^-24 relative to their (N 2^-24) share of the sum)
    const double gam = ((double)N * N + 3.0 * N + 16.0) * 0x1p-48;
    const double fmax_d = P.fmax;

    // per-atom test data (FP64): sphere threshold (1 - |d_i^T c|) / ||d_i|| (Lemmas 2, 3); the dome's
    // d_i^T c0, t_i = d_i^T d_* / (||d_i|| ||d_*||), sqrt(1 - t_i^2) and 1 / ||d_i|| (Lemma 4)
    const double ni = own ? P.colnorm[ai] : 1.0;
    double thr_a = 0.0, dc0_a = 0.0, tt_a = 0.0, st_a = 0.0, ini_a = 0.0;
    if (own && (test == 1 || test == 2)) thr_a = (1.0 - fabs(b_a * inv_lam - coef * tv_a)) / ni;
    if (own && test == 3) {
        dc0_a = b_a / (lam * ni);
        tt_a = tv_a / (ni * nstar);
        st_a = sqrt(fmax(1.0 - tt_a * tt_a, 0.0));
        ini_a = 1.0 / ni;
    }
    // the test with radius radS (sphere) or, for the dome, R and rho = sqrt(R^2 - psi^2): the dome maximum
    // of +-d_i^T theta is dc0 + R where t R <= -psi, else dc0 - psi t + rho sqrt(1 - t^2)
    auto killed = [&](double radS, double RS, double rho) -> bool {
        if (test == 3) {
            const double up = tt_a * RS <= -psi_dome ? dc0_a + RS : dc0_a - psi_dome * tt_a + rho * st_a;
            const double dn = -tt_a * RS <= -psi_dome ? -dc0_a + RS : -dc0_a + psi_dome * tt_a + rho * st_a;
            return (ini_a - up > P.eps_test) && (ini_a - dn > P.eps_test);
        }
        return thr_a - radS > P.eps_test;
    };

    // ---------------------------------------- static test (Algorithm 1) and the starting point
    bool active = own;
    if (own) {
        bool kill = false;
        if (!P.dynamic && test != 0) {
            const double mup = lstar * (1.0 + 1e-12);
            const double mu = dual_scale(-yy, yy, lam, mup);
            const double R2 = fmax(yy / (lam * lam) + 2.0 * mu * yy / lam + mu * mu * yy, 0.0);
            const double Rr = sqrt(R2 * (1.0 + 4.0 * gam)) * (1.0 + 1e-13);
            const double rad0 = test == 2 ? sqrt(fmax(R2 * (1.0 + 4.0 * gam) - delta * delta, 0.0)) * (1.0 + 1e-13) : Rr;
            kill = killed(rad0, Rr, sqrt(fmax(Rr * Rr - psi_dome * psi_dome, 0.0)));
        }
        active = !kill;
        if (slog) slog[ai] = kill ? -1 : 0;
    }
    // the sphere test thr_i - rad > eps as (thr_i - eps)^2 > rad^2 (no square root per iteration)
    const double q_a = thr_a - P.eps_test;
    const double q2_a = q_a > 0.0 ? q_a * q_a : -1.0;
    // iterates in float-float (about 48 bits): the per-atom arithmetic stays on the FP32 pipes
    FF x_a = (active && P.x0) ? ff_from_double(P.x0[ai]) : FF{0.f, 0.f};
    FF u_a = x_a;
    const FF invL_f = ff_from_double(invL), thrL_f = ff_from_double(thrL);
    const int nwr = (N + 31) / 32;  // warps holding rows

    // ---------------------------------------- iterations
    //
    // One cluster barrier per iteration t: every CTA's parts of D ubar_{t-1} and D xbar_{t-1} over its
    // nonzero atoms travel with its max |z_{t-1}|, before the test of iteration t-1 (which needs the
    // cluster's max) is applied.  Atoms that this test screens leave the iterates (Algorithm 3); when one
    // of them was nonzero (possible only if some CTA's (thr - eps)^2 over its nonzero atoms exceeds the
    // squared radius, which every CTA sees), a second exchange subtracts their parts.
    const bool fista = P.alg == 1;
    const bool dyn = P.dynamic && test != 0;
    // the exchanges are pulled: a CTA writes its vectors and scalars into its own shared memory before the
    // barrier and reads the others' after it (distributed shared memory).  Slots k = 0, 1: the exchange of
    // iteration t in k = t & 1; k = 2: the correction exchange.  Vectors: [k][u, x][N].
    FF* const pv = reinterpret_cast<FF*>(Dl + (size_t)N * pitch);
    auto slot = [&](int k) -> FF* { return pv + (size_t)k * 2 * N; };
    __shared__ SmScal ssc[3];
    __shared__ double s_prim;  // the primal value of the gap, from warp 6 to warp 7 (overlapped order)
    __shared__ double s_lf;
    __shared__ long long s_cols_corr, s_cols_synth;
    __shared__ double s_out_gap, s_out_primal;
    __shared__ int s_wc[kSmThreads / 32], s_wc2[kSmThreads / 32];
    __shared__ float2 s_mx[kSmThreads / 32];
    __shared__ float s_mq[kSmThreads / 32];
    __shared__ FF s_bt;
    __shared__ float s_mloc_h, s_mloc_l;
    __shared__ int s_wa[kSmThreads / 32], s_al[kSmThreads];
    __shared__ FF s_z[kSmThreads];
    if (tid == 0) {
        s_lf = 1.0;
        s_cols_corr = 0;
        s_cols_synth = 0;
        s_out_gap = INFINITY;
        s_out_primal = 0.0;
        s_mloc_h = s_mloc_l = 0.f;
    }
    // threads of the scalar chains: warps with neither atoms nor rows when there are such
    const bool spare = na_loc <= kSmThreads - 64 && N <= kSmThreads - 64;
    // (with a spare warp both chains run in it, on lanes 0 and 1, as one instruction stream)
    const int t_rad = spare ? kSmThreads - 32 : 0, t_gap = spare ? kSmThreads - 31 : 32;
    const int aux = spare ? kSmThreads / 32 - 1 : 0;
    // with the spare warps and a sphere test (which rarely needs a correction exchange), warps 0..5
    // correlate the atoms that were active before the test of iteration t-1 while warp 7 runs the
    // Lemma 8 chain and warp 6 the primal half of the duality gap; the atoms that test screens then
    // drop their z
    const bool ovl = spare && !(dyn && test == 3);
    constexpr int kOvlThreads = kSmThreads - 32;  // warps 0..6: the list of the overlapped order
    // (thr - eps)^2 rounded up to FP32, for the conservative "may screen a nonzero atom" check
    const float q2f_a = q2_a > 0.0 ? __double2float_ru(q2_a) : 0.f;
    int stop_t = 0, t_last = 1;
    double lm_beta = 0.0, lm_sunc = 0.0, lm_m2a = 0.0, lm_cup = 0.0;  // radius and gap threads
    if (tid < kSmThreads / 32) s_wa[tid] = 0;  // the spare warp holds no atoms
    __syncthreads();
    for (int t = 1;; t++) {
        t_last = t;
        const int kb = t & 1;
        // ---- (1) this CTA's nonzeros of (ubar_{t-1}, x_{t-1}) in atom order (the test of t-1 pending)
        const bool nzt = active && (u_a.h != 0.f || x_a.h != 0.f);
        const unsigned bal = __ballot_sync(0xffffffffu, nzt);
        float mq = nzt ? q2f_a : 0.f;
        Dot2f l1;
        if (active && x_a.h != 0.f) dot2_merge(l1, fabsf(x_a.h), x_a.h < 0.f ? -x_a.l : x_a.l);
        l1 = dot2_warp_reduce(l1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mq = fmaxf(mq, __shfl_xor_sync(0xffffffffu, mq, o));
        if (lane == 0) {
            s_wc[warp] = __popc(bal);
            s_red[warp][0] = l1.s;
            s_red[warp][1] = l1.c;
            s_mq[warp] = mq;
        }
        __syncthreads();
        int off = 0, nl = 0;
        for (int w = 0; w < kSmThreads / 32; w++) {
            const int cw = s_wc[w];
            off += w < warp ? cw : 0;
            nl += cw;
        }
        if (nzt) {
            const int pos = off + __popc(bal & ((1u << lane) - 1u));
            s_lc[pos] = a;
            s_lu[pos] = u_a;
            s_lx[pos] = x_a;
        }
        if (warp == 0) {
            Dot2f acc;
            float m = 0.f;
            if (lane < kSmThreads / 32) {
                acc.s = s_red[lane][0];
                acc.c = s_red[lane][1];
                m = s_mq[lane];
            }
            acc = dot2_warp_reduce(acc);  // a fixed shuffle tree
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) {
                SmScal v;
                v.l1s = acc.s;
                v.l1c = acc.c;
                v.mq = m;
                v.mh = s_mloc_h;
                v.ml = s_mloc_l;
                v.pad = 0;
                ssc[kb] = v;
                s_cols_synth += nl;
            }
        }
        __syncthreads();
        if (tid < N) {
            Dot2f au, ax;
            for (int k = 0; k < nl; k++) {
                const int c = s_lc[k];
                const FF d = FF{Dh[tid * pitch + c], Dl[tid * pitch + c]};
                sm_acc(au, d, s_lu[k]);
                sm_acc(ax, d, s_lx[k]);
            }
            const FF wu0 = ff_two_sum(au.s, au.c), wx0 = ff_two_sum(ax.s, ax.c);
            reinterpret_cast<float2*>(slot(kb))[tid] = make_float2(wu0.h, wu0.l);
            reinterpret_cast<float2*>(slot(kb))[N + tid] = make_float2(wx0.h, wx0.l);
        }
        cluster_arrive();
        if (tid == t_gap) {
            // FISTA coefficient of this iteration, (l_{t-1} - 1) / l_t (Table 1), for the step after the test
            double bt = 0.0;
            if (fista) {
                if (t <= P.fista_n) {
                    bt = P.fista[2 * (t - 1)];
                    s_lf = P.fista[2 * (t - 1) + 1];
                } else {
                    const double lf = s_lf, ln = 0.5 * (1.0 + sqrt(1.0 + 4.0 * lf * lf));
                    bt = (lf - 1.0) / ln;
                    s_lf = ln;
                }
            }
            s_bt = ff_from_double(bt);
        }
        // the Lemma 8 terms of theta_{t-1} that do not need max |z_{t-1}|, computed by the threads that use
        // them while the other CTAs arrive
        if (t > 1 && (tid == t_rad || tid == t_gap)) {
            const double alpha = s_sc[4], beta = s_sc[5];  // of theta_{t-1}
            lm_beta = beta;
            lm_sunc = beta > 0.0 ? alpha * inv_lam * fast_rcp(beta) : 0.0;  // unclipped scaling
            lm_m2a = -2.0 * alpha * inv_lam;
            // rounding bound of the float-float max |z| per unit ||theta|| ||d||, times ||theta|| (up)
            lm_cup = tid == t_rad ? gam * fmax_d * (fast_sqrt(beta) * (1.0 + 1e-6)) : 0.0;
        }
        cluster_wait();

        // the auxiliary lane's parts of ||xbar_{t-1}||_1, fetched first (merged in the gap chain) so that
        // their loads overlap the Lemma 8 chain of the same warp
        float l1p_s[kSmMaxC], l1p_c[kSmMaxC];
        if ((warp == aux || (ovl && warp == aux - 1)) && lane == 3) {
#pragma unroll
            for (int c = 0; c < kSmMaxC; c++) {
                if (c < C) {
                    const SmScal* q = cl.map_shared_rank(&ssc[kb], c);
                    l1p_s[c] = q->l1s;
                    l1p_c[c] = q->l1c;
                }
            }
        }
        // ---- (2) the test of iteration t-1 (Lemma 8 with the cluster's max |z_{t-1}|, Lemmas 2-4)
        if (t > 1 && (tid == t_rad || tid == t_gap)) {
            const double beta = lm_beta, s_unc = lm_sunc, m2a = lm_m2a;
            float qh[kSmMaxC], ql[kSmMaxC], qq[kSmMaxC];
#pragma unroll
            for (int c = 0; c < kSmMaxC; c++) {
                if (c < C) {
                    const SmScal* q = cl.map_shared_rank(&ssc[kb], c);
                    qh[c] = q->mh;
                    ql[c] = q->ml;
                    qq[c] = q->mq;
                }
            }
            float mh = 0.f, ml = 0.f, mqc = 0.f;
#pragma unroll
            for (int c = 0; c < kSmMaxC; c++) {
                if (c < C) {
                    if (qh[c] > mh || (qh[c] == mh && ql[c] > ml)) { mh = qh[c]; ml = ql[c]; }
                    mqc = fmaxf(mqc, qq[c]);
                }
            }
            const double m_nom = (double)mh + (double)ml;
            // Lemma 8 on both threads in one instruction stream: the gap thread (lm_cup = 0) with the
            // nominal max |z_{t-1}|, the dual point of the gap of iteration t-1; the radius thread with an
            // upper bound on max |z| given the float-float rounding of z, for the test
            const double m_use = m_nom + lm_cup;
            double mu_s = s_unc;
            if (m_use > 0.0 && fabs(s_unc) * m_use > 1.0) mu_s = copysign(rcp_lo(m_use), s_unc);
            const double R2l = fmax(fma(mu_s, fma(mu_s, beta, m2a), yy_l2), 0.0);
            if (tid == t_gap) {
                s_sc[19] = R2l;
            } else {
                // R^2 enlarged by the bound of the errors of ||y||^2, theta^T y and ||theta||^2
                const double R2s = R2l + 4.0 * gam * (yy_l2 + mu_s * mu_s * beta);
                // squared sphere radius (Lemma 2: R; Lemma 3: sqrt(R^2 - delta^2)), rounded up a little
                const double rad2 = (test == 2 ? fmax(R2s - delta * delta, 0.0) : R2s) * (1.0 + 3e-13);
                s_sc[14] = rad2;
                if (test == 3) {
                    const double Rs = fast_sqrt(R2s) * (1.0 + 1e-13);
                    s_sc[15] = Rs;
                    s_sc[17] = sqrt(fmax(Rs * Rs - psi_dome * psi_dome, 0.0));
                }
                // a correction exchange when the test may screen a nonzero atom (the dome: always)
                s_si[3] = dyn && (test == 3 || (double)mqc > rad2);
            }
        }
        // theta_t's parts from every CTA in rank order, while the radius is computed
        FF wu = FF{0.f, 0.f}, wx = FF{0.f, 0.f};
        if (tid < N) {
            float2 pu[kSmMaxC], px[kSmMaxC];  // every part's (8-byte) load issued before the first is added
#pragma unroll
            for (int c = 0; c < kSmMaxC; c++) {
                if (c < C) {
                    const float2* const q = reinterpret_cast<const float2*>(cl.map_shared_rank(slot(kb), c));
                    pu[c] = q[tid];
                    px[c] = q[N + tid];
                }
            }
#pragma unroll
            for (int c = 0; c < kSmMaxC; c++) {
                if (c < C) {
                    wu = ff_add(wu, FF{pu[c].x, pu[c].y});
                    wx = ff_add(wx, FF{px[c].x, px[c].y});
                }
            }
        }
        // ---- theta_t = D ubar_{t-1} - y (Table 1), the residual D xbar_{t-1} - y and their sums, while
        // the radius is computed (redone below in the rare case of a correction)
        Dot2f qa, qb, qr;
        if (tid < N) {
            const FF y = s_y[tid];
            const FF th = ff_sub(wu, y), rx = ff_sub(wx, y);
            s_th[tid] = th;
            sm_acc(qa, th, y);    // theta^T y
            sm_acc(qb, th, th);   // ||theta||^2
            sm_acc(qr, rx, rx);   // ||D xbar_{t-1} - y||^2
        }
        if (!ovl || warp != aux) {  // (the spare warp of the overlapped order has no rows and is busy)
            qa = dot2_warp_reduce(qa);
            qb = dot2_warp_reduce(qb);
            qr = dot2_warp_reduce(qr);
            if (lane == 0 && warp < nwr) {
                s_red[warp][0] = qa.s; s_red[warp][1] = qa.c;
                s_red[warp][2] = qb.s; s_red[warp][3] = qb.c;
                s_red[warp][4] = qr.s; s_red[warp][5] = qr.c;
            }
        }
        if (tid == 0 && t == 1) s_si[3] = 0;

        // the duality gap of iteration t-1 and the stopping rule: lanes 0..2 of one warp sum the three row
        // sums over the row warps in order, lane 3 ||xbar_{t-1}||_1 from the C parts in rank order (minus
        // the parts of a correction exchange), lane 0 then takes the primal value; the gap needs the
        // nominal Lemma 8 point as well (s_sc[19], from the gap thread)
        auto primal_part = [&](bool with_corr) -> double {
            Dot2f acc;
            if (lane < 3) {
                for (int w = 0; w < nwr; w++) dot2_merge(acc, s_red[w][2 * lane], s_red[w][2 * lane + 1]);
            } else if (lane == 3) {
#pragma unroll
                for (int c = 0; c < kSmMaxC; c++)
                    if (c < C) dot2_merge(acc, l1p_s[c], l1p_c[c]);
                if (with_corr) {
                    float rs[kSmMaxC], rcs[kSmMaxC];
#pragma unroll
                    for (int c = 0; c < kSmMaxC; c++) {
                        if (c < C) {
                            const SmScal* r = cl.map_shared_rank(&ssc[2], c);
                            rs[c] = -r->l1s;
                            rcs[c] = -r->l1c;
                        }
                    }
#pragma unroll
                    for (int c = 0; c < kSmMaxC; c++)
                        if (c < C) dot2_merge(acc, rs[c], rcs[c]);
                }
            }
            const double sv = acc.value();
            const double alpha = __shfl_sync(0xffffffffu, sv, 0), beta = __shfl_sync(0xffffffffu, sv, 1);
            const double rr = __shfl_sync(0xffffffffu, sv, 2), l1v = __shfl_sync(0xffffffffu, sv, 3);
            double primal = 0.0;
            if (lane == 0) {
                // P(xbar_{t-1}) = lambda ||xbar_{t-1}||_1 + 1/2 ||D xbar_{t-1} - y||^2
                primal = fma(lam, l1v, 0.5 * rr);
                s_sc[4] = alpha;  // of theta_t, for the test of iteration t
                s_sc[5] = beta;
            }
            return primal;
        };
        auto gap_final = [&](double primal) {  // lane 0
            int stop = 0;
            if (t > 1) {
                // P(xbar_{t-1}) - Dual(mu theta_{t-1}), Dual(v) = 1/2||y||^2 - lambda^2/2 ||v - y/lambda||^2
                const double gap = fma(hlam2, s_sc[19], primal - hyy);
                s_out_gap = gap;
                s_out_primal = primal;
                stop = (P.tol > 0.0 && gap <= tol_abs && (t - 1) % P.gap_every == 0) || (t - 1 >= P.max_iter);
            }
            s_si[2] = stop;
        };
        auto gap_chain = [&](bool with_corr) {
            const double primal = primal_part(with_corr);
            if (lane == 0) gap_final(primal);
        };
        // z_t = d^T theta_t over the listed atoms s_al[0..nact), G lanes per atom; each lane sums rows
        // q, q + G, ... on two chains and the G partial sums merge by a fixed shuffle tree
        auto correlate = [&](int G, int nact) {
            const int j = tid / G, q = tid - j * G;
            float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
            if (j < nact) {
                const int aj = s_al[j];
                int r = q;
                for (; r + G < N; r += 2 * G) {
                    sm_dot_step(s0, c0, Dh[r * pitch + aj], Dl[r * pitch + aj], s_th[r]);
                    sm_dot_step(s1, c1, Dh[(r + G) * pitch + aj], Dl[(r + G) * pitch + aj], s_th[r + G]);
                }
                if (r < N) sm_dot_step(s0, c0, Dh[r * pitch + aj], Dl[r * pitch + aj], s_th[r]);
            }
            Dot2f acc;
            acc.s = s0;
            acc.c = c0;
            dot2_merge(acc, s1, c1);
            for (int o = 1; o < G; o <<= 1) {
                const float os = __shfl_xor_sync(0xffffffffu, acc.s, o), oc = __shfl_xor_sync(0xffffffffu, acc.c, o);
                dot2_merge(acc, os, oc);
            }
            if (q == 0 && j < nact) s_z[j] = ff_two_sum(acc.s, acc.c);
        };
        // this thread's atom in the list of the atoms correlated, and the warp's ballot of them
        unsigned bact = 0;
        int apos = 0;
        if (ovl) {
            if (warp != aux) {
                // the atoms active before the test of iteration t-1, correlated by warps 0..5 while warp 7
                // runs the Lemma 8 chain and warp 6 the primal part of the gap; those the test screens then
                // drop their z
                bact = __ballot_sync(0xffffffffu, active);
                if (lane == 0) s_wa[warp] = __popc(bact);
                named_sync(1, kOvlThreads);  // also publishes the row sums to warp 6
                int offa = 0, nact = 0;
                for (int w = 0; w < kSmThreads / 32; w++) {
                    const int cw = s_wa[w];
                    offa += w < warp ? cw : 0;
                    nact += cw;
                }
                apos = offa + __popc(bact & ((1u << lane) - 1u));
                if (active) s_al[apos] = a;
                int G = 1;
                while (G < 32 && 2 * G * nact <= kOvlThreads - 32) G *= 2;
                named_sync(1, kOvlThreads);
                if (warp < aux - 1) {
                    correlate(G, nact);
                } else {
                    const double primal = primal_part(false);
                    if (lane == 0) s_prim = primal;
                    named_arrive(2, 64);  // the primal value, to warp 7
                }
            } else {
                named_sync(2, 64);  // warp 6's primal value; s_sc[19] is this warp's own
                if (lane == 0) gap_final(s_prim);
            }
        }
        __syncthreads();
        const int corr = s_si[3];
        // dynamic screening with theta_{t-1} (Algorithm 3): the screened atoms leave xbar and ubar
        bool scr = false;
        if (t > 1 && dyn && active && (test == 3 ? killed(0.0, s_sc[15], s_sc[17]) : q2_a > s_sc[14])) {
            scr = true;
            active = false;
            if (slog) slog[ai] = t - 1;
        }
        if (corr) {
            // the screened atoms that were nonzero: their parts (and |x|) are taken back out
            const bool sn = scr && nzt;
            const unsigned b2 = __ballot_sync(0xffffffffu, sn);
            Dot2f cl1;
            if (sn && x_a.h != 0.f) dot2_merge(cl1, fabsf(x_a.h), x_a.h < 0.f ? -x_a.l : x_a.l);
            cl1 = dot2_warp_reduce(cl1);
            if (lane == 0) {
                s_wc2[warp] = __popc(b2);
                s_red[warp][2] = cl1.s;
                s_red[warp][3] = cl1.c;
            }
            __syncthreads();
            int off2 = 0, n2 = 0;
            for (int w = 0; w < kSmThreads / 32; w++) {
                const int cw = s_wc2[w];
                off2 += w < warp ? cw : 0;
                n2 += cw;
            }
            if (sn) {
                const int pos = off2 + __popc(b2 & ((1u << lane) - 1u));
                s_lc[pos] = a;
                s_lu[pos] = u_a;
                s_lx[pos] = x_a;
            }
            if (warp == 0) {
                Dot2f acc;
                if (lane < kSmThreads / 32) {
                    acc.s = s_red[lane][2];
                    acc.c = s_red[lane][3];
                }
                acc = dot2_warp_reduce(acc);
                if (lane == 0) {
                    SmScal v;
                    v.l1s = acc.s;
                    v.l1c = acc.c;
                    v.mh = v.ml = v.mq = 0.f;
                    v.pad = 0;
                    ssc[2] = v;
                }
            }
            __syncthreads();
            if (tid < N) {
                Dot2f au, ax;
                for (int k = 0; k < n2; k++) {
                    const int c = s_lc[k];
                    const FF d = FF{Dh[tid * pitch + c], Dl[tid * pitch + c]};
                    sm_acc(au, d, s_lu[k]);
                    sm_acc(ax, d, s_lx[k]);
                }
                const FF cu0 = ff_two_sum(au.s, au.c), cx0 = ff_two_sum(ax.s, ax.c);
                reinterpret_cast<float2*>(slot(2))[tid] = make_float2(cu0.h, cu0.l);
                reinterpret_cast<float2*>(slot(2))[N + tid] = make_float2(cx0.h, cx0.l);
            }
            cl.sync();
            if (tid < N) {
                float2 pu[kSmMaxC], px[kSmMaxC];
#pragma unroll
                for (int c = 0; c < kSmMaxC; c++) {
                    if (c < C) {
                        const float2* const q = reinterpret_cast<const float2*>(cl.map_shared_rank(slot(2), c));
                        pu[c] = q[tid];
                        px[c] = q[N + tid];
                    }
                }
#pragma unroll
                for (int c = 0; c < kSmMaxC; c++) {
                    if (c < C) {
                        wu = ff_sub(wu, FF{pu[c].x, pu[c].y});
                        wx = ff_sub(wx, FF{px[c].x, px[c].y});
                    }
                }
            }
        }
        if (scr) {
            x_a = FF{0.f, 0.f};
            u_a = FF{0.f, 0.f};
        }
        if (corr) {
            // theta and its sums again, from the corrected parts
            qa = Dot2f();
            qb = Dot2f();
            qr = Dot2f();
            if (tid < N) {
                const FF y = s_y[tid];
                const FF th = ff_sub(wu, y), rx = ff_sub(wx, y);
                s_th[tid] = th;
                sm_acc(qa, th, y);    // theta^T y
                sm_acc(qb, th, th);   // ||theta||^2
                sm_acc(qr, rx, rx);   // ||D xbar_{t-1} - y||^2
            }
            qa = dot2_warp_reduce(qa);
            qb = dot2_warp_reduce(qb);
            qr = dot2_warp_reduce(qr);
            if (lane == 0 && warp < nwr) {
                s_red[warp][0] = qa.s; s_red[warp][1] = qa.c;
                s_red[warp][2] = qb.s; s_red[warp][3] = qb.c;
                s_red[warp][4] = qr.s; s_red[warp][5] = qr.c;
            }
            __syncthreads();
        }
        if (!ovl || corr) {
            bact = __ballot_sync(0xffffffffu, active);
            if (lane == 0) s_wa[warp] = __popc(bact);
            __syncthreads();
            // ---- z_t over this CTA's active atoms, G lanes per atom (G: a power of two up to 32, as many
            // as the atoms leave, the auxiliary warp apart), while the auxiliary warp takes the gap
            int offa = 0, nact = 0;
            for (int w = 0; w < kSmThreads / 32; w++) {
                const int cw = s_wa[w];
                offa += w < warp ? cw : 0;
                nact += cw;
            }
            apos = offa + __popc(bact & ((1u << lane) - 1u));
            if (active) s_al[apos] = a;
            const int nlanes = aux > 0 ? kSmThreads - 32 : kSmThreads;
            int G = 1;
            while (G < 32 && 2 * G * nact <= nlanes) G *= 2;
            __syncthreads();
            if (warp == aux) gap_chain(corr != 0);
            correlate(G, nact);
            __syncthreads();
        }
        // x_t = soft(ubar_{t-1} - z / L, lambda / L) and u_t (Table 1)
        FF xn = x_a, un = u_a, az = FF{0.f, 0.f};
        if (active) {
            const FF z = s_z[apos];
            az = z.h < 0.f ? ff_neg(z) : z;
            xn = it_soft(ff_sub(u_a, ff_mul(z, invL_f)), thrL_f);
            un = fista ? it_momentum(xn, x_a, s_bt) : xn;
        }
        {
            // this CTA's max |z_t| exactly, on float-float pairs (lexicographic on (hi, lo))
            float mh = az.h, ml = az.l;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, mh, o), ol = __shfl_xor_sync(0xffffffffu, ml, o);
                if (oh > mh || (oh == mh && ol > ml)) { mh = oh; ml = ol; }
            }
            if (lane == 0) {
                s_mx[warp] = make_float2(mh, ml);
                s_wc2[warp] = __popc(bact);
            }
            __syncthreads();
            if (warp == 0) {
                float2 v = lane < kSmThreads / 32 ? s_mx[lane] : make_float2(0.f, 0.f);
                int nact = lane < kSmThreads / 32 ? s_wc2[lane] : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float oh = __shfl_xor_sync(0xffffffffu, v.x, o), ol = __shfl_xor_sync(0xffffffffu, v.y, o);
                    if (oh > v.x || (oh == v.x && ol > v.y)) v = make_float2(oh, ol);
                }
                nact = warp_sum(nact);
                if (lane == 0) {
                    s_mloc_h = v.x;
                    s_mloc_l = v.y;
                    stop_t = s_si[2];
                    if (!stop_t) s_cols_corr += nact;  // this CTA's atoms correlated at iteration t
                }
            }
        }
        if (s_si[2]) break;  // the gap of iteration t-1 met the rule (published before the z barrier)
        x_a = xn;
        u_a = un;
    }
    (void)stop_t;

    // ---------------------------------------- xbar of the last completed iteration
    if (own) P.x_out[ai] = active ? ff_to_double(x_a) : 0.0;
    // the result's counts: active atoms and nonzeros of xbar, columns correlated and synthesised, summed
    // over the cluster
    {
        const unsigned ba = __ballot_sync(0xffffffffu, active), bz = __ballot_sync(0xffffffffu, active && x_a.h != 0.f);
        if (lane == 0) {
            s_wc[warp] = __popc(ba);
            s_wc2[warp] = __popc(bz);
        }
        __syncthreads();
        if (tid == 0) {
            int na = 0, nz = 0;
            for (int w = 0; w < kSmThreads / 32; w++) {
                na += s_wc[w];
                nz += s_wc2[w];
            }
            s_iv[0] = na;
            s_iv[1] = nz;
        }
    }
    cl.sync();
    if (rank == 0 && tid == 0) {
        long long na = 0, nz = 0, corr = (long long)K * (need_n ? 2 : 1), synth = 0;
        for (int c = 0; c < C; c++) {
            na += cl.map_shared_rank(s_iv, c)[0];
            nz += cl.map_shared_rank(s_iv, c)[1];
            corr += *cl.map_shared_rank(&s_cols_corr, c);
            synth += *cl.map_shared_rank(&s_cols_synth, c);
        }
        R->iters = t_last - 1;
        R->status = (P.tol > 0.0 && !(s_out_gap <= tol_abs)) ? kDevNotConverged : kDevOk;
        R->n_active = na;
        R->nnz = nz;
        R->gap = s_out_gap;
        R->primal = s_out_primal;
        R->dual = s_out_primal - s_out_gap;
        R->lambda = lam;
        R->lambda_max = lstar;
        R->cols_corr = corr;
        R->cols_synth = synth;
        R->cols_lowp = 0;
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

// ------------------------------------------------------------ host side

// The float-float copy of a small FP64 dictionary: entry (r, i) as hi = RN(d), lo = RN(d - hi).
__global__ void small_split_kernel(const double* D, long long ld, int N, int K, float2* out)
{
    const long long n = (long long)N * K;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const long long i = q / N, r = q - i * N;
        const double d = D[i * ld + r];
        const float h = (float)d;
        out[q] = make_float2(h, (float)(d - (double)h));
    }
}

bool small_dict_eligible(int dtype, int is_group, long long N, long long K)
{
    return dtype == DS_FP64 && !is_group && N >= 1 && N <= kSmMaxN && K >= 1 && K <= (long long)kSmMaxC * kSmThreads;
}

cudaError_t small_dict_split(const double* D, long long ld, int N, int K, float2* out, cudaStream_t s)
{
    const long long n = (long long)N * K;
    const int blocks = (int)std::min<long long>(1024, (n + 255) / 256);
    small_split_kernel<<<blocks, 256, 0, s>>>(D, ld, N, K, out);
    return cudaGetLastError();
}

// the dictionary slice (hi, lo) and the exchange slots (3 x 2 float-float vectors of N)
static size_t small_dyn_smem(int N, int pitch, int C)
{
    (void)C;
    return (size_t)2 * N * pitch * sizeof(float) + (size_t)3 * 2 * N * sizeof(FF);
}

// Cluster size for the one-cluster solve of P, or 0 when P is not a small FP64 Lasso problem it
// handles (ISTA / FISTA with a fixed step, one lambda, no history, at most 256 rows).
int small_cluster_size(const SolveP<double>& P, size_t smem_optin, int* pitch)
{
    if (P.is_group || P.step_mode != 0 || (P.alg != 0 && P.alg != 1) || P.n_lambda != 1 || P.hist ||
        P.colnorm_w || !P.colnorm || !P.Dff || P.abort_flag || P.test < 0 || P.test > 3)
        return 0;
    if (P.N < 1 || P.N > kSmMaxN || P.K < 1) return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, small_kernel) != cudaSuccess) return 0;
    for (int C = 2; C <= kSmMaxC; C *= 2) {
        const int nl = (P.K + C - 1) / C;
        if (nl > kSmThreads) continue;
        const int pt = nl | 1;  // odd pitch: a warp's rows fall in distinct banks
        if (fa.sharedSizeBytes + small_dyn_smem(P.N, pt, C) + 16 * 1024 > smem_optin) continue;
        *pitch = pt;
        return C;
    }
    return 0;
}

cudaError_t launch_small(const SolveP<double>& P, int C, int pitch, size_t smem_optin, cudaStream_t s)
{
    static int dyn_set[64] = {};  // per device: the dynamic shared memory the kernel may use so far
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int dyn = (int)small_dyn_smem(P.N, pitch, C);
    if (dev >= 64 || dyn > dyn_set[dev]) {
        e = cudaFuncSetAttribute(small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        if (dev < 64) dyn_set[dev] = dyn;
    }
    (void)smem_optin;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kSmThreads);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, small_kernel, &cfg);
    if (e != cudaSuccess) return e;
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    return cudaLaunchKernelEx(&cfg, small_kernel, P, pitch);
}

}  // namespace ds
