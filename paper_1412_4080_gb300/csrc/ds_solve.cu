// ds_solve.cu -- persistent cooperative kernel running a whole screened
// ISTA/FISTA solve (Algorithm 3 with the Table 1 updates) on one GB300.
//
// One CTA per SM stays resident for the whole solve.  Every iteration t is
// three grid phases separated by bounded grid barriers:
//
//   (A) scatter + synthesis   compact the active set kept by the previous
//                             test (Algorithm 3, screening of D and X) and
//                             form theta_t = D ubar_{t-1} - y and D xbar_{t-1}
//                             over the nonzeros only (row tiles), with FP64
//                             partials of theta^T y, ||theta||^2 and
//                             ||D xbar - y||^2;
//   (B) correlation + prox    stop test on the gap of iteration t-1, then
//                             z = D_A^T theta_t over the active atoms (the
//                             dominant HBM stream, theta staged in shared
//                             memory, 16-byte vector loads, warp-shuffle dots)
//                             fused with the proximal step (soft threshold,
//                             eq. softTh / group soft threshold, eq. gr_softTh)
//                             and the max |z| (or max ||z_g||/w_g) partials;
//   (C) screening + momentum  dual scaling (Lemma 8), radius of the chosen
//                             test (Lemmas 2-7), the test itself against the
//                             thresholds precomputed from D^T c, the FISTA
//                             extrapolation, and per-CTA nonzero lists.
//
// Reductions are per-CTA partials summed in a fixed order by every CTA, so all
// CTAs take identical decisions and the results do not depend on timing.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "ds_internal.h"

namespace ds {

constexpr int kThreads = 512;
constexpr int kU = 4;         // 16-byte vectors per lane per GEMV item
constexpr int kRowTile = 32;  // rows per synthesis tile

template <typename T>
struct Ws {
    GridBarrier* bar;
    T* theta;
    double* b;
    double* tv;
    double* thr;
    double* nvec;
    int* act[2];
    int* aoff[2];
    // iterates are kept in FP64 whatever the dictionary type: in FP32, u - z/L
    // would quantise z to multiples of L ulp(x), a KKT floor near 1e-6 relative
    double* xc[2];
    double* uc[2];
    double* xn;
    double* un;
    int* keep;
    int* nz_col;
    double* nz_u;
    double* nz_x;
    int* s_alo;
    int* c_kg;
    int* c_ka;
    int* c_nz;
    int* c_nnzx;
    double* p_m;
    double* p_l1;
    double* p_a;
    double* p_b;
    double* p_r;
    double* p_v;
    int* p_i;
};

template <typename T>
struct SolveP {
    const T* D;
    int N, K, ld, nG, is_group;
    const int* goff;
    const double* w;
    const double* spec;
    const double* colnorm;
    double fmax, gamma, eps_test;
    const T* y;
    const T* x0;
    int n_lambda;
    const double* lambdas;  // device copy
    int lambda_rel;
    int alg, test, dynamic, max_iter;
    double tol, L;
    T* x_out;
    long long ldx;
    DevResult* res;
    double* hist;
    int hist_rows;
    Ws<T> ws;
    int RA, nchunk, npad;
};

// ------------------------------------------------------------------ helpers

template <typename T> __device__ __forceinline__ T soft_thr(T v, T t)
{
    T a = fabs(v) - t;
    return a > T(0) ? (v > T(0) ? a : -a) : T(0);
}

__device__ __forceinline__ double dual_scale(double alpha, double beta, double lam, double m)
{
    // Lemma 8: [theta^T y / (lambda ||theta||^2)] projected on [-1/m, 1/m]
    if (!(beta > 0.0)) return 0.0;
    double s = alpha / (lam * beta);
    if (m > 0.0) {
        double lim = 1.0 / m;
        s = fmin(fmax(s, -lim), lim);
    }
    return s;
}

// Maximum of d^T theta over {||theta - c0|| <= R} cap {n^T theta <= off} for unit d,
// unit n, t = n^T d, dc0 = d^T c0 and psi = n^T c0 - off >= 0 (dynamic form of Lemma 4).
__device__ __forceinline__ double dome_max(double dc0, double t, double psi, double R)
{
    if (t * R <= -psi) return dc0 + R;
    double rho2 = fmax(R * R - psi * psi, 0.0);
    double s2 = fmax(1.0 - t * t, 0.0);
    return dc0 - psi * t + sqrt(rho2) * sqrt(s2);
}

// synthesis term d * c with an FP64 coefficient c: for FP32 dictionaries c is split
// into hi + lo floats and d * hi is accumulated with error-free transformations
__device__ __forceinline__ void syn_add(Dot2f& acc, float d, double c)
{
    const float hi = (float)c;
    const float lo = (float)(c - (double)hi);
    acc.add(d, hi);
    acc.c = fmaf(d, lo, acc.c);
}
__device__ __forceinline__ void syn_add(Dot2d& acc, double d, double c) { acc.add(d, c); }

__device__ __forceinline__ float4 v4zero(float4*) { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ double2 v4zero(double2*) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float vdot(float4 a, float4 b, float s)
{
    s = fmaf(a.x, b.x, s);
    s = fmaf(a.y, b.y, s);
    s = fmaf(a.z, b.z, s);
    s = fmaf(a.w, b.w, s);
    return s;
}
__device__ __forceinline__ double vdot(double2 a, double2 b, double s)
{
    s = fma(a.x, b.x, s);
    s = fma(a.y, b.y, s);
    return s;
}
__device__ __forceinline__ void vdot2(float4 a, float hi0, float hi1, float hi2, float hi3, Dot2f& acc)
{
    acc.add(a.x, hi0);
    acc.add(a.y, hi1);
    acc.add(a.z, hi2);
    acc.add(a.w, hi3);
}

// Column slice [p_lo, p_hi) of the active list owned by CTA b, balanced in atoms
// and cut at group boundaries.  Returns the atom offset of p_lo.
template <typename T>
__device__ __forceinline__ void cta_slice(const SolveP<T>& P, const int* aoff, int nA_g, int nA_a, int b, int G,
                                          int* p_lo, int* p_hi, int* a_lo)
{
    __shared__ int s_slice[3];
    if (threadIdx.x == 0) {
        if (!P.is_group) {
            s_slice[0] = (int)((long long)b * nA_g / G);
            s_slice[1] = (int)((long long)(b + 1) * nA_g / G);
            s_slice[2] = s_slice[0];
        } else {
            int bounds[2];
            for (int k = 0; k < 2; k++) {
                long long target = (long long)(b + k) * nA_a / G;
                int lo = 0, hi = nA_g;  // first p with aoff[p] >= target
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (__ldcg(aoff + mid) < target) lo = mid + 1;
                    else hi = mid;
                }
                bounds[k] = lo;
            }
            s_slice[0] = bounds[0];
            s_slice[1] = bounds[1];
            s_slice[2] = bounds[0] < nA_g ? __ldcg(aoff + bounds[0]) : nA_a;
        }
    }
    __syncthreads();
    *p_lo = s_slice[0];
    *p_hi = s_slice[1];
    *a_lo = s_slice[2];
    __syncthreads();
}

// --------------------------------------------------------------- the kernel

template <typename T>
__device__ __forceinline__ bool solve_body(const SolveP<T>& P)
{
    using V = typename Vec4<T>::type;
    constexpr int EV = 16 / sizeof(T);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* th_s = reinterpret_cast<T*>(smem_raw);
    T* zpart = th_s + P.npad;
    int* cols_s = reinterpret_cast<int*>(zpart + (size_t)P.RA * P.nchunk);

    __shared__ int s_tmp[32];
    __shared__ double s_dred[32];
    __shared__ int s_ired[32];
    __shared__ int s_pref[1025];
    __shared__ double s_red[2][kThreads / 32][kRowTile];
    __shared__ double s_sc[16];
    __shared__ int s_si[8];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kThreads / 32;
    const int b = blockIdx.x, G = gridDim.x;
    const Ws<T>& W = P.ws;
    unsigned int gen = 0;
    if (tid == 0) gen = ld_volatile_u32(&W.bar->gen);
    // gen is only meaningful in thread 0, which is the only thread that reads it

    const int N = P.N, K = P.K, ld = P.ld, nG = P.nG;
    const int ldv = ld / EV;
    const int total_warps = G * nw;
    const int gwarp = b * nw + warp;
    bool ok = true;

    // ---------------------------------------------------- P0a: b = D^T y, ||y||^2
    for (int r = tid; r < P.npad; r += kThreads) th_s[r] = r < N ? P.y[r] : T(0);
    __syncthreads();
    {
        const V* yv = reinterpret_cast<const V*>(th_s);
        for (int i = gwarp; i < K; i += total_warps) {
            const V* col = reinterpret_cast<const V*>(P.D + (size_t)i * ld);
            typename Dot2<T>::type acc;
            for (int v = lane; v < ldv; v += 32) {
                V d = __ldg(col + v);
                V q = yv[v];
                if constexpr (EV == 4) {
                    acc.add(d.x, q.x); acc.add(d.y, q.y); acc.add(d.z, q.z); acc.add(d.w, q.w);
                } else {
                    acc.add(d.x, q.x); acc.add(d.y, q.y);
                }
            }
            double s = warp_sum(acc.value());
            if (lane == 0) W.b[i] = s;
        }
        double yy = 0.0;
        for (int r = b * kThreads + tid; r < N; r += G * kThreads) {
            double v = (double)P.y[r];
            yy += v * v;
        }
        yy = warp_sum(yy);
        if (lane == 0) s_dred[warp] = yy;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int k = 0; k < nw; k++) s += s_dred[k];
            W.p_a[b] = s;
        }
    }
    ok = grid_sync(W.bar, G, gen);
    if (!ok) return false;

    // --------------------------------- P0b: lambda_* (Sec. 2.2.2 / eq. gstar)
    {
        double best = -1.0;
        int arg = 0x7fffffff;
        for (int g = b * kThreads + tid; g < nG; g += G * kThreads) {
            double s;
            if (!P.is_group) {
                s = fabs(__ldcg(W.b + g));
            } else {
                double q = 0.0;
                for (int i = P.goff[g]; i < P.goff[g + 1]; i++) {
                    double v = __ldcg(W.b + i);
                    q += v * v;
                }
                s = sqrt(q) / P.w[g];
            }
            if (s > best || (s == best && g < arg)) { best = s; arg = g; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oa = __shfl_xor_sync(0xffffffffu, arg, o);
            if (ob > best || (ob == best && oa < arg)) { best = ob; arg = oa; }
        }
        if (lane == 0) { s_dred[warp] = best; s_ired[warp] = arg; }
        __syncthreads();
        if (tid == 0) {
            double bb = -1.0;
            int ba = 0x7fffffff;
            for (int k = 0; k < nw; k++)
                if (s_dred[k] > bb || (s_dred[k] == bb && s_ired[k] < ba)) { bb = s_dred[k]; ba = s_ired[k]; }
            W.p_v[b] = bb;
            W.p_i[b] = ba;
        }
    }
    ok = grid_sync(W.bar, G, gen);
    if (!ok) return false;

    {
        // every CTA reduces the same partials in the same order
        if (warp == 0) {
            double bb = -1.0;
            int ba = 0x7fffffff;
            for (int k = lane; k < G; k += 32) {
                double v = __ldcg(W.p_v + k);
                int a = __ldcg(W.p_i + k);
                if (v > bb || (v == bb && a < ba)) { bb = v; ba = a; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double ob = __shfl_xor_sync(0xffffffffu, bb, o);
                int oa = __shfl_xor_sync(0xffffffffu, ba, o);
                if (ob > bb || (ob == bb && oa < ba)) { bb = ob; ba = oa; }
            }
            double yy = warp_sum_fixed(W.p_a, G, lane);
            if (lane == 0) { s_sc[0] = bb; s_si[0] = ba; s_sc[1] = yy; }
        }
        __syncthreads();
    }
    const double lstar = s_sc[0];
    const int star = s_si[0];
    const double yy = s_sc[1];
    if (P.n_lambda == 0) {  // lambda_max query only
        if (b == 0 && tid == 0) { P.res[0].lambda_max = lstar; P.res[0].status = kDevOk; }
        return true;
    }

    const bool need_n = P.test == 2 || P.test == 3 || P.test == 5;  // DST3, DOME, DGST3
    double nn = 0.0, nty = 0.0, wstar2 = 1.0;
    if (need_n && lstar > 0.0) {
        // ---------------- n = D_{g*} D_{g*}^T y / lambda_*  (Lemma 6; Lasso: n = d_*)
        const int c0 = P.is_group ? P.goff[star] : star;
        const int c1 = P.is_group ? P.goff[star + 1] : star + 1;
        double nq = 0.0;
        for (int r = b * kThreads + tid; r < N; r += G * kThreads) {
            double s = 0.0;
            for (int i = c0; i < c1; i++) s += (double)P.D[(size_t)i * ld + r] * (__ldcg(W.b + i) / lstar);
            W.nvec[r] = s;
            nq += s * s;
        }
        nq = warp_sum(nq);
        __syncthreads();
        if (lane == 0) s_dred[warp] = nq;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int k = 0; k < nw; k++) s += s_dred[k];
            W.p_r[b] = s;
        }
        ok = grid_sync(W.bar, G, gen);
        if (!ok) return false;
        if (warp == 0) {
            double s = warp_sum_fixed(W.p_r, G, lane);
            if (lane == 0) s_sc[2] = s;
        }
        // stage n in shared memory (hi/lo split for FP32 dictionaries)
        if constexpr (EV == 4) {
            float* nh = reinterpret_cast<float*>(smem_raw);
            float* nl = nh + P.npad;
            for (int r = tid; r < P.npad; r += kThreads) {
                double v = r < N ? __ldcg(W.nvec + r) : 0.0;
                float h = (float)v;
                nh[r] = h;
                nl[r] = (float)(v - (double)h);
            }
        } else {
            for (int r = tid; r < P.npad; r += kThreads) th_s[r] = r < N ? (T)__ldcg(W.nvec + r) : T(0);
        }
        __syncthreads();
        nn = s_sc[2];
        {
            double q = 0.0;
            for (int i = c0; i < c1; i++) {
                double v = __ldcg(W.b + i);
                q += v * v;
            }
            nty = q / lstar;  // n^T y = ||D_{g*}^T y||^2 / lambda_*
        }
        if (P.is_group) wstar2 = P.w[star] * P.w[star];
        // ---------------- tv = D^T n (compensated)
        for (int i = gwarp; i < K; i += total_warps) {
            const V* col = reinterpret_cast<const V*>(P.D + (size_t)i * ld);
            double s;
            if constexpr (EV == 4) {
                const float4* nh4 = reinterpret_cast<const float4*>(smem_raw);
                const float4* nl4 = nh4 + P.npad / 4;
                Dot2f acc;
                float lo = 0.f;
                for (int v = lane; v < ldv; v += 32) {
                    float4 d = __ldg(reinterpret_cast<const float4*>(col) + v);
                    float4 h = nh4[v], l = nl4[v];
                    vdot2(d, h.x, h.y, h.z, h.w, acc);
                    lo = fmaf(d.x, l.x, lo); lo = fmaf(d.y, l.y, lo); lo = fmaf(d.z, l.z, lo); lo = fmaf(d.w, l.w, lo);
                }
                s = warp_sum(acc.value() + (double)lo);
            } else {
                const V* nv = reinterpret_cast<const V*>(th_s);
                Dot2d acc;
                for (int v = lane; v < ldv; v += 32) {
                    V d = __ldg(col + v);
                    V q = nv[v];
                    acc.add(d.x, q.x);
                    acc.add(d.y, q.y);
                }
                s = warp_sum(acc.value());
            }
            if (lane == 0) W.tv[i] = s;
        }
        ok = grid_sync(W.bar, G, gen);
        if (!ok) return false;
    }

    // ================================================================ lambdas
    for (int j = 0; j < P.n_lambda; j++) {
        const double lam = P.lambda_rel ? P.lambdas[j] * lstar : P.lambdas[j];
        T* xout = P.x_out + (size_t)j * P.ldx;
        DevResult* R = P.res + j;
        if (!(lam < lstar)) {
            // x = 0 and theta = y / lambda is dual optimal (Sec. 2.2.2)
            for (int i = b * kThreads + tid; i < K; i += G * kThreads) xout[i] = T(0);
            if (b == 0 && tid == 0) {
                R->iters = 0; R->status = kDevOk; R->n_active = 0; R->nnz = 0;
                R->gap = 0.0; R->primal = 0.5 * yy; R->dual = 0.5 * yy; R->lambda = lam; R->lambda_max = lstar;
            }
            continue;
        }
        const bool record = (j == 0) && P.hist != nullptr;
        const double psi = lstar / lam - 1.0;
        // DST3 / DGST3 centre c = y/lam - coef n, offset delta = ||y/lam - c|| (Lemmas 3, 6)
        const double coef = need_n && nn > 0.0 ? (nty / lam - wstar2) / nn : 0.0;
        const double delta = need_n && nn > 0.0 ? fabs(nty / lam - wstar2) / sqrt(nn) : 0.0;
        const double nstar = P.is_group ? 1.0 : P.colnorm[star];
        const double psi_dome = psi / nstar;
        const double invL = 1.0 / P.L;
        const double thrL = lam / P.L;
        const bool ista = P.alg == 0;
        const bool dyn_test = P.dynamic && P.test != 0;

        // ------------------------------------------------ (C0) initial state
        int cur = 0;
        {
            int p_lo = (int)((long long)b * nG / G), p_hi = (int)((long long)(b + 1) * nG / G);
            if (P.is_group) {
                // cut at group boundaries, balanced in atoms
                int bounds[2];
                for (int k = 0; k < 2; k++) {
                    long long target = (long long)(b + k) * K / G;
                    int lo = 0, hi = nG;
                    while (lo < hi) {
                        int mid = (lo + hi) >> 1;
                        if (P.goff[mid] < target) lo = mid + 1;
                        else hi = mid;
                    }
                    bounds[k] = lo;
                }
                p_lo = bounds[0];
                p_hi = bounds[1];
            }
            const int a_lo = P.is_group ? (p_lo < nG ? P.goff[p_lo] : K) : p_lo;
            // static screening (Algorithm 1): the test at theta = -y, m = lambda_*
            double rad0 = 0.0;
            const bool stat = !P.dynamic && P.test != 0;
            if (stat) {
                double mup = lstar * (1.0 + 1e-12);
                double mu = dual_scale(-yy, yy, lam, mup);
                double R2 = yy / (lam * lam) + 2.0 * mu * yy / lam + mu * mu * yy;
                R2 = fmax(R2, 0.0);
                rad0 = (P.test == 2 || P.test == 5) ? sqrt(fmax(R2 - delta * delta, 0.0)) : sqrt(R2);
            }
            int nz_base = 0, kg = 0, ka = 0;
            for (int base = p_lo; base < p_hi; base += kThreads) {
                int p = base + tid;
                bool valid = p < p_hi;
                int kept = 0, cnt = 0;
                int lo_a = 0, hi_a = 0;
                if (valid) {
                    lo_a = P.is_group ? P.goff[p] : p;
                    hi_a = P.is_group ? P.goff[p + 1] : p + 1;
                    W.act[cur][p] = p;
                    if (P.is_group) W.aoff[cur][p] = lo_a;
                    // threshold of the sphere tests: (w_g - ||(D^T c)_g||) / ||D_g||  (Lemma 7)
                    double th = 0.0;
                    if (P.test == 1 || P.test == 2 || P.test == 4 || P.test == 5) {
                        double q = 0.0;
                        for (int i = lo_a; i < hi_a; i++) {
                            double dtc = __ldcg(W.b + i) / lam - ((P.test == 2 || P.test == 5) ? coef * __ldcg(W.tv + i) : 0.0);
                            q += dtc * dtc;
                        }
                        double wg = P.is_group ? P.w[p] : 1.0;
                        double sg = P.is_group ? P.spec[p] : P.colnorm[p];
                        th = (wg - sqrt(q)) / sg;
                        W.thr[p] = th;
                    }
                    bool kill = false;
                    if (stat) {
                        if (P.test == 3) {
                            double ni = P.colnorm[p];
                            double dc0 = __ldcg(W.b + p) / (lam * ni);
                            double tt = __ldcg(W.tv + p) / (ni * nstar);
                            double up = dome_max(dc0, tt, psi_dome, rad0);
                            double dn = dome_max(-dc0, -tt, psi_dome, rad0);
                            kill = (1.0 / ni - up > P.eps_test) && (1.0 / ni - dn > P.eps_test);
                        } else {
                            kill = th - rad0 > P.eps_test;
                        }
                    }
                    kept = !kill;
                    W.keep[p] = kept;
                    for (int i = lo_a; i < hi_a; i++) {
                        double xv = P.x0 ? (double)P.x0[i] : 0.0;
                        if (!kept) xv = 0.0;
                        W.xn[i] = xv;
                        W.un[i] = xv;
                        cnt += xv != 0.0;
                    }
                    kg += kept;
                    ka += kept ? hi_a - lo_a : 0;
                }
                int tot;
                int pos = block_exclusive_scan(cnt, s_tmp, &tot);
                if (valid && cnt) {
                    int e = a_lo + nz_base + pos;
                    for (int i = lo_a; i < hi_a; i++) {
                        double xv = W.xn[i];
                        if (xv != 0.0) {
                            W.nz_col[e] = i;
                            W.nz_u[e] = xv;
                            W.nz_x[e] = xv;
                            e++;
                        }
                    }
                }
                nz_base += tot;
            }
            int tkg, tka, dummy;
            block_exclusive_scan(kg, s_tmp, &tkg);
            block_exclusive_scan(ka, s_tmp, &tka);
            (void)dummy;
            if (tid == 0) {
                W.s_alo[b] = a_lo;
                W.c_kg[b] = tkg;
                W.c_ka[b] = tka;
                W.c_nz[b] = nz_base;
                W.c_nnzx[b] = nz_base;
                W.p_l1[b] = 0.0;
            }
            if (b == G - 1 && tid == 0 && P.is_group) W.aoff[cur][nG] = K;
        }
        ok = grid_sync(W.bar, G, gen);
        if (!ok) return false;

        int nA_g = nG, nA_a = K;  // sizes of the list `cur` refers to
        double alpha = 0.0, beta = 0.0, mu_nom = 0.0, R_nom = 0.0, rad = 0.0, lf = 1.0;
        double gap = INFINITY, primal = 0.0;
        int t = 1;
        int iters = 0;
        long long nnz_last = 0;
        // work counters (dictionary columns read), the precompute passes charged to the first lambda
        long long cols_corr = j == 0 ? (long long)K * (need_n ? 2 : 1) : 0, cols_synth = 0;
        for (;; t++) {
            // ======================================== (A) scatter + synthesis
            {
                int p_lo, p_hi, a_lo;
                cta_slice(P, P.is_group ? W.aoff[cur] : nullptr, nA_g, nA_a, b, G, &p_lo, &p_hi, &a_lo);
                const int nxt = cur ^ 1;
                if (warp == 0) {
                    long long g0 = 0, a0 = 0;
                    for (int k = lane; k < b; k += 32) { g0 += __ldcg(W.c_kg + k); a0 += __ldcg(W.c_ka + k); }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        g0 += __shfl_xor_sync(0xffffffffu, g0, o);
                        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                    }
                    if (lane == 0) { s_si[1] = (int)g0; s_si[2] = (int)a0; }
                }
                __syncthreads();
                int gb = s_si[1], ab = s_si[2];
                for (int base = p_lo; base < p_hi; base += kThreads) {
                    int p = base + tid;
                    bool valid = p < p_hi;
                    int k = valid ? __ldcg(W.keep + p) : 0;
                    int lo_a = 0, sz = 0;
                    if (valid) {
                        lo_a = P.is_group ? __ldcg(W.aoff[cur] + p) : p;
                        sz = P.is_group ? (p + 1 < nA_g ? __ldcg(W.aoff[cur] + p + 1) : nA_a) - lo_a : 1;
                    }
                    int tg, ta;
                    int pg = block_exclusive_scan(k, s_tmp, &tg);
                    int pa = block_exclusive_scan(k ? sz : 0, s_tmp, &ta);
                    if (k) {
                        int ng = gb + pg, na = ab + pa;
                        W.act[nxt][ng] = __ldcg(W.act[cur] + p);
                        if (P.is_group) W.aoff[nxt][ng] = na;
                        for (int q = 0; q < sz; q++) {
                            W.xc[nxt][na + q] = __ldcg(W.xn + lo_a + q);
                            W.uc[nxt][na + q] = __ldcg(W.un + lo_a + q);
                        }
                    }
                    gb += tg;
                    ab += ta;
                }
                if (b == G - 1 && tid == 0 && P.is_group) W.aoff[nxt][gb] = ab;

                // synthesis over row tiles: w_u = D ubar, w_x = D xbar, from the nonzero lists
                if (tid < G) s_pref[tid + 1] = __ldcg(W.c_nz + tid);
                if (tid == 0) s_pref[0] = 0;
                __syncthreads();
                if (tid == 0)
                    for (int k = 1; k <= G; k++) s_pref[k] += s_pref[k - 1];
                __syncthreads();
                const int E = s_pref[G];
                cols_synth += E;
                double pa_ = 0.0, pb_ = 0.0, pr_ = 0.0;
                const int ntiles = (N + kRowTile - 1) / kRowTile;
                for (int tile = b; tile < ntiles; tile += G) {
                    const int r = tile * kRowTile + lane;
                    const bool rv = r < N;
                    // compensated accumulation: theta = D u - y is a small difference of two
                    // large vectors, so the sum is carried to twice the working precision
                    typename Dot2<T>::type au, ax;
                    for (int e0 = warp; e0 < E; e0 += nw * 4) {
                        int cols[4];
                        double uv[4], xv[4];
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            int e = e0 + q * nw;
                            cols[q] = -1;
                            uv[q] = 0.0;
                            xv[q] = 0.0;
                            if (e < E) {
                                int lo = 0, hi = G;  // largest k with s_pref[k] <= e
                                while (hi - lo > 1) {
                                    int mid = (lo + hi) >> 1;
                                    if (s_pref[mid] <= e) lo = mid;
                                    else hi = mid;
                                }
                                int idx = __ldcg(W.s_alo + lo) + (e - s_pref[lo]);
                                cols[q] = __ldcg(W.nz_col + idx);
                                uv[q] = __ldcg(W.nz_u + idx);
                                xv[q] = __ldcg(W.nz_x + idx);
                            }
                        }
                        T dv[4];
#pragma unroll
                        for (int q = 0; q < 4; q++) dv[q] = (cols[q] >= 0 && rv) ? __ldg(P.D + (size_t)cols[q] * ld + r) : T(0);
#pragma unroll
                        for (int q = 0; q < 4; q++) {
                            syn_add(au, dv[q], uv[q]);
                            syn_add(ax, dv[q], xv[q]);
                        }
                    }
                    s_red[0][warp][lane] = au.value();
                    s_red[1][warp][lane] = ax.value();
                    __syncthreads();
                    if (warp == 0) {
                        double wu = 0.0, wx = 0.0;
                        for (int k = 0; k < nw; k++) { wu += s_red[0][k][lane]; wx += s_red[1][k][lane]; }
                        if (rv) {
                            const double yv = (double)P.y[r];
                            const T th = (T)(wu - yv);
                            W.theta[r] = th;
                            pa_ += (double)th * yv;
                            pb_ += (double)th * (double)th;
                            const double rx = wx - yv;
                            pr_ += rx * rx;
                        }
                    }
                    __syncthreads();
                }
                if (warp == 0) {
                    pa_ = warp_sum(pa_);
                    pb_ = warp_sum(pb_);
                    pr_ = warp_sum(pr_);
                    if (lane == 0) { W.p_a[b] = pa_; W.p_b[b] = pb_; W.p_r[b] = pr_; }
                }
                cur = nxt;
            }
            ok = grid_sync(W.bar, G, gen);
            if (!ok) return false;

            // ================================ (B) stop test, correlation + prox
            {
                if (warp == 0) {
                    double a_ = warp_sum_fixed(W.p_a, G, lane);
                    double b_ = warp_sum_fixed(W.p_b, G, lane);
                    double r_ = warp_sum_fixed(W.p_r, G, lane);
                    double l1 = warp_sum_fixed(W.p_l1, G, lane);
                    long long ng = warp_sum_fixed(W.c_kg, G, lane);
                    long long na = warp_sum_fixed(W.c_ka, G, lane);
                    long long nx = warp_sum_fixed(W.c_nnzx, G, lane);
                    if (lane == 0) {
                        s_sc[3] = a_; s_sc[4] = b_; s_sc[5] = r_; s_sc[6] = l1;
                        s_si[3] = (int)ng; s_si[4] = (int)na; s_si[5] = (int)nx;
                    }
                }
                __syncthreads();
                const double rho = s_sc[5], l1 = s_sc[6];
                nA_g = s_si[3];
                nA_a = s_si[4];
                nnz_last = s_si[5];
                bool stop = false;
                if (t > 1) {
                    // gap of iteration t-1: P(xbar) - Dual(mu theta), Dual(v) = 1/2||y||^2 - lambda^2/2 ||v - y/lambda||^2
                    primal = 0.5 * rho + lam * l1;
                    gap = primal - 0.5 * yy + 0.5 * lam * lam * R_nom * R_nom;
                    iters = t - 1;
                    if (record && b == 0 && tid == 0 && t - 1 <= P.hist_rows) {
                        double* h = P.hist + (size_t)(t - 2) * 6;
                        h[0] = (double)nA_a; h[1] = (double)nnz_last; h[2] = R_nom; h[3] = rad; h[4] = gap; h[5] = mu_nom;
                    }
                    stop = (P.tol > 0.0 && gap <= P.tol * 0.5 * yy) || (t - 1 >= P.max_iter);
                }
                alpha = s_sc[3];
                beta = s_sc[4];
                if (stop) break;
                cols_corr += nA_a;

                // stage theta_t
                for (int r = tid; r < P.npad; r += kThreads) th_s[r] = r < N ? __ldcg(W.theta + r) : T(0);
                int p_lo, p_hi, a_lo;
                cta_slice(P, P.is_group ? W.aoff[cur] : nullptr, nA_g, nA_a, b, G, &p_lo, &p_hi, &a_lo);
                double mloc = 0.0;
                const V* thv = reinterpret_cast<const V*>(th_s);
                int p = p_lo;
                while (p < p_hi) {
                    // gather a round of whole groups, at most RA atoms
                    int p_end = p, natoms = 0;
                    if (!P.is_group) {
                        p_end = min(p_hi, p + P.RA);
                        natoms = p_end - p;
                    } else {
                        while (p_end < p_hi) {
                            int g = __ldcg(W.act[cur] + p_end);
                            int sz = P.goff[g + 1] - P.goff[g];
                            if (natoms + sz > P.RA) break;
                            natoms += sz;
                            p_end++;
                        }
                    }
                    const int abase = P.is_group ? __ldcg(W.aoff[cur] + p) : p;
                    if (!P.is_group) {
                        for (int a = tid; a < natoms; a += kThreads) cols_s[a] = __ldcg(W.act[cur] + p + a);
                    } else {
                        for (int q = p + tid; q < p_end; q += kThreads) {
                            int g = __ldcg(W.act[cur] + q);
                            int off = __ldcg(W.aoff[cur] + q) - abase;
                            for (int i = P.goff[g]; i < P.goff[g + 1]; i++) cols_s[off + i - P.goff[g]] = i;
                        }
                    }
                    __syncthreads();
                    // z = D_A^T theta: items (atom, row chunk), two per warp in flight
                    const int nchunk = P.nchunk;
                    const int nitems = natoms * nchunk;
                    for (int j0 = warp * 2; j0 < nitems; j0 += nw * 2) {
                        const int j1 = j0 + 1;
                        const bool h1 = j1 < nitems;
                        const int a0 = j0 / nchunk, c0 = j0 - a0 * nchunk;
                        const int a1 = h1 ? j1 / nchunk : a0, c1 = h1 ? j1 - a1 * nchunk : c0;
                        const V* col0 = reinterpret_cast<const V*>(P.D + (size_t)cols_s[a0] * ld);
                        const V* col1 = reinterpret_cast<const V*>(P.D + (size_t)cols_s[a1] * ld);
                        V d0[kU], d1[kU];
#pragma unroll
                        for (int k = 0; k < kU; k++) {
                            const int v0 = c0 * (32 * kU) + k * 32 + lane;
                            const int v1 = c1 * (32 * kU) + k * 32 + lane;
                            d0[k] = v0 < ldv ? __ldg(col0 + v0) : v4zero((V*)nullptr);
                            d1[k] = (h1 && v1 < ldv) ? __ldg(col1 + v1) : v4zero((V*)nullptr);
                        }
                        T s0 = T(0), s1 = T(0);
#pragma unroll
                        for (int k = 0; k < kU; k++) {
                            s0 = vdot(d0[k], thv[c0 * (32 * kU) + k * 32 + lane], s0);
                            s1 = vdot(d1[k], thv[c1 * (32 * kU) + k * 32 + lane], s1);
                        }
                        s0 = warp_sum(s0);
                        s1 = warp_sum(s1);
                        if (lane == 0) {
                            zpart[a0 * nchunk + c0] = s0;
                            if (h1) zpart[a1 * nchunk + c1] = s1;
                        }
                    }
                    __syncthreads();
                    // proximal step (Table 1): x = prox_{lambda/L Omega}(u - z / L)
                    for (int a = tid; a < natoms; a += kThreads) {
                        T z = T(0);
                        for (int c = 0; c < nchunk; c++) z += zpart[a * nchunk + c];
                        if (!P.is_group) {
                            const int ap = abase + a;
                            double v = __ldcg(W.uc[cur] + ap) - (double)z * invL;
                            W.xn[ap] = soft_thr(v, thrL);
                            mloc = fmax(mloc, (double)fabs(z));
                        } else {
                            zpart[a * nchunk] = z;
                        }
                    }
                    if (P.is_group) {
                        __syncthreads();
                        for (int q = p + tid; q < p_end; q += kThreads) {
                            int g = __ldcg(W.act[cur] + q);
                            int off = __ldcg(W.aoff[cur] + q);
                            int sz = P.goff[g + 1] - P.goff[g];
                            double zq = 0.0, vq = 0.0;
                            for (int i = 0; i < sz; i++) {
                                T z = zpart[(off - abase + i) * nchunk];
                                double v = __ldcg(W.uc[cur] + off + i) - (double)z * invL;
                                zq += (double)z * (double)z;
                                vq += v * v;
                            }
                            const double wg = P.w[g];
                            const double nv = sqrt(vq);
                            // group soft threshold: max(0, (||v_g|| - t w_g) / ||v_g||) v_g
                            const double f = nv > 0.0 ? fmax(0.0, (nv - thrL * wg) / nv) : 0.0;
                            for (int i = 0; i < sz; i++) {
                                T z = zpart[(off - abase + i) * nchunk];
                                double v = __ldcg(W.uc[cur] + off + i) - (double)z * invL;
                                W.xn[off + i] = f * v;
                            }
                            mloc = fmax(mloc, sqrt(zq) / wg);
                        }
                    }
                    __syncthreads();
                    p = p_end;
                }
                mloc = warp_max(mloc);
                if (lane == 0) s_dred[warp] = mloc;
                __syncthreads();
                if (tid == 0) {
                    double m = 0.0;
                    for (int k = 0; k < nw; k++) m = fmax(m, s_dred[k]);
                    W.p_m[b] = m;
                }
            }
            ok = grid_sync(W.bar, G, gen);
            if (!ok) return false;

            // ===================================== (C) screening + momentum
            {
                if (warp == 0) {
                    double m = warp_max_fixed(W.p_m, G, lane);
                    if (lane == 0) s_sc[7] = m;
                }
                __syncthreads();
                const double m_nom = s_sc[7];
                // rigorous upper bound on max |d_i^T theta| given the FP rounding of z
                const double m_up = m_nom + P.gamma * sqrt(beta) * P.fmax;
                mu_nom = dual_scale(alpha, beta, lam, m_nom);
                const double mu_s = dual_scale(alpha, beta, lam, m_up);
                const double R2n = fmax(yy / (lam * lam) - 2.0 * mu_nom * alpha / lam + mu_nom * mu_nom * beta, 0.0);
                const double R2s = fmax(yy / (lam * lam) - 2.0 * mu_s * alpha / lam + mu_s * mu_s * beta, 0.0);
                R_nom = sqrt(R2n);
                const double Rs = sqrt(R2s);
                rad = (P.test == 2 || P.test == 5) ? sqrt(fmax(R2s - delta * delta, 0.0)) : Rs;
                // FISTA: l_t = (1 + sqrt(1 + 4 l_{t-1}^2)) / 2, coefficient (l_{t-1} - 1) / l_t
                double bt = 0.0;
                if (!ista) {
                    double ln = 0.5 * (1.0 + sqrt(1.0 + 4.0 * lf * lf));
                    bt = (lf - 1.0) / ln;
                    lf = ln;
                }
                int p_lo, p_hi, a_lo;
                cta_slice(P, P.is_group ? W.aoff[cur] : nullptr, nA_g, nA_a, b, G, &p_lo, &p_hi, &a_lo);
                int nz_base = 0, kg = 0, ka = 0, nzx = 0;
                double l1 = 0.0;
                for (int base = p_lo; base < p_hi; base += kThreads) {
                    int p = base + tid;
                    bool valid = p < p_hi;
                    int kept = 0, cnt = 0, lo_a = 0, sz = 0, gid = 0;
                    if (valid) {
                        gid = __ldcg(W.act[cur] + p);
                        lo_a = P.is_group ? __ldcg(W.aoff[cur] + p) : p;
                        sz = P.is_group ? (p + 1 < nA_g ? __ldcg(W.aoff[cur] + p + 1) : nA_a) - lo_a : 1;
                        bool kill = false;
                        if (dyn_test) {
                            if (P.test == 3) {
                                // Lemma 4 (dynamic dome): max over the dome of |d_i^T theta| < 1
                                double ni = P.colnorm[gid];
                                double dc0 = __ldcg(W.b + gid) / (lam * ni);
                                double tt = __ldcg(W.tv + gid) / (ni * nstar);
                                double up = dome_max(dc0, tt, psi_dome, Rs);
                                double dn = dome_max(-dc0, -tt, psi_dome, Rs);
                                kill = (1.0 / ni - up > P.eps_test) && (1.0 / ni - dn > P.eps_test);
                            } else {
                                kill = __ldcg(W.thr + gid) - rad > P.eps_test;
                            }
                        }
                        kept = !kill;
                        W.keep[p] = kept;
                        if (kept) {
                            double gq = 0.0;
                            for (int q = 0; q < sz; q++) {
                                double xv = __ldcg(W.xn + lo_a + q);
                                double xo = __ldcg(W.xc[cur] + lo_a + q);
                                double uv = ista ? xv : xv + bt * (xv - xo);
                                W.un[lo_a + q] = uv;
                                cnt += (uv != 0.0 || xv != 0.0);
                                nzx += xv != 0.0;
                                gq += xv * xv;
                            }
                            l1 += (P.is_group ? P.w[gid] : 1.0) * sqrt(gq);
                            kg += 1;
                            ka += sz;
                        }
                    }
                    int tot;
                    int pos = block_exclusive_scan(cnt, s_tmp, &tot);
                    if (cnt) {
                        int e = a_lo + nz_base + pos;
                        for (int q = 0; q < sz; q++) {
                            double xv = __ldcg(W.xn + lo_a + q);
                            double uv = __ldcg(W.un + lo_a + q);
                            if (uv != 0.0 || xv != 0.0) {
                                const int col = P.is_group ? P.goff[gid] + q : gid;
                                W.nz_col[e] = col;
                                W.nz_u[e] = uv;
                                W.nz_x[e] = xv;
                                e++;
                            }
                        }
                    }
                    nz_base += tot;
                }
                int tkg, tka, tnx;
                block_exclusive_scan(kg, s_tmp, &tkg);
                block_exclusive_scan(ka, s_tmp, &tka);
                block_exclusive_scan(nzx, s_tmp, &tnx);
                l1 = warp_sum(l1);
                if (lane == 0) s_dred[warp] = l1;
                __syncthreads();
                if (tid == 0) {
                    double s = 0.0;
                    for (int k = 0; k < nw; k++) s += s_dred[k];
                    W.p_l1[b] = s;
                    W.s_alo[b] = a_lo;
                    W.c_kg[b] = tkg;
                    W.c_ka[b] = tka;
                    W.c_nz[b] = nz_base;
                    W.c_nnzx[b] = tnx;
                }
            }
            ok = grid_sync(W.bar, G, gen);
            if (!ok) return false;
        }

        // ------------------------------------------------------------ output
        for (int i = b * kThreads + tid; i < K; i += G * kThreads) xout[i] = T(0);
        ok = grid_sync(W.bar, G, gen);
        if (!ok) return false;
        {
            int p_lo, p_hi, a_lo;
            cta_slice(P, P.is_group ? W.aoff[cur] : nullptr, nA_g, nA_a, b, G, &p_lo, &p_hi, &a_lo);
            for (int p = p_lo + tid; p < p_hi; p += kThreads) {
                int gid = __ldcg(W.act[cur] + p);
                int lo_a = P.is_group ? __ldcg(W.aoff[cur] + p) : p;
                int c0 = P.is_group ? P.goff[gid] : gid;
                int sz = P.is_group ? P.goff[gid + 1] - P.goff[gid] : 1;
                for (int q = 0; q < sz; q++) xout[c0 + q] = (T)__ldcg(W.xc[cur] + lo_a + q);
            }
            if (b == 0 && tid == 0) {
                R->iters = iters;
                R->status = (P.tol > 0.0 && !(gap <= P.tol * 0.5 * yy)) ? kDevNotConverged : kDevOk;
                R->n_active = nA_a;
                R->nnz = nnz_last;
                R->gap = gap;
                R->primal = primal;
                R->dual = primal - gap;
                R->lambda = lam;
                R->lambda_max = lstar;
                R->cols_corr = cols_corr;
                R->cols_synth = cols_synth;
            }
        }
        ok = grid_sync(W.bar, G, gen);
        if (!ok) return false;
    }
    return true;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) solve_kernel(const SolveP<T> P)
{
    if (!solve_body<T>(P) && blockIdx.x == 0 && threadIdx.x == 0) {
        const int n = P.n_lambda > 0 ? P.n_lambda : 1;
        for (int j = 0; j < n; j++) P.res[j].status = kDevTimeout;
    }
}

// ------------------------------------------------------------ host launcher

template <typename T>
static ds_status launch_t(ds_ctx* ctx, const ds_dict* dict, const void* y_dev, const void* x0_dev, int n_lambda,
                          const double* lambdas_host, const ds_options* opt, void* xout_dev, int64_t ldx,
                          DevResult* res_host, float* ms)
{
    constexpr int EV = 16 / sizeof(T);
    const int N = (int)dict->N, K = (int)dict->K, nG = dict->nG;
    const int chunk = 32 * EV * kU;
    const int nchunk = (N + chunk - 1) / chunk;
    const int npad = nchunk * chunk;
    const int G = ctx->num_sms;
    if (G > kThreads) return DS_ERR_UNSUPPORTED;  // per-CTA prefix arrays are filled one per thread

    // shared memory: theta + zpart + cols, and room for n (hi/lo) in the precompute
    size_t fixed = npad * sizeof(T);
    size_t budget = ctx->smem_optin > 48 * 1024 ? ctx->smem_optin - 40 * 1024 : 48 * 1024;
    if (fixed + 64 * (nchunk * sizeof(T) + 4) > budget) return DS_ERR_UNSUPPORTED;
    int RA = (int)std::min<size_t>(512, (budget - fixed) / (nchunk * sizeof(T) + 4));
    if (dict->is_group && RA < dict->max_gsize) return DS_ERR_UNSUPPORTED;
    size_t smem = fixed + (size_t)RA * (nchunk * sizeof(T) + 4);
    smem = std::max(smem, (size_t)npad * 8);
    if (smem > budget) return DS_ERR_UNSUPPORTED;

    // workspace
    Bump bp{nullptr, 0};
    auto layout = [&](Ws<T>& w, double** lam_dev, DevResult** res_dev) {
        w.bar = bp.take<GridBarrier>(1);
        w.theta = bp.take<T>(npad);
        w.b = bp.take<double>(K);
        w.tv = bp.take<double>(K);
        w.thr = bp.take<double>(nG);
        w.nvec = bp.take<double>(N);
        for (int k = 0; k < 2; k++) {
            w.act[k] = bp.take<int>(nG);
            w.aoff[k] = bp.take<int>(nG + 1);
            w.xc[k] = bp.take<double>(K);
            w.uc[k] = bp.take<double>(K);
        }
        w.xn = bp.take<double>(K);
        w.un = bp.take<double>(K);
        w.keep = bp.take<int>(nG);
        w.nz_col = bp.take<int>(K);
        w.nz_u = bp.take<double>(K);
        w.nz_x = bp.take<double>(K);
        w.s_alo = bp.take<int>(G);
        w.c_kg = bp.take<int>(G);
        w.c_ka = bp.take<int>(G);
        w.c_nz = bp.take<int>(G);
        w.c_nnzx = bp.take<int>(G);
        w.p_m = bp.take<double>(G);
        w.p_l1 = bp.take<double>(G);
        w.p_a = bp.take<double>(G);
        w.p_b = bp.take<double>(G);
        w.p_r = bp.take<double>(G);
        w.p_v = bp.take<double>(G);
        w.p_i = bp.take<int>(G);
        *lam_dev = bp.take<double>(std::max(n_lambda, 1));
        *res_dev = bp.take<DevResult>(std::max(n_lambda, 1));
    };
    Ws<T> w;
    double* lam_dev;
    DevResult* res_dev;
    layout(w, &lam_dev, &res_dev);
    ds_status st = ctx_reserve(ctx, bp.off + 256);
    if (st != DS_OK) return st;
    bp = Bump{reinterpret_cast<char*>(ctx->ws), 0};
    layout(w, &lam_dev, &res_dev);

    SolveP<T> P;
    P.D = reinterpret_cast<const T*>(dict->D);
    P.N = N; P.K = K; P.ld = (int)dict->ld; P.nG = nG; P.is_group = dict->is_group;
    P.goff = dict->goff; P.w = dict->w; P.spec = dict->spec; P.colnorm = dict->colnorm;
    P.fmax = dict->fmax;
    {
        // worst-case rounding of the FP GEMV: each product goes through at most
        // kU*EV FMAs in a lane, 5 shuffle additions and nchunk chunk additions
        const double u = sizeof(T) == 4 ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53);
        const double k = kU * EV + 5 + nchunk;
        P.gamma = 1.01 * k * u / (1.0 - k * u);
    }
    P.eps_test = sizeof(T) == 4 ? 1e-9 : 1e-11;
    P.y = reinterpret_cast<const T*>(y_dev);
    P.x0 = reinterpret_cast<const T*>(x0_dev);
    P.n_lambda = n_lambda;
    P.lambdas = lam_dev;
    P.lambda_rel = opt ? opt->lambda_rel : 0;
    P.alg = opt ? opt->alg : 1;
    P.test = opt ? opt->test : 0;
    P.dynamic = opt ? opt->dynamic : 1;
    P.max_iter = opt ? opt->max_iter : 1;
    P.tol = opt ? opt->tol_gap_rel : 0.0;
    P.L = (opt && opt->L > 0) ? opt->L : dict->L;
    P.x_out = reinterpret_cast<T*>(xout_dev);
    P.ldx = ldx;
    P.res = res_dev;
    P.hist = ctx->hist;
    P.hist_rows = ctx->hist_rows;
    P.ws = w;
    P.RA = RA;
    P.nchunk = nchunk;
    P.npad = npad;

    cudaStream_t s = ctx->stream;
    if (n_lambda > 0 &&
        cudaMemcpyAsync(lam_dev, lambdas_host, sizeof(double) * n_lambda, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaMemsetAsync(w.bar, 0, sizeof(GridBarrier), s) != cudaSuccess) return DS_ERR_CUDA;
    if (cudaMemsetAsync(res_dev, 0, sizeof(DevResult) * std::max(n_lambda, 1), s) != cudaSuccess) return DS_ERR_CUDA;

    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(solve_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(ctx->smem_optin - 40 * 1024)) != cudaSuccess)
            return DS_ERR_CUDA;
        attr_set = true;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, solve_kernel<T>, kThreads, smem) != cudaSuccess)
        return DS_ERR_CUDA;
    if (occ < 1) return DS_ERR_UNSUPPORTED;

    void* args[] = {(void*)&P};
    ctx->launches++;
    cudaEventRecord(ctx->ev0, s);
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)solve_kernel<T>, dim3(G), dim3(kThreads), args, smem, s);
    if (e != cudaSuccess) {
        fprintf(stderr, "dscreen: solve launch failed: %s\n", cudaGetErrorString(e));
        return DS_ERR_CUDA;
    }
    cudaEventRecord(ctx->ev1, s);
    if (cudaMemcpyAsync(res_host, res_dev, sizeof(DevResult) * std::max(n_lambda, 1), cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return DS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return DS_ERR_CUDA;
    if (ms) cudaEventElapsedTime(ms, ctx->ev0, ctx->ev1);
    for (int j = 0; j < std::max(n_lambda, 1); j++)
        if (res_host[j].status == kDevTimeout) return DS_ERR_TIMEOUT;
    return DS_OK;
}

ds_status launch_solve(ds_ctx* ctx, const ds_dict* dict, const void* y_dev, const void* x0_dev, int n_lambda,
                       const double* lambdas_host, const ds_options* opt, void* xout_dev, int64_t ldx,
                       DevResult* res_host, float* ms)
{
    if (dict->dtype == DS_FP32)
        return launch_t<float>(ctx, dict, y_dev, x0_dev, n_lambda, lambdas_host, opt, xout_dev, ldx, res_host, ms);
    return launch_t<double>(ctx, dict, y_dev, x0_dev, n_lambda, lambdas_host, opt, xout_dev, ldx, res_host, ms);
}

ds_status launch_lambda_max(ds_ctx* ctx, const ds_dict* dict, const void* y_dev, double* lmax)
{
    DevResult r[1];
    ds_status st = launch_solve(ctx, dict, y_dev, nullptr, 0, nullptr, nullptr, nullptr, 0, r, nullptr);
    if (st == DS_OK) *lmax = r[0].lambda_max;
    return st;
}

}  // namespace ds
