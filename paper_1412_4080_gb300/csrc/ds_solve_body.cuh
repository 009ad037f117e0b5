// ds_solve_body.cuh -- device side of a screened ISTA/FISTA solve run by a team
// of CTAs (Algorithm 3 with the Table 1 updates): the per-solve workspace and
// parameters, float-float iterate arithmetic, and solve_body(), shared by the
// single-solve kernel (team = whole grid) and the multi-team kernels of the
// batched and served modes (team = a few CTAs, or one).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdio>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "ds_internal.h"

namespace ds {

constexpr int kThreads = 512;
constexpr int kMaxG = 160;  // CTAs of the persistent grid (one per SM) handled by the fixed reductions
constexpr int kU = 4;         // 16-byte vectors per lane per GEMV item
constexpr int kRowTile = 32;  // rows per synthesis tile
constexpr int kSyn = 8;       // dictionary loads in flight per lane in the synthesis
constexpr int kSpec = 2;      // entries of every nonzero list fetched with its length
// adaptive steps (readings of the rules Table 1 cites): SpaRSA's sufficient-decrease constant (its
// window of 5 accepted objective values is in ScalarState) and the rejections allowed per iteration,
// after which the last attempt is kept
constexpr double kSparsaSigma = 1e-5;
constexpr int kRetryCap = 40;

// Iterates (x, u) and per-CTA partial sums: float-float pairs for FP32
// dictionaries, doubles for FP64 ones.
template <typename T> struct IterT;
template <> struct IterT<float> { using type = FF; };
template <> struct IterT<double> { using type = double; };

template <typename T>
struct Ws {
    using X = typename IterT<T>::type;
    GridBarrier* bar;
    T* theta;
    double* b;
    double* tv;
    double* thr;
    double* nvec;
    int* act[2];
    int* aoff[2];
    // FP32 dictionaries, sphere tests: (threshold - eps) rounded down to FP32, in list order
    float* thrc[2];
    // FP32 dictionaries, dynamic dome (Lemma 4), per atom and lambda: d_i^T c0, t_i = d_*^T d_i,
    // sqrt(1 - t_i^2), 1/||d_i|| - eps rounded down
    float4* domef;
    // iterates carry about twice the dictionary's precision: in plain FP32,
    // u - z/L would quantise z to multiples of L ulp(x), a KKT floor near 1e-6
    X* xc[2];
    X* uc[2];
    int* keep;
    int* nz_col;
    X* nz_u;
    X* nz_x;
    int* nz_t;  // test data of the entry's group: FP32 threshold bits (FP32 sphere tests) or group id
    int* c_ka;
    int* c_nz;
    int* c_nnzx;
    T* p_m;
    X* p_l1;
    X* p_a;
    X* p_b;
    X* p_r;
    double* p_v;
    int* p_i;
    double* p_cn;
    // adaptive steps (backtracking, SpaRSA, TwIST): a second theta buffer (the last accepted
    // theta while a step is being tried), and per atom, at the positions of the step's iterates,
    // the correlation z_t, the point the gradient step started from and x_{t-1}; per-CTA partials
    // of ||xbar_t - base||^2 and ||D xbar_t - y - theta_acc||^2 = ||D (xbar_t - base)||^2
    T* theta2;
    T* zS;
    X* bS;
    X* pS;
    X* p_sq;
    X* p_dq;
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
    int alg, test, dynamic, max_iter, warm_start;
    int step_mode;       // 0 fixed L (or Chambolle-Pock), 1 backtracking (ISTA/FISTA), 2 SpaRSA, 3 TwIST
    double bt_L0;        // first L of the backtracking
    double tw_a, tw_b;   // TwIST's alpha and beta
    int gap_every;       // the stopping rule is evaluated every gap_every iterations
    double cp_tau0, cp_sigma0, cp_gamma;  // Chambolle-Pock (alg 2): initial steps and gamma
    double tol, L;
    T* x_out;
    long long ldx;
    DevResult* res;
    double* hist;
    int hist_rows;
    int* scr_log;  // non-null: per lambda j < scr_rows, K ints: the iteration whose test screened each atom
    int scr_rows;
    Ws<T> ws;
    int RA, nchunk, npad;
    int syn_cap;          // nonzero-list entries the dynamic shared buffer holds (multiple of 16)
    double* colnorm_w;    // non-null: the kernel computes ||d_i|| here (and fmax) in its first pass
    const double* fista;  // FISTA table: (coefficient (l_{t-1} - 1) / l_t, l_t) for t = 1..fista_n
    int fista_n;
    const volatile int* abort_flag;  // non-null: a nonzero value ends the solve at the next check
    // low-precision working copy (precision variant): bulk iterations read it, FP32 polish follows
    const void* Dlo;
    int lo_kind, ld_lo;
    const float* lo_scale;
    double emax, gamma_lo, lo_switch;
    // the one-cluster solve of small FP64 Lasso problems: the dictionary as float-float pairs (K x N)
    // and the single lambda as given (lambda_rel applies to it)
    const float2* Dff;
    double lam0;
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

template <typename T> __device__ __forceinline__ T round_up_to(double v);
template <> __device__ __forceinline__ float round_up_to<float>(double v) { return __double2float_ru(v); }
template <> __device__ __forceinline__ double round_up_to<double>(double v) { return v; }

// ---- iterate arithmetic (float-float for FP32 dictionaries, FP64 otherwise)
// max over a group of ||z_g|| / w_g, rounded up so that the maximum stays an upper bound of the exact
// value: FP32 with directed rounding (the pair summed up, 2^-20 for the error of the compensated sum);
// FP64 as computed
__device__ __forceinline__ float group_zmax(const Dot2f& zq, double wg)
{
    const float s = __fmul_ru(__fadd_ru(zq.s, zq.c), 1.000001f);
    return __fdiv_ru(__fsqrt_ru(s), __double2float_rd(wg));
}
__device__ __forceinline__ double group_zmax(const Dot2d& zq, double wg) { return sqrt(zq.value()) / wg; }

__device__ __forceinline__ FF ldcg_x(const FF* p)
{
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return FF{v.x, v.y};
}
__device__ __forceinline__ double ldcg_x(const double* p) { return __ldcg(p); }
__device__ __forceinline__ bool it_nz(FF a) { return a.h != 0.f; }
__device__ __forceinline__ bool it_nz(double a) { return a != 0.0; }
__device__ __forceinline__ FF it_zero(FF*) { return FF{0.f, 0.f}; }
__device__ __forceinline__ double it_zero(double*) { return 0.0; }
__device__ __forceinline__ FF it_from(float v, FF*) { return FF{v, 0.f}; }
__device__ __forceinline__ double it_from(double v, double*) { return v; }
__device__ __forceinline__ float it_round(FF a) { return a.h + a.l; }
__device__ __forceinline__ double it_round(double a) { return a; }
__device__ __forceinline__ double it_dbl(FF a) { return ff_to_double(a); }
__device__ __forceinline__ double it_dbl(double a) { return a; }
__device__ __forceinline__ FF it_cast(double a, FF*) { return ff_from_double(a); }
__device__ __forceinline__ double it_cast(double a, double*) { return a; }
// gradient step v = u - z * (1/L)
__device__ __forceinline__ FF it_grad_step(FF u, float z, float invL) { return ff_sub(u, ff_prod(z, invL)); }
__device__ __forceinline__ double it_grad_step(double u, double z, double invL) { return fma(-z, invL, u); }
// soft threshold (eq. softTh): sign(v) max(|v| - thr, 0)
__device__ __forceinline__ FF it_soft(FF v, FF thr)
{
    if (v.h > 0.f) {
        const FF a = ff_sub(v, thr);
        return a.h > 0.f ? a : FF{0.f, 0.f};
    }
    if (v.h < 0.f) {
        const FF a = ff_add(v, thr);
        return a.h < 0.f ? a : FF{0.f, 0.f};
    }
    return FF{0.f, 0.f};
}
__device__ __forceinline__ double it_soft(double v, double thr)
{
    const double a = fabs(v) - thr;
    return a > 0.0 ? copysign(a, v) : 0.0;
}
// FISTA extrapolation u = x + bt (x - xo)
__device__ __forceinline__ FF it_momentum(FF x, FF xo, FF bt) { return ff_add(x, ff_mul(ff_sub(x, xo), bt)); }
__device__ __forceinline__ double it_momentum(double x, double xo, double bt) { return fma(bt, x - xo, x); }
__device__ __forceinline__ FF it_scale(FF v, FF f) { return ff_mul(v, f); }
__device__ __forceinline__ FF it_diff(FF a, FF b) { return ff_sub(a, b); }
// TwIST's two-step combination (1 - a) x_{t-2} + (a - b) x_{t-1} + b p
__device__ __forceinline__ FF it_twist(FF x2, FF x1, FF p, double a, double b)
{
    return ff_add(ff_add(ff_mul(x2, ff_from_double(1.0 - a)), ff_mul(x1, ff_from_double(a - b))),
                  ff_mul(p, ff_from_double(b)));
}
__device__ __forceinline__ double it_twist(double x2, double x1, double p, double a, double b)
{
    return fma(1.0 - a, x2, fma(a - b, x1, b * p));
}
__device__ __forceinline__ double it_diff(double a, double b) { return a - b; }
__device__ __forceinline__ double it_scale(double v, double f) { return v * f; }
// accumulators: |x| and x^2
__device__ __forceinline__ void acc_abs(Dot2f& acc, FF x)
{
    const float sg = x.h < 0.f ? -1.f : 1.f;
    dot2_merge(acc, sg * x.h, sg * x.l);
}
__device__ __forceinline__ void acc_abs(Dot2d& acc, double x) { acc.s += fabs(x); }
__device__ __forceinline__ void acc_sq(Dot2f& acc, FF x)
{
    acc.add(x.h, x.h);
    acc.c = fmaf(2.f * x.h, x.l, acc.c);
}
__device__ __forceinline__ void acc_sq(Dot2d& acc, double x) { acc.s = fma(x, x, acc.s); }
__device__ __forceinline__ void acc_add_dbl(Dot2f& acc, double v)
{
    const FF f = ff_from_double(v);
    dot2_merge(acc, f.h, f.l);
}
__device__ __forceinline__ void acc_add_dbl(Dot2d& acc, double v) { acc.s += v; }
// synthesis term acc += d * c
__device__ __forceinline__ void syn_add(Dot2f& acc, float d, FF c)
{
    acc.add(d, c.h);
    acc.c = fmaf(d, c.l, acc.c);
}
__device__ __forceinline__ void syn_add(Dot2d& acc, double d, double c) { acc.add(d, c); }
// per-CTA partials
__device__ __forceinline__ void part_put(FF* p, const Dot2f& a) { *p = FF{a.s, a.c}; }
__device__ __forceinline__ void part_put(double* p, const Dot2d& a) { *p = a.s; }
__device__ __forceinline__ double part_sum_fixed(const FF* p, int n, int lane)
{
    Dot2f acc;
    for (int i = lane; i < n; i += 32) {
        const float2 v = __ldcg(reinterpret_cast<const float2*>(p + i));
        dot2_merge(acc, v.x, v.y);
    }
    return dot2_warp_sum(acc);
}
__device__ __forceinline__ double part_sum_fixed(const double* p, int n, int lane) { return warp_sum_fixed(p, n, lane); }
template <int Q> __device__ __forceinline__ double part_sum_regs(const FF (&v)[Q])
{
    Dot2f acc;
#pragma unroll
    for (int q = 0; q < Q; q++) dot2_merge(acc, v[q].h, v[q].l);
    return dot2_warp_sum(acc);
}
template <int Q> __device__ __forceinline__ double part_sum_regs(const double (&v)[Q])
{
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < Q; q++) acc += v[q];
    return warp_sum(acc);
}
__device__ __forceinline__ Dot2f acc_warp_reduce(Dot2f a) { return dot2_warp_reduce(a); }
__device__ __forceinline__ Dot2d acc_warp_reduce(Dot2d a)
{
    a.s = warp_sum(a.s);
    return a;
}
__device__ __forceinline__ void acc_merge_acc(Dot2f& a, const Dot2f& b) { dot2_merge(a, b.s, b.c); }
__device__ __forceinline__ void acc_merge_acc(Dot2d& a, const Dot2d& b) { a.s += b.s; }
// theta_r = w_u - y_r, computed from the compensated sum and rounded once
__device__ __forceinline__ float theta_from(const Dot2f& wu, float y)
{
    const FF t = ff_two_sum(wu.s, -y);
    return t.h + (t.l + wu.c);
}
__device__ __forceinline__ double theta_from(const Dot2d& wu, double y) { return wu.s - y; }
// (w_x - y_r)^2 into an accumulator
__device__ __forceinline__ void acc_resid_sq(Dot2f& acc, const Dot2f& wx, float y)
{
    FF t = ff_two_sum(wx.s, -y);
    t = ff_fast_two_sum(t.h, t.l + wx.c);
    acc_sq(acc, t);
}
__device__ __forceinline__ void acc_resid_sq(Dot2d& acc, const Dot2d& wx, double y)
{
    const double r = wx.s - y;
    acc.s = fma(r, r, acc.s);
}
// ((w_x - y_r) - th)^2 into an accumulator: th is the residual of the last accepted step, so the
// difference is D (xbar - base) for the adaptive steps, formed from w_x - y in double length first
__device__ __forceinline__ void acc_diff_sq(Dot2f& acc, const Dot2f& wx, float y, float th)
{
    FF t = ff_two_sum(wx.s, -y);
    t = ff_fast_two_sum(t.h, t.l + wx.c);
    const FF d = ff_two_sum(t.h, -th);
    acc_sq(acc, ff_two_sum(d.h, d.l + t.l));
}
__device__ __forceinline__ void acc_diff_sq(Dot2d& acc, const Dot2d& wx, double y, double th)
{
    const double d = (wx.s - y) - th;
    acc.s = fma(d, d, acc.s);
}

// float-float (or FP64) partial sums parked in one 8-byte shared slot
__device__ __forceinline__ void acc_store(double* slot, const Dot2f& a)
{
    *reinterpret_cast<float2*>(slot) = make_float2(a.s, a.c);
}
__device__ __forceinline__ void acc_store(double* slot, const Dot2d& a) { *slot = a.s; }
__device__ __forceinline__ void acc_merge(Dot2f& a, const double* slot)
{
    const float2 v = *reinterpret_cast<const float2*>(slot);
    dot2_merge(a, v.x, v.y);
}
__device__ __forceinline__ void acc_merge(Dot2d& a, const double* slot) { a.s += *slot; }

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

// ---- correlation from the low-precision copy: one 512-row chunk per item, like
// the FP32 path (BF16: two 16-byte vectors of 8 values per lane; FP8: one of 16),
// accumulated in FP32 against theta in shared memory.
__device__ __forceinline__ float bf16_lo(unsigned int w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(unsigned int w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ float dot_lo_bf16(uint4 d, float4 t0, float4 t1, float s)
{
    s = fmaf(bf16_lo(d.x), t0.x, s);
    s = fmaf(bf16_hi(d.x), t0.y, s);
    s = fmaf(bf16_lo(d.y), t0.z, s);
    s = fmaf(bf16_hi(d.y), t0.w, s);
    s = fmaf(bf16_lo(d.z), t1.x, s);
    s = fmaf(bf16_hi(d.z), t1.y, s);
    s = fmaf(bf16_lo(d.w), t1.z, s);
    s = fmaf(bf16_hi(d.w), t1.w, s);
    return s;
}
__device__ __forceinline__ float2 fp8x2_to_float2(unsigned int w16)
{
    const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w16 & 0xffffu), __NV_E4M3);
    return __half22float2(*reinterpret_cast<const __half2*>(&h));
}
__device__ __forceinline__ float dot_lo_fp8_word(unsigned int w, float4 t, float s)
{
    const float2 a = fp8x2_to_float2(w), b = fp8x2_to_float2(w >> 16);
    s = fmaf(a.x, t.x, s);
    s = fmaf(a.y, t.y, s);
    s = fmaf(b.x, t.z, s);
    s = fmaf(b.y, t.w, s);
    return s;
}

template <int KIND, int IPW>
__device__ __noinline__ void gemv_lowp(const void* Dlo, int ld_lo, const float* lo_scale, const float* th_s,
                                          float* zpart, const int* cols_s, int natoms, int nchunk, int lane, int warp,
                                          int nw)
{
    constexpr int VPI = KIND == 1 ? 2 : 1;   // 16-byte vectors per item per lane
    constexpr int EPV = KIND == 1 ? 8 : 16;  // elements per vector
    constexpr int ES = KIND == 1 ? 2 : 1;    // bytes per element
    const int ldv = ld_lo / EPV;
    const float4* thv = reinterpret_cast<const float4*>(th_s);
    const int nitems = natoms * nchunk;
    for (int j0 = warp * IPW; j0 < nitems; j0 += nw * IPW) {
        uint4 dv[IPW][VPI];
        int aa[IPW], cc[IPW];
#pragma unroll
        for (int q = 0; q < IPW; q++) {
            const int j = j0 + q < nitems ? j0 + q : j0;
            aa[q] = j / nchunk;
            cc[q] = j - aa[q] * nchunk;
            const uint4* col =
                reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(Dlo) + (size_t)cols_s[aa[q]] * ld_lo * ES);
#pragma unroll
            for (int k = 0; k < VPI; k++) {
                const int v = cc[q] * (32 * VPI) + k * 32 + lane;
                dv[q][k] = (j0 + q < nitems && v < ldv) ? __ldg(col + v) : make_uint4(0u, 0u, 0u, 0u);
            }
        }
#pragma unroll
        for (int q = 0; q < IPW; q++) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < VPI; k++) {
                const int v = cc[q] * (32 * VPI) + k * 32 + lane;
                if (KIND == 1) {
                    s = dot_lo_bf16(dv[q][k], thv[2 * v], thv[2 * v + 1], s);
                } else {
                    s = dot_lo_fp8_word(dv[q][k].x, thv[4 * v], s);
                    s = dot_lo_fp8_word(dv[q][k].y, thv[4 * v + 1], s);
                    s = dot_lo_fp8_word(dv[q][k].z, thv[4 * v + 2], s);
                    s = dot_lo_fp8_word(dv[q][k].w, thv[4 * v + 3], s);
                }
            }
            s = warp_sum(s);
            if (KIND == 2) s *= __ldg(lo_scale + cols_s[aa[q]]);
            if (lane == 0 && j0 + q < nitems) zpart[aa[q] * nchunk + cc[q]] = s;
        }
    }
}

// ---- correlation from the FP32 dictionary: item (atom, 512-row chunk), IPW items
// of kU 16-byte vectors per lane in flight per warp (the loads of a round are all
// issued before the first product), theta read from shared memory; each item's
// dot product is summed in the same order whatever IPW is.
template <int IPW>
__device__ __noinline__ void gemv_f32(const float* D, int ld, const float* th_s, float* zpart, const int* cols_s,
                                      int natoms, int nchunk, int lane, int warp, int nw)
{
    const int ldv = ld / 4;
    const float4* thv = reinterpret_cast<const float4*>(th_s);
    const int nitems = natoms * nchunk;
    for (int j0 = warp * IPW; j0 < nitems; j0 += nw * IPW) {
        float4 dv[IPW][kU];
        int aa[IPW], cc[IPW];
#pragma unroll
        for (int q = 0; q < IPW; q++) {
            const int j = j0 + q < nitems ? j0 + q : j0;
            aa[q] = j / nchunk;
            cc[q] = j - aa[q] * nchunk;
            const float4* col = reinterpret_cast<const float4*>(D + (size_t)cols_s[aa[q]] * ld);
#pragma unroll
            for (int k = 0; k < kU; k++) {
                const int v = cc[q] * (32 * kU) + k * 32 + lane;
                dv[q][k] = (j0 + q < nitems && v < ldv) ? __ldg(col + v) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        float s[IPW];
#pragma unroll
        for (int q = 0; q < IPW; q++) {
            s[q] = 0.f;
#pragma unroll
            for (int k = 0; k < kU; k++) s[q] = vdot(dv[q][k], thv[cc[q] * (32 * kU) + k * 32 + lane], s[q]);
        }
        if constexpr (IPW == 4) {
            // the four sums in one butterfly: at offsets 16 and 8 each lane keeps the items of its half and
            // sends the others, so lanes 8q .. 8q+7 end up with item q (the same pairs as warp_sum)
            const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
            float k0 = h16 ? s[2] : s[0], k1 = h16 ? s[3] : s[1];
            k0 += __shfl_xor_sync(0xffffffffu, h16 ? s[0] : s[2], 16);
            k1 += __shfl_xor_sync(0xffffffffu, h16 ? s[1] : s[3], 16);
            float v = h8 ? k1 : k0;
            v += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            const int q = (h16 ? 2 : 0) + (h8 ? 1 : 0);
            if ((lane & 7) == 0 && j0 + q < nitems) zpart[aa[q] * nchunk + cc[q]] = v;
        } else {
#pragma unroll
            for (int q = 0; q < IPW; q++) {
                const float v = warp_sum(s[q]);
                if (lane == 0 && j0 + q < nitems) zpart[aa[q] * nchunk + cc[q]] = v;
            }
        }
    }
}

// --------------------------------------------------------------- the kernel

// Per-solve scalar state that only thread 0 of each CTA updates, kept in shared
// memory so that it occupies no registers in the other threads.
struct ScalarState {
    double alpha, beta, mu_nom, R2n, R2s_last, rad, lf, s_unc, sqrt_beta, gap, primal, best_gap;
    double cp_tau, cp_sigma;  // Chambolle-Pock: tau_{t-1}, sigma_{t-1}
    long long cols_corr, cols_synth, cols_lowp;
    int iters, since_best, low, t0;  // t0: iteration at which the current FISTA sequence started
    // adaptive steps: the step constant being tried (backtracking L, SpaRSA alpha), the last
    // accepted objective values (SpaRSA's nonmonotone window, TwIST's reference), the attempt's
    // FISTA coefficient, rejections of the current step and TwIST's shrinkage-step fallback
    double Lstep, Fprev, bt_att;
    double Fh[5];
    int nh, hpos, tries, fallback;
    // Lemma 8 terms of the newest theta, committed only once its step is accepted
    double n_alpha, n_beta, n_m2a, n_s_unc, n_sqrt_beta;
    float n_s_unc_f, n_sqb_f;
};

// Asynchronous copies global -> shared (cp.async): prefetched values wait in shared memory, not
// in registers, until the thread that issued them reads them after pf_wait().
__device__ __forceinline__ void pf4(void* s, const void* g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void pf8(void* s, const void* g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void pf_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The first kSpec entries of one CTA's nonzero list, fetched with its length.
template <typename X>
struct __align__(8) SpecSlot {
    X u[kSpec], x[kSpec];
    int col[kSpec], t[kSpec];
};

// CTA-uniform constants of a launch and of its current lambda, kept in shared memory:
// the persistent kernel needs its registers for the loads it keeps in flight.
template <typename T>
struct SolveK {
    double fmax_d, nn, nty, wstar2;
    double lam, inv_lam, yy_l2, psi, coef, delta, nstar, psi_dome, thrL, rad2_slack;
    double hyy, hlam2, tol_abs, delta2, m2a;  // 1/2||y||^2, lambda^2/2, tol 1/2||y||^2, delta^2, -2 theta^T y / lambda
    float gfm, gfm_lo;   // FP32 max |z| rounding bound per unit ||theta|| (master, low-precision copy), rounded up
    float sqb_f, s_unc_f;  // ||theta|| (rounded up) and the unclipped Lemma 8 scaling, FP32
    float bt_h, bt_l;      // FISTA coefficient of the iteration as a float-float pair
    float dome_f[4];  // FP32 dome test of the current iteration: R, psi, rho (rounded up), branch threshold
    int* slog;  // screening log of the current lambda (null: not recorded)
    T* thN;     // theta written by the synthesis (A) and correlated in (B)
    T* thA;     // adaptive steps: the theta of the last accepted step
    T invL;
    T cp_sig, cp_inv1ps;  // Chambolle-Pock: sigma_{t-1} and 1 / (1 + sigma_{t-1}) of the next dual update
    typename IterT<T>::type thrX;
};

// One solve (or lambda path) by a team of G CTAs (rank b) that synchronise on
// `bar`; `gen` is the calling thread's running barrier target.
// ADAPT = false compiles the fixed-step rows only (ISTA, FISTA, Chambolle-Pock without backtracking):
// the adaptive-step code below is then absent from the kernel, and so is its register pressure.
template <typename T, bool ADAPT = true, int GRP = -1>
__device__ __forceinline__ bool solve_body(const SolveP<T>& P, const int b, const int G, GridBarrier* bar,
                                           unsigned int& gen)
{
    const int SM = ADAPT ? P.step_mode : 0;  // adaptive step rule of this solve (0: fixed step)
    const bool is_grp = GRP < 0 ? P.is_group != 0 : GRP == 1;  // Group-Lasso (GRP: fixed at compile time)
    using V = typename Vec4<T>::type;
    using X = typename IterT<T>::type;
    using Acc = typename Dot2<T>::type;
    constexpr int EV = 16 / sizeof(T);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* th_s = reinterpret_cast<T*>(smem_raw);
    T* zpart = th_s + P.npad;
    int* cols_s = reinterpret_cast<int*>(zpart + (size_t)P.RA * P.nchunk);

    __shared__ int s_tmp[32];
    __shared__ double s_dred[32];
    __shared__ int s_ired[32];
    __shared__ int s_pref[1025];
    __shared__ int s_alo_s[kThreads];
    __shared__ int s_kg[kMaxG];
    __shared__ float s_radf;
    __shared__ double s_red[2][kThreads / 32][kRowTile];
    __shared__ double s_sc[16];
    __shared__ int s_si[16];
    __shared__ ScalarState S_;
    __shared__ SolveK<T> C_;
    // per-thread prefetch slots (cp.async): two ints, a float and two iterate values
    __shared__ int s_pf_i0[kThreads], s_pf_i1[kThreads], s_pf_i2[kThreads];
    __shared__ float s_pf_f0[kThreads];
    __shared__ __align__(8) X s_pf_u[kThreads];
    __shared__ __align__(8) X s_pf_x[kThreads];
    // the nonzero-list heads of every CTA, in the synthesis merge buffer (free when they are read)
    static_assert(sizeof(SpecSlot<X>) * kMaxG <= sizeof(double) * 2 * (kThreads / 32) * kRowTile, "spec slots");
    SpecSlot<X>* const s_spec = reinterpret_cast<SpecSlot<X>*>(&s_red[0][0][0]);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kThreads / 32;
    const Ws<T>& W = P.ws;
    auto xbuf = [&](int i) -> X* { return i == 0 ? W.xc[0] : W.xc[1]; };
    auto ubuf = [&](int i) -> X* { return i == 0 ? W.uc[0] : W.uc[1]; };

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
        const bool norms = P.colnorm_w != nullptr;
        double cmax = 0.0;
        for (int i = gwarp; i < K; i += total_warps) {
            const V* col = reinterpret_cast<const V*>(P.D + (size_t)i * ld);
            typename Dot2<T>::type acc, nrm;
            for (int v = lane; v < ldv; v += 32) {
                V d = __ldg(col + v);
                V q = yv[v];
                if constexpr (EV == 4) {
                    acc.add(d.x, q.x); acc.add(d.y, q.y); acc.add(d.z, q.z); acc.add(d.w, q.w);
                    if (norms) {
                        // rows N..ld-1 of a caller's D are not part of the atom
                        const int r0 = v * 4;
                        if (r0 + 3 >= N) {
                            d.x = r0 < N ? d.x : 0.f;
                            d.y = r0 + 1 < N ? d.y : 0.f;
                            d.z = r0 + 2 < N ? d.z : 0.f;
                            d.w = 0.f;
                        }
                        nrm.add(d.x, d.x); nrm.add(d.y, d.y); nrm.add(d.z, d.z); nrm.add(d.w, d.w);
                    }
                } else {
                    acc.add(d.x, q.x); acc.add(d.y, q.y);
                    if (norms) { nrm.add(d.x, d.x); nrm.add(d.y, d.y); }
                }
            }
            double s = warp_sum(acc.value());
            if (lane == 0) W.b[i] = s;
            if (norms) {
                const double c = sqrt(warp_sum(nrm.value()));
                if (lane == 0) P.colnorm_w[i] = c;
                cmax = fmax(cmax, c);
            }
        }
        if (norms) {
            cmax = warp_max(cmax);
            if (lane == 0) s_dred[warp] = cmax;
            __syncthreads();
            if (tid == 0) {
                double m = 0.0;
                for (int k = 0; k < nw; k++) m = fmax(m, s_dred[k]);
                W.p_cn[b] = m;
            }
            __syncthreads();
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
            Acc s;
            for (int k = 0; k < nw; k++) acc_add_dbl(s, s_dred[k]);
            part_put(W.p_a + b, s);
        }
    }
    ok = grid_sync(bar, G, gen);
    if (!ok) return false;
    // column norms computed above: their maximum bounds the GEMV rounding (Lasso)
    const double* colnorm = P.colnorm_w ? P.colnorm_w : P.colnorm;
    if (tid == 0) C_.fmax_d = P.fmax;
    const double& fmax_d = C_.fmax_d;
    if (P.colnorm_w) {
        if (warp == 0) {
            const double m = warp_max_fixed(W.p_cn, G, lane);
            if (lane == 0) s_sc[11] = m * (1.0 + 1e-12);
        }
        __syncthreads();
        if (tid == 0) C_.fmax_d = s_sc[11];
    }

    // --------------------------------- P0b: lambda_* (Sec. 2.2.2 / eq. gstar)
    {
        double best = -1.0;
        int arg = 0x7fffffff;
        for (int g = b * kThreads + tid; g < nG; g += G * kThreads) {
            double s;
            if (!is_grp) {
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
    ok = grid_sync(bar, G, gen);
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
            double yy = part_sum_fixed(W.p_a, G, lane);
            if (lane == 0) { s_sc[0] = bb; s_si[0] = ba; s_sc[1] = yy; }
        }
        __syncthreads();
    }
    const double& lstar = s_sc[0];
    const int& star = s_si[0];
    const double& yy = s_sc[1];
    if (P.n_lambda == 0) {  // lambda_max query only
        if (b == 0 && tid == 0) { P.res[0].lambda_max = lstar; P.res[0].status = kDevOk; }
        return true;
    }

    const bool need_n = P.test == 2 || P.test == 3 || P.test == 5;  // DST3, DOME, DGST3
    if (tid == 0) { C_.nn = 0.0; C_.nty = 0.0; C_.wstar2 = 1.0; }
    if (need_n && lstar > 0.0) {
        // ---------------- n = D_{g*} D_{g*}^T y / lambda_*  (Lemma 6; Lasso: n = d_*)
        const int c0 = is_grp ? P.goff[star] : star;
        const int c1 = is_grp ? P.goff[star + 1] : star + 1;
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
            Acc s;
            for (int k = 0; k < nw; k++) acc_add_dbl(s, s_dred[k]);
            part_put(W.p_r + b, s);
        }
        ok = grid_sync(bar, G, gen);
        if (!ok) return false;
        if (warp == 0) {
            double s = part_sum_fixed(W.p_r, G, lane);
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
        if (tid == 0) {
            C_.nn = s_sc[2];
            double q = 0.0;
            for (int i = c0; i < c1; i++) {
                double v = __ldcg(W.b + i);
                q += v * v;
            }
            C_.nty = q / lstar;  // n^T y = ||D_{g*}^T y||^2 / lambda_*
            if (is_grp) C_.wstar2 = P.w[star] * P.w[star];
        }
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
        ok = grid_sync(bar, G, gen);
        if (!ok) return false;
    }

    // fixed slice of every CTA for the whole launch: groups [slice(k), slice(k+1)), cut at group
    // boundaries and balanced in atoms; s_alo_s[k] = its first atom (start of its nonzero list)
    auto slice_start = [&](int k) -> int {
        if (k >= G) return nG;
        if (!is_grp) return (int)((long long)k * nG / G);
        const long long target = (long long)k * K / G;
        int lo = 0, hi = nG;  // first g with goff[g] >= target
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (P.goff[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    const int g_lo = slice_start(b), g_hi = slice_start(b + 1);
    const int a_lo0 = is_grp ? (g_lo < nG ? P.goff[g_lo] : K) : g_lo;
    const int a_hi0 = is_grp ? (g_hi < nG ? P.goff[g_hi] : K) : g_hi;
    for (int k = tid; k < G; k += kThreads) {
        const int gk = slice_start(k);
        s_alo_s[k] = is_grp ? (gk < nG ? P.goff[gk] : K) : gk;
    }
    __syncthreads();

    // ================================================================ lambdas
    const double &nn = C_.nn, &nty = C_.nty, &wstar2 = C_.wstar2;
    for (int j = 0; j < P.n_lambda; j++) {
        __syncthreads();  // every thread is done with the previous lambda's constants
        if (tid == 0) {
            const double lm = P.lambda_rel ? P.lambdas[j] * lstar : P.lambdas[j];
            C_.lam = lm;
            C_.inv_lam = 1.0 / lm;
            C_.yy_l2 = yy / (lm * lm);
            C_.psi = lstar / lm - 1.0;
            // DST3 / DGST3 centre c = y/lam - coef n, offset delta = ||y/lam - c|| (Lemmas 3, 6)
            C_.coef = need_n && nn > 0.0 ? (nty / lm - wstar2) / nn : 0.0;
            C_.delta = need_n && nn > 0.0 ? fabs(nty / lm - wstar2) / sqrt(nn) : 0.0;
            C_.nstar = is_grp ? 1.0 : colnorm[star];
            C_.psi_dome = C_.psi / C_.nstar;
            C_.invL = (T)(1.0 / P.L);
            C_.thrL = lm / P.L;
            C_.thrX = it_cast(C_.thrL, (X*)nullptr);
            // absolute slack on the radius^2 for the FP64 rounding of its terms (all <= ||y||^2/lambda^2)
            C_.rad2_slack = 1e-14 * yy / (lm * lm);
            C_.gfm = __double2float_ru(P.gamma * fmax_d);
            C_.gfm_lo = __double2float_ru(P.emax + P.gamma_lo * (fmax_d + P.emax));
            C_.hyy = 0.5 * yy;
            C_.hlam2 = 0.5 * lm * lm;
            C_.tol_abs = P.tol * 0.5 * yy;
            C_.delta2 = C_.delta * C_.delta;
            C_.slog = (P.scr_log && j < P.scr_rows) ? P.scr_log + (size_t)j * K : nullptr;
            C_.thN = W.theta;
            C_.thA = W.theta2;
        }
        __syncthreads();
        const double &lam = C_.lam, &psi = C_.psi, &coef = C_.coef, &delta = C_.delta, &nstar = C_.nstar;
        const double &psi_dome = C_.psi_dome, &thrL = C_.thrL, &rad2_slack = C_.rad2_slack;
        const double &inv_lam = C_.inv_lam, &yy_l2 = C_.yy_l2;
        const T& invL = C_.invL;
        const X& thrX = C_.thrX;
        T* xout = P.x_out + (size_t)j * P.ldx;
        DevResult* R = P.res + j;
        if (!(lam < lstar)) {
            // x = 0 and theta = y / lambda is dual optimal (Sec. 2.2.2); each CTA writes its own slice
            // (a warm-started next lambda reads it back in the same CTA)
            for (int i = a_lo0 + tid; i < a_hi0; i += kThreads) {
                xout[i] = T(0);
                if (C_.slog) C_.slog[i] = 0;
            }
            if (b == 0 && tid == 0) {
                R->iters = 0; R->status = kDevOk; R->n_active = 0; R->nnz = 0;
                R->gap = 0.0; R->primal = 0.5 * yy; R->dual = 0.5 * yy; R->lambda = lam; R->lambda_max = lstar;
            }
            continue;
        }
        const bool record = (j == 0) && P.hist != nullptr;
        const bool ista = P.alg == 0;
        const bool fista = P.alg == 1;
        const bool cp = P.alg == 2;  // Chambolle-Pock (Table 1)
        const bool dyn_test = P.dynamic && P.test != 0;
        const bool sphere = P.test == 1 || P.test == 2 || P.test == 4 || P.test == 5;
        // FP32 dictionaries run the sphere tests in FP32: thresholds rounded down, radius rounded up
        const bool f32_sphere = sizeof(T) == 4 && sphere;
        const bool f32_dome = sizeof(T) == 4 && P.test == 3;  // (the dome is a Lasso test)

        // ------------------------------------------------ (C0) initial state
        // Every CTA owns the fixed slice [g_lo, g_hi) of the groups for the whole solve and keeps the
        // survivors of each test compacted inside it: act / aoff / thrc[cur] at g_lo + k (k < n_own) list
        // the live groups, the iterates of their atoms sit at a_lo0 + (0 .. na_own) of the buffers iO.
        int cur = 0, iO = 0;
        int n_own = 0, na_own = 0;
        {
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
            int nzc = 0;
            // starting point: x0, or (warm-started path) the previous lambda's solution, which this CTA
            // wrote itself (the slices are the same for every lambda)
            const T* const x0 = (P.warm_start && j > 0) ? P.x_out + (size_t)(j - 1) * P.ldx : P.x0;
            for (int base = g_lo; base < g_hi; base += kThreads) {
                const int g = base + tid;
                const bool valid = g < g_hi;
                int kept = 0, lo_a = 0, hi_a = 0, cnt = 0;
                float thf = 0.f;
                if (valid) {
                    lo_a = is_grp ? P.goff[g] : g;
                    hi_a = is_grp ? P.goff[g + 1] : g + 1;
                    // threshold of the sphere tests: (w_g - ||(D^T c)_g||) / ||D_g||  (Lemma 7)
                    double th = 0.0;
                    if (sphere) {
                        double q = 0.0;
                        for (int i = lo_a; i < hi_a; i++) {
                            double dtc = __ldcg(W.b + i) / lam - ((P.test == 2 || P.test == 5) ? coef * __ldcg(W.tv + i) : 0.0);
                            q += dtc * dtc;
                        }
                        double wg = is_grp ? P.w[g] : 1.0;
                        double sg = is_grp ? P.spec[g] : colnorm[g];
                        th = (wg - sqrt(q)) / sg;
                        W.thr[g] = th;
                        thf = __double2float_rd(th - P.eps_test);
                    }
                    if (f32_dome && P.dynamic) {
                        const double ni = colnorm[g];
                        const double dc0 = __ldcg(W.b + g) / (lam * ni);
                        const double tt = __ldcg(W.tv + g) / (ni * nstar);
                        W.domef[g] = make_float4((float)dc0, (float)tt, (float)sqrt(fmax(1.0 - tt * tt, 0.0)),
                                                 __double2float_rd(1.0 / ni - P.eps_test));
                    }
                    bool kill = false;
                    if (stat) {
                        if (P.test == 3) {
                            double ni = colnorm[g];
                            double dc0 = __ldcg(W.b + g) / (lam * ni);
                            double tt = __ldcg(W.tv + g) / (ni * nstar);
                            double up = dome_max(dc0, tt, psi_dome, rad0);
                            double dn = dome_max(-dc0, -tt, psi_dome, rad0);
                            kill = (1.0 / ni - up > P.eps_test) && (1.0 / ni - dn > P.eps_test);
                        } else {
                            kill = th - rad0 > P.eps_test;
                        }
                    }
                    kept = !kill;
                    // screening log: -1 for the static test (Algorithm 1), 0 until screened
                    if (C_.slog)
                        for (int i = lo_a; i < hi_a; i++) C_.slog[i] = kill ? -1 : 0;
                    if (kept && x0)
                        for (int i = lo_a; i < hi_a; i++) cnt += x0[i] != T(0);
                }
                int tot, totc;
                // packed scan of (groups, atoms): 512 groups of at most kMaxGroup atoms fit 20 bits
                const int pre = block_exclusive_scan(kept ? ((1 << 20) | (hi_a - lo_a)) : 0, s_tmp, &tot);
                const int pc = block_exclusive_scan(cnt, s_tmp, &totc);
                if (kept) {
                    const int ng = n_own + (pre >> 20), na = na_own + (pre & 0xfffff);
                    W.act[0][g_lo + ng] = g;
                    if (is_grp) W.aoff[0][g_lo + ng] = a_lo0 + na;
                    if (f32_sphere) W.thrc[0][g_lo + ng] = thf;
                    int e = a_lo0 + nzc + pc;
                    for (int i = lo_a; i < hi_a; i++) {
                        const X xv = x0 ? it_from(x0[i], (X*)nullptr) : it_zero((X*)nullptr);
                        W.xc[0][a_lo0 + na + i - lo_a] = xv;
                        W.uc[0][a_lo0 + na + i - lo_a] = xv;
                        if (it_nz(xv)) {
                            // u_0 = x_0: the warm start's nonzeros feed the first synthesis
                            W.nz_col[e] = i;
                            W.nz_u[e] = xv;
                            W.nz_x[e] = xv;
                            W.nz_t[e] = f32_sphere ? __float_as_int(thf) : g;
                            e++;
                        }
                    }
                }
                n_own += tot >> 20;
                na_own += tot & 0xfffff;
                nzc += totc;
            }
            if (cp)
                for (int r = b * kRowTile + (tid / kRowTile) * G * kRowTile + tid % kRowTile; r < N;
                     r += (kThreads / kRowTile) * G * kRowTile)
                    W.theta[r] = T(0);
            if (tid == 0) {
                W.c_nz[b] = nzc;
                W.c_ka[b] = na_own;
                W.c_nnzx[b] = nzc;
                Acc z0;
                part_put(W.p_l1 + b, z0);
            }
        }
        ok = grid_sync(bar, G, gen);
        if (!ok) return false;

        // scalar state, meaningful in thread 0 (the values every thread needs go through s_sc)
        double &alpha = S_.alpha, &beta = S_.beta, &mu_nom = S_.mu_nom, &R2n = S_.R2n, &R2s_last = S_.R2s_last;
        double &rad = S_.rad, &lf = S_.lf, &s_unc = S_.s_unc, &sqrt_beta = S_.sqrt_beta;
        double &gap = S_.gap, &primal = S_.primal, &best_gap = S_.best_gap;
        int &iters = S_.iters, &since_best = S_.since_best, &low = S_.low, &t0 = S_.t0;
        // work counters (dictionary columns read), the precompute passes charged to the first lambda
        long long &cols_corr = S_.cols_corr, &cols_synth = S_.cols_synth, &cols_lowp = S_.cols_lowp;
        if (tid == 0) {
            alpha = beta = mu_nom = R2n = R2s_last = rad = s_unc = sqrt_beta = primal = 0.0;
            lf = 1.0;
            gap = best_gap = INFINITY;
            iters = since_best = t0 = 0;
            S_.cp_tau = P.cp_tau0;
            S_.cp_sigma = P.cp_sigma0;
            C_.cp_sig = (T)P.cp_sigma0;
            C_.cp_inv1ps = (T)(1.0 / (1.0 + P.cp_sigma0));
            // precision variant: bulk phase on the low-precision copy, then FP32 polish
            low = (P.lo_kind != 0 && sizeof(T) == 4 && SM == 0) ? 1 : 0;
            S_.Lstep = SM == 1 ? P.bt_L0 : P.L;
            S_.tries = S_.fallback = S_.nh = S_.hpos = 0;
            S_.Fprev = INFINITY;
            S_.bt_att = 0.0;
            cols_corr = j == 0 ? (long long)K * (need_n ? 2 : 1) : 0;
            cols_synth = cols_lowp = 0;
        }
        __syncthreads();
        bool lowB = false;  // this iteration's correlation reads the low-precision copy
        int t = 1;
        for (;; t++) {
            const bool test_now = dyn_test && t > 1;  // this (A) applies the test of iteration t-1
            // ============== (A) test of iteration t-1 + synthesis theta_t = D ubar_{t-1} - y, D xbar_{t-1}
            {
                // every CTA's nonzero-list length, with the first kSpec entries fetched in the same trip
                // (the copies are issued by warps 2.. so that warps 0 and 1 start Lemma 8 at once: slot s
                // is issued by thread s + 64, modulo the block)
                const int ps = (tid + kThreads - 64) % kThreads;
                int cnz = 0;
                if (tid < G) cnz = __ldcg(W.c_nz + tid);
                if (ps < G) {
                    const int e0 = s_alo_s[ps];
#pragma unroll
                    for (int q = 0; q < kSpec; q++) {
                        const int e = e0 + q;
                        if (e < K) {
                            pf4(&s_spec[ps].col[q], W.nz_col + e);
                            pf4(&s_spec[ps].t[q], W.nz_t + e);
                            pf8(&s_spec[ps].u[q], W.nz_u + e);
                            pf8(&s_spec[ps].x[q], W.nz_x + e);
                        }
                    }
                }
                // the own slice's test inputs (one group per slot; Group-Lasso also the group and its first
                // atom) and x_{t-1} (one atom per slot), for the owner test
                const bool opf = tid < n_own;
                if (ps < n_own) {
                    if (f32_sphere) pf4(&s_pf_i0[ps], W.thrc[cur] + g_lo + ps);
                    else pf4(&s_pf_i0[ps], W.act[cur] + g_lo + ps);
                    if (is_grp) {
                        pf4(&s_pf_i1[ps], W.act[cur] + g_lo + ps);
                        pf4(&s_pf_i2[ps], W.aoff[cur] + g_lo + ps);
                    }
                }
                const int nxs = min(na_own, kThreads);  // atoms of the slice whose x_{t-1} is staged
                if (ps < nxs) pf8(&s_pf_x[ps], xbuf(iO) + a_lo0 + ps);
                if (t > 1 && warp <= 1) {
                    // warps 0 and 1 reduce the same per-CTA maxima of |z_{t-1}| in the same order
                    T mv[kMaxG / 32];
#pragma unroll
                    for (int jj = 0; jj < kMaxG / 32; jj++) mv[jj] = lane + 32 * jj < G ? __ldcg(W.p_m + lane + 32 * jj) : T(0);
                    T mf = T(0);
#pragma unroll
                    for (int jj = 0; jj < kMaxG / 32; jj++) mf = fmax(mf, mv[jj]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) mf = fmax(mf, __shfl_xor_sync(0xffffffffu, mf, o));
                    const double m_nom = (double)mf;
                    if (warp == 1 && lane == 0) {
                        // Lemma 8 with the nominal max |z|: the dual point of the gap (a stopping rule)
                        mu_nom = (m_nom > 0.0 && fabs(s_unc) * m_nom > 1.0) ? copysign(fast_rcp(m_nom), s_unc) : s_unc;
                        R2n = fmax(fma(mu_nom, fma(mu_nom, beta, C_.m2a), yy_l2), 0.0);
                    }
                    if (warp == 0 && lane == 0) {
                        // Lemma 8 with a rigorous upper bound on max |z| given the FP rounding of z, for
                        // the screening radius (copy: |z_i - zlo_i| <= ||d_i - dlo_i|| ||theta|| + the FP32
                        // rounding of dlo_i^T theta).  Any |mu| <= 1 / max|z| gives a feasible dual point, so
                        // the clip uses 1 / m_up rounded down.
                        double mu_s = s_unc;
                        if (sizeof(T) == 8) {
                            const double m_up = m_nom + P.gamma * fmax_d * sqrt_beta;
                            if (m_up > 0.0 && fabs(s_unc) * m_up > 1.0) mu_s = copysign(fast_rcp(m_up), s_unc);
                        } else {
                            // in FP32, rounded up: m_up = m + (rounding bound per unit ||theta||) ||theta||
                            const float m_up = __fmaf_ru(lowB ? C_.gfm_lo : C_.gfm, C_.sqb_f, (float)mf);
                            if (m_up > 0.f) {
                                const float r_dn = m_up < 3.0e38f ? __frcp_rd(m_up) : 0.f;
                                if (fabsf(C_.s_unc_f) > r_dn) mu_s = (double)copysignf(r_dn, C_.s_unc_f);
                            }
                        }
                        // R^2 = ||y/lambda - mu theta||^2
                        const double R2s = fmax(fma(mu_s, fma(mu_s, beta, C_.m2a), yy_l2), 0.0);
                        R2s_last = R2s;
                        if (f32_sphere) {
                            // radius of the sphere test (DST3/DGST3: sqrt(R^2 - delta^2)), rounded up to FP32
                            const double r2 = ((P.test == 2 || P.test == 5) ? R2s - C_.delta2 : R2s) + rad2_slack;
                            s_radf = __fsqrt_ru(__double2float_ru(r2));
                        }
                        if (f32_dome) {
                            // FP32 dome: R and rho = sqrt(R^2 - psi^2) rounded up; the second branch of the
                            // dome maximum is taken only clear of its boundary t R = -psi
                            const float Rf = __fsqrt_ru(__double2float_ru(R2s));
                            const float pf = (float)psi_dome;
                            C_.dome_f[0] = Rf;
                            C_.dome_f[1] = pf;
                            C_.dome_f[2] = __fsqrt_ru(__double2float_ru(fmax(R2s - psi_dome * psi_dome, 0.0)));
                            C_.dome_f[3] = -pf + 1e-5f * (pf + Rf);
                        }
                        if (!(f32_sphere || f32_dome) || record) {
                            // radii rounded up a little: a larger radius only screens less
                            const double Rs = fast_sqrt(R2s) * (1.0 + 1e-13);
                            rad = (P.test == 2 || P.test == 5) ? fast_sqrt(fmax(R2s - delta * delta, 0.0)) * (1.0 + 1e-13) : Rs;
                            s_sc[8] = rad;
                            s_sc[9] = Rs;
                        }
                    }
                }
                // directory of the per-CTA nonzero lists (exclusive prefix of their lengths)
                int totE;
                const int exE = block_exclusive_scan(cnz, s_tmp, &totE);
                if (tid < G) s_pref[tid] = exE;
                if (tid == 0) s_pref[G] = totE;
                pf_wait();  // this thread's copies have landed; the barrier below publishes them
                const bool long_lists = __syncthreads_or(cnz > kSpec) != 0;
                const float radF = s_radf;
                const double radB = s_sc[8], RsB = s_sc[9];
                // the test of iteration t-1 on one group, from its list data (FP32 threshold or group id);
                // the owner of the group and every CTA that sums one of its atoms take the same decision
                auto killed = [&](int td) -> bool {
                    if (f32_sphere) return __int_as_float(td) > radF;
                    if (f32_dome) {
                        // max over the dome of +-d_i^T theta (dynamic Lemma 4) in FP32: the dome maximum is
                        // dc0 + R for t R <= -psi, else dc0 - psi t + rho sqrt(1 - t^2) (never above dc0 + R);
                        // the slack covers the rounding of the stored constants and of these few operations
                        const float4 dd = __ldcg(W.domef + td);
                        const float Rf = C_.dome_f[0], pf = C_.dome_f[1], rf = C_.dome_f[2], tb = C_.dome_f[3];
                        const float up = dd.y * Rf > tb ? fmaf(rf, dd.z, fmaf(-pf, dd.y, dd.x)) : dd.x + Rf;
                        const float dn = -dd.y * Rf > tb ? fmaf(rf, dd.z, fmaf(pf, dd.y, -dd.x)) : Rf - dd.x;
                        const float sl = 1e-6f * (fabsf(dd.x) + pf * fabsf(dd.y) + rf * dd.z + Rf);
                        return dd.w > up + sl && dd.w > dn + sl;
                    }
                    if (P.test == 3) {
                        // Lemma 4 (dynamic dome): max over the dome of |d_i^T theta| < 1
                        const double ni = colnorm[td];
                        const double dc0 = __ldcg(W.b + td) / (lam * ni);
                        const double tt = __ldcg(W.tv + td) / (ni * nstar);
                        const double up = dome_max(dc0, tt, psi_dome, RsB);
                        const double dn = dome_max(-dc0, -tt, psi_dome, RsB);
                        return (1.0 / ni - up > P.eps_test) && (1.0 / ni - dn > P.eps_test);
                    }
                    return __ldcg(W.thr + td) - radB > P.eps_test;
                };

                // synthesis over row tiles: w_u = D ubar, w_x = D xbar from the nonzero lists of all CTAs,
                // staged in shared memory; atoms screened by the test of iteration t-1 contribute zero
                const int E = totE;
                if (tid == 0) cols_synth += E;
                Acc pa_, pb_, pr_, pdq_;
                const int ntiles = (N + kRowTile - 1) / kRowTile;
                const int cap = P.syn_cap;
                int* const sl_col = reinterpret_cast<int*>(smem_raw);
                X* const sl_u = reinterpret_cast<X*>(smem_raw + (size_t)cap * sizeof(int));
                X* const sl_x = sl_u + cap;
                const bool one = E <= cap;
                if (one && b < ntiles) {
                    if (tid < G) {
                        const int nq = min(cnz, kSpec);
#pragma unroll
                        for (int q = 0; q < kSpec; q++) {
                            if (q < nq) {
                                const bool kq = test_now && killed(s_spec[tid].t[q]);
                                sl_col[exE + q] = s_spec[tid].col[q];
                                sl_u[exE + q] = kq ? it_zero((X*)nullptr) : s_spec[tid].u[q];
                                sl_x[exE + q] = kq ? it_zero((X*)nullptr) : s_spec[tid].x[q];
                            }
                        }
                    }
                    // the entries beyond the first kSpec of a list
                    for (int e = tid; long_lists && e < E; e += kThreads) {
                        int lo = 0, hi = G;  // largest k with s_pref[k] <= e
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (s_pref[mid] <= e) lo = mid;
                            else hi = mid;
                        }
                        const int loc = e - s_pref[lo];
                        if (loc >= kSpec) {
                            const int idx = s_alo_s[lo] + loc;
                            const bool kq = test_now && killed(__ldcg(W.nz_t + idx));
                            sl_col[e] = __ldcg(W.nz_col + idx);
                            sl_u[e] = kq ? it_zero((X*)nullptr) : ldcg_x(W.nz_u + idx);
                            sl_x[e] = kq ? it_zero((X*)nullptr) : ldcg_x(W.nz_x + idx);
                        }
                    }
                    __syncthreads();
                }
                for (int tile = b; tile < ntiles; tile += G) {
                    const int r = tile * kRowTile + lane;
                    const bool rv = r < N;
                    const T yv = (warp == 0 && rv) ? P.y[r] : T(0);
                    // compensated accumulation: theta = D u - y is a small difference of two
                    // large vectors, so the sum is carried to twice the working precision
                    typename Dot2<T>::type au, ax;
                    for (int c0 = 0; c0 < E; c0 += cap) {
                        const int ce = min(cap, E - c0);
                        if (!one) {
                            __syncthreads();
                            for (int e = tid; e < ce; e += kThreads) {
                                const int ee = c0 + e;
                                int lo = 0, hi = G;
                                while (hi - lo > 1) {
                                    const int mid = (lo + hi) >> 1;
                                    if (s_pref[mid] <= ee) lo = mid;
                                    else hi = mid;
                                }
                                const int idx = s_alo_s[lo] + (ee - s_pref[lo]);
                                const bool kq = test_now && killed(__ldcg(W.nz_t + idx));
                                sl_col[e] = __ldcg(W.nz_col + idx);
                                sl_u[e] = kq ? it_zero((X*)nullptr) : ldcg_x(W.nz_u + idx);
                                sl_x[e] = kq ? it_zero((X*)nullptr) : ldcg_x(W.nz_x + idx);
                            }
                            __syncthreads();
                        }
                        // warp w sums entries w, w + nw, w + 2 nw, ... (kSyn loads in flight a lane)
                        for (int e0 = warp; e0 < ce; e0 += nw * kSyn) {
                            T dv[kSyn];
#pragma unroll
                            for (int q = 0; q < kSyn; q++) {
                                const int e = e0 + q * nw;
                                dv[q] = (e < ce && rv) ? __ldg(P.D + (size_t)sl_col[e] * ld + r) : T(0);
                            }
#pragma unroll
                            for (int q = 0; q < kSyn; q++) {
                                const int e = e0 + q * nw;
                                if (e < ce) {
                                    syn_add(au, dv[q], sl_u[e]);
                                    syn_add(ax, dv[q], sl_x[e]);
                                }
                            }
                        }
                    }
                    acc_store(&s_red[0][warp][lane], au);
                    acc_store(&s_red[1][warp][lane], ax);
                    __syncthreads();
                    if (warp == 0) {
                        typename Dot2<T>::type wu, wx;
                        for (int k = 0; k < nw; k++) {
                            acc_merge(wu, &s_red[0][k][lane]);
                            acc_merge(wx, &s_red[1][k][lane]);
                        }
                        if (rv) {
                            // Table 1: theta_t = D ubar_{t-1} - y; Chambolle-Pock averages it with theta_{t-1}:
                            // theta_t = (theta_{t-1} + sigma_{t-1} (D ubar_{t-1} - y)) / (1 + sigma_{t-1})
                            const T th = cp ? (__ldcg(W.theta + r) + C_.cp_sig * (T)theta_from(wu, yv)) * C_.cp_inv1ps
                                            : (T)theta_from(wu, yv);
                            // adaptive steps: ||D (xbar_{t-1} - base)||^2 against the last accepted theta
                            if (SM && t > 1) acc_diff_sq(pdq_, wx, yv, __ldcg(C_.thA + r));
                            C_.thN[r] = th;
                            pa_.add(th, yv);
                            pb_.add(th, th);
                            acc_resid_sq(pr_, wx, yv);
                        }
                    }
                    __syncthreads();
                }

                // owner test of iteration t-1 on the slice's live groups: keep flags, and ||x_{t-1}||_1,
                // nonzeros and sizes of the survivors (Algorithm 3)
                int kg = 0, ka = 0, nzx = 0;
                Acc l1, sqa;
                const bool want_sq = SM == 1 || SM == 2;
                for (int base = 0; base < n_own; base += kThreads) {
                    const int k = base + tid;
                    if (k < n_own) {
                        const bool first = base == 0 && opf;
                        const int td = first ? s_pf_i0[tid]
                                             : (f32_sphere ? __float_as_int(__ldcg(W.thrc[cur] + g_lo + k))
                                                           : __ldcg(W.act[cur] + g_lo + k));
                        const bool kill = test_now && killed(td);
                        W.keep[g_lo + k] = !kill;
                        if (kill && C_.slog) {
                            // screening log: the test of iteration t-1 screened this group's atoms
                            const int gs = f32_sphere ? __ldcg(W.act[cur] + g_lo + k) : td;
                            const int i0 = is_grp ? P.goff[gs] : gs, i1 = is_grp ? P.goff[gs + 1] : gs + 1;
                            for (int i = i0; i < i1; i++) C_.slog[i] = t - 1;
                        }
                        if (want_sq && t > 1) {
                            // backtracking / SpaRSA: ||xbar_{t-1} - base||^2 over the atoms of the step
                            // (the screened ones contribute their base point: xbar is 0 there)
                            int lo_a = a_lo0 + k, sz = 1;
                            if (is_grp) {
                                const int gid = f32_sphere ? __ldcg(W.act[cur] + g_lo + k) : td;
                                lo_a = __ldcg(W.aoff[cur] + g_lo + k);
                                sz = P.goff[gid + 1] - P.goff[gid];
                            }
                            for (int q = 0; q < sz; q++) {
                                const X bq = ldcg_x(W.bS + lo_a + q);
                                acc_sq(sqa, kill ? bq : it_diff(ldcg_x(xbuf(iO) + lo_a + q), bq));
                            }
                        }
                        if (!kill) {
                            if (!is_grp) {
                                const X xv = first ? s_pf_x[tid] : ldcg_x(xbuf(iO) + a_lo0 + k);
                                acc_abs(l1, xv);
                                nzx += it_nz(xv);
                                ka += 1;
                            } else {
                                const int gid = first ? s_pf_i1[tid] : (f32_sphere ? __ldcg(W.act[cur] + g_lo + k) : td);
                                const int lo_a = first ? s_pf_i2[tid] : __ldcg(W.aoff[cur] + g_lo + k);
                                const int sz = P.goff[gid + 1] - P.goff[gid];
                                Acc gq;
                                for (int q = 0; q < sz; q++) {
                                    const int j = lo_a - a_lo0 + q;  // the atom's place in the slice
                                    const X xv = j < nxs ? s_pf_x[j] : ldcg_x(xbuf(iO) + lo_a + q);
                                    acc_sq(gq, xv);
                                    nzx += it_nz(xv);
                                }
                                acc_add_dbl(l1, P.w[gid] * sqrt(gq.value()));
                                ka += sz;
                            }
                            kg += 1;
                        }
                    }
                }
                // per-CTA totals: one warp-level reduction and a single block barrier
                const int rkg = warp_sum(kg), rka = warp_sum(ka), rnx = warp_sum(nzx);
                const Acc rl1 = acc_warp_reduce(l1);
                const Acc rsq = want_sq ? acc_warp_reduce(sqa) : sqa;
                if (warp == 0) {
                    pa_ = acc_warp_reduce(pa_);
                    pb_ = acc_warp_reduce(pb_);
                    pr_ = acc_warp_reduce(pr_);
                    if (lane == 0) { part_put(W.p_a + b, pa_); part_put(W.p_b + b, pb_); part_put(W.p_r + b, pr_); }
                    if (SM) {
                        pdq_ = acc_warp_reduce(pdq_);
                        if (lane == 0) part_put(W.p_dq + b, pdq_);
                    }
                }
                if (lane == 0) {
                    s_ired[warp] = rkg; s_tmp[warp] = rka; s_kg[warp] = rnx; acc_store(&s_red[0][warp][0], rl1);
                    if (want_sq) acc_store(&s_red[1][warp][0], rsq);
                }
                __syncthreads();
                if (tid == 0) {
                    int tkg = 0, tka = 0, tnx = 0;
                    Acc tl1, tsq;
                    for (int k = 0; k < nw; k++) {
                        tkg += s_ired[k];
                        tka += s_tmp[k];
                        tnx += s_kg[k];
                        acc_merge(tl1, &s_red[0][k][0]);
                        if (want_sq) acc_merge(tsq, &s_red[1][k][0]);
                    }
                    part_put(W.p_l1 + b, tl1);
                    if (want_sq) part_put(W.p_sq + b, tsq);
                    s_si[12] = tkg;  // kept groups of the slice: (B) skips the compaction when nothing was screened
                    W.c_ka[b] = tka;
                    W.c_nnzx[b] = tnx;
                }
            }
            ok = grid_sync(bar, G, gen);
            if (!ok) return false;

            // ======= (B) stop test, compaction of the test of t-1, correlation + prox + momentum
            {
                // the first round's keep flags, groups and thresholds (Lasso: and iterates; Group-Lasso: and
                // first atoms), fetched while warps 0 and 1 reduce the partials
                const int n0 = min(n_own, is_grp ? kThreads : P.RA);
                {
                    const int ps = (tid + kThreads - 64) % kThreads;  // issued by warps 2.. first
                    if (ps < n0) {
                        pf4(&s_pf_i0[ps], W.keep + g_lo + ps);
                        pf4(&s_pf_i1[ps], W.act[cur] + g_lo + ps);
                        if (f32_sphere) pf4(&s_pf_f0[ps], W.thrc[cur] + g_lo + ps);
                        if (is_grp) {
                            pf4(&s_pf_i2[ps], W.aoff[cur] + g_lo + ps);
                        } else {
                            pf8(&s_pf_u[ps], ubuf(iO) + a_lo0 + ps);
                            pf8(&s_pf_x[ps], xbuf(iO) + a_lo0 + ps);
                        }
                    }
                }
                if (warp >= 2) {
                    // stage theta_t in shared memory
                    constexpr int kST = kThreads - 64, kSU = 8;
                    for (int r0 = tid - 64; r0 < P.npad; r0 += kSU * kST) {
                        T v[kSU];
#pragma unroll
                        for (int q = 0; q < kSU; q++) {
                            const int r = r0 + q * kST;
                            v[q] = r < N ? __ldcg(C_.thN + r) : T(0);
                        }
#pragma unroll
                        for (int q = 0; q < kSU; q++) {
                            const int r = r0 + q * kST;
                            if (r < P.npad) th_s[r] = v[q];
                        }
                    }
                }
                if (warp == 1) {
                    // theta_t^T y and ||theta_t||^2: the parts of Lemma 8 that do not need max |z|
                    X va[kMaxG / 32], vb[kMaxG / 32];
#pragma unroll
                    for (int q = 0; q < kMaxG / 32; q++) {
                        const int k = lane + 32 * q;
                        const bool in = k < G;
                        va[q] = in ? ldcg_x(W.p_a + k) : it_zero((X*)nullptr);
                        vb[q] = in ? ldcg_x(W.p_b + k) : it_zero((X*)nullptr);
                    }
                    const double a_ = part_sum_regs<kMaxG / 32>(va);
                    const double b_ = part_sum_regs<kMaxG / 32>(vb);
                    if (lane == 0) {
                        // with an adaptive step the terms wait in S_.n_* until the step is accepted: a
                        // rejected step is redone and the test of t-1 must keep theta_{t-1}'s terms
                        const bool hold = SM != 0;
                        (hold ? S_.n_alpha : alpha) = a_;
                        (hold ? S_.n_beta : beta) = b_;
                        (hold ? S_.n_m2a : C_.m2a) = -2.0 * a_ * inv_lam;
                        // the unclipped scaling of Lemma 8 in FP32: R^2 is stationary in mu there, and any
                        // mu gives a valid sphere, so its rounding moves R^2 by a second-order amount only
                        if (sizeof(T) == 8) {
                            (hold ? S_.n_s_unc : s_unc) = b_ > 0.0 ? a_ * inv_lam * fast_rcp(b_) : 0.0;
                            (hold ? S_.n_sqrt_beta : sqrt_beta) = (double)sqrtf((float)b_) * (1.0 + 1e-6);
                        } else {
                            const float bf = (float)b_;
                            const float su = bf > 0.f ? (float)a_ * (float)inv_lam / bf : 0.f;
                            (hold ? S_.n_s_unc_f : C_.s_unc_f) = su;
                            (hold ? S_.n_s_unc : s_unc) = (double)su;
                            // an upper bound of ||theta|| is all the rounding bound of the radius needs
                            const float sq = __fmul_ru(__fsqrt_ru(bf), 1.000001f);
                            (hold ? S_.n_sqb_f : C_.sqb_f) = sq;
                            (hold ? S_.n_sqrt_beta : sqrt_beta) = (double)sq;
                        }
                    }
                }
                if (warp == 0) {
                    // FISTA coefficient of this iteration, fetched ahead of the reductions
                    const int tf_pre = t - t0;
                    const bool tab_pre = P.alg == 1 && tf_pre >= 1 && tf_pre <= P.fista_n;
                    const double bt_pre = tab_pre ? __ldg(P.fista + 2 * (tf_pre - 1)) : 0.0;
                    const double lf_pre = tab_pre ? __ldg(P.fista + 2 * (tf_pre - 1) + 1) : 0.0;
                    // every load of the per-CTA partials is issued before any is combined
                    X vr[kMaxG / 32], vl[kMaxG / 32];
                    int ia[kMaxG / 32], ix[kMaxG / 32];
#pragma unroll
                    for (int q = 0; q < kMaxG / 32; q++) {
                        const int k = lane + 32 * q;
                        const bool in = k < G;
                        vr[q] = in ? ldcg_x(W.p_r + k) : it_zero((X*)nullptr);
                        vl[q] = in ? ldcg_x(W.p_l1 + k) : it_zero((X*)nullptr);
                        ia[q] = in ? __ldcg(W.c_ka + k) : 0;
                        ix[q] = in ? __ldcg(W.c_nnzx + k) : 0;
                    }
                    const double r_ = part_sum_regs<kMaxG / 32>(vr);
                    const double l1 = part_sum_regs<kMaxG / 32>(vl);
                    double sq_ = 0.0, dq_ = 0.0;
                    if (SM) {
                        // adaptive steps: ||xbar_{t-1} - base||^2 and ||D (xbar_{t-1} - base)||^2
#pragma unroll
                        for (int q = 0; q < kMaxG / 32; q++) {
                            const int k = lane + 32 * q;
                            const bool in = k < G;
                            vr[q] = in ? ldcg_x(W.p_sq + k) : it_zero((X*)nullptr);
                            vl[q] = in ? ldcg_x(W.p_dq + k) : it_zero((X*)nullptr);
                        }
                        sq_ = part_sum_regs<kMaxG / 32>(vr);
                        dq_ = part_sum_regs<kMaxG / 32>(vl);
                    }
                    int na = 0, nx = 0;
#pragma unroll
                    for (int q = 0; q < kMaxG / 32; q++) { na += ia[q]; nx += ix[q]; }
                    na = warp_sum(na);
                    nx = warp_sum(nx);
                    if (lane == 0) {
                        int stop = 0, retry = 0;
                        if (SM) {
                            // the step that produced x_{t-1} (backtracking, SpaRSA, TwIST): its acceptance
                            // test at xbar_{t-1}; a rejected step is redone with a larger L (alpha) or, for
                            // TwIST, as the plain shrinkage step, before anything else of this phase
                            const double Fcur = fma(lam, l1, 0.5 * r_);  // F(xbar_{t-1}) (t = 1: F(x_0))
                            if (t == 1) {
                                S_.Fh[0] = Fcur;
                                S_.nh = 1;
                                S_.hpos = 1;
                                S_.Fprev = Fcur;
                            } else {
                                bool acc_ok;
                                if (SM == 1) {
                                    // Beck-Teboulle's upper model of the quadratic loss, with a slack for the
                                    // rounding of D xbar - y and of the accepted theta
                                    const double u = sizeof(T) == 4 ? 0x1p-24 : 0x1p-53;
                                    acc_ok = dq_ <= S_.Lstep * sq_ + 16.0 * u * u * (beta + r_);
                                } else if (SM == 2) {
                                    double Fmax = S_.Fh[0];
                                    for (int q = 1; q < S_.nh; q++) Fmax = fmax(Fmax, S_.Fh[q]);
                                    acc_ok = Fcur <= Fmax - 0.5 * kSparsaSigma * S_.Lstep * sq_;
                                } else {
                                    acc_ok = S_.fallback || t == 2 || Fcur <= S_.Fprev;
                                }
                                if (!acc_ok && S_.tries < kRetryCap) {
                                    retry = 1;
                                    S_.tries++;
                                    if (SM == 3) S_.fallback = 1;
                                    else S_.Lstep *= 2.0;
                                } else {
                                    S_.tries = 0;
                                    S_.fallback = 0;
                                    if (SM == 2 && sq_ > 0.0)  // Barzilai-Borwein: ||D s||^2 / ||s||^2
                                        S_.Lstep = fmin(fmax(dq_ / sq_, 1e-10 * P.L), 1e10 * P.L);
                                    S_.Fh[S_.hpos] = Fcur;
                                    S_.hpos = (S_.hpos + 1) % 5;
                                    if (S_.nh < 5) S_.nh++;
                                    S_.Fprev = Fcur;
                                }
                            }
                            // the step constant of the step taken next (or redone)
                            const double Ls = SM == 3 ? P.L : S_.Lstep;
                            C_.invL = (T)(1.0 / Ls);
                            C_.thrL = lam / Ls;
                            C_.thrX = it_cast(lam / Ls, (X*)nullptr);
                        }
                        if (t > 1 && !retry) {
                            // P(xbar) - Dual(mu theta), Dual(v) = 1/2||y||^2 - lambda^2/2 ||v - y/lambda||^2
                            primal = fma(lam, l1, 0.5 * r_);
                            gap = fma(C_.hlam2, R2n, primal - C_.hyy);
                            iters = t - 1;
                            if (low) {
                                // the nominal gap rests on the copy's correlations: stop only on the
                                // rigorous one (dual point scaled with the bounded max), and switch to the
                                // FP32 master once the bulk phase reaches its tolerance or stalls
                                const double gap_safe = fma(C_.hlam2, R2s_last, primal - C_.hyy);
                                if (gap < 0.99 * best_gap) {
                                    best_gap = gap;
                                    since_best = 0;
                                } else {
                                    since_best++;
                                }
                                if (!(P.tol > 0.0 && gap_safe <= P.tol * 0.5 * yy) &&
                                    (gap <= P.lo_switch * 0.5 * yy || since_best >= 25)) {
                                    // FP32 polish: a fresh FISTA sequence warm-started at the bulk iterate
                                    low = 0;
                                    t0 = t - 1;
                                    lf = 1.0;
                                }
                                gap = gap_safe;
                            }
                            if (record && b == 0 && t - 1 <= P.hist_rows) {
                                double* h = P.hist + (size_t)(t - 2) * 6;
                                h[0] = (double)na; h[1] = (double)nx; h[2] = sqrt(R2n); h[3] = rad; h[4] = gap; h[5] = mu_nom;
                            }
                            stop = (P.tol > 0.0 && gap <= C_.tol_abs && (t - 1) % P.gap_every == 0) || (t - 1 >= P.max_iter);
                            // an owner shutting down (the server) may end the solve early, every 16 iterations
                            if (P.abort_flag && (t & 15) == 0 && *P.abort_flag) stop = 1;
                        }
                        double bt = 0.0;
                        if (retry) {
                            bt = S_.bt_att;  // the redone step keeps its FISTA coefficient
                        } else if (cp) {
                            // Chambolle-Pock: x_t = prox_{lambda tau_{t-1}}(x_{t-1} - tau_{t-1} z), then
                            // phi_t = 1 / sqrt(1 + 2 gamma tau_{t-1}), tau_t = phi_t tau_{t-1},
                            // sigma_t = sigma_{t-1} / phi_t, ubar_t = x_t + phi_t (x_t - x_{t-1})
                            const double tau = S_.cp_tau;
                            C_.invL = (T)tau;
                            C_.thrL = lam * tau;
                            C_.thrX = it_cast(lam * tau, (X*)nullptr);
                            const double phi = P.cp_gamma > 0.0 ? 1.0 / sqrt(1.0 + 2.0 * P.cp_gamma * tau) : 1.0;
                            S_.cp_tau = phi * tau;
                            S_.cp_sigma /= phi;
                            C_.cp_sig = (T)S_.cp_sigma;
                            C_.cp_inv1ps = (T)(1.0 / (1.0 + S_.cp_sigma));
                            bt = phi;
                        } else if (fista) {
                            // FISTA: l_t = (1 + sqrt(1 + 4 l_{t-1}^2)) / 2, coefficient (l_{t-1} - 1) / l_t,
                            // read from the table (the sequence depends on t only)
                            const int tf = t - t0;  // index in the current FISTA sequence
                            if (tf == tf_pre && tab_pre) {
                                bt = bt_pre;
                                lf = lf_pre;
                            } else if (tf <= P.fista_n) {
                                bt = P.fista[2 * (tf - 1)];
                                lf = P.fista[2 * (tf - 1) + 1];
                            } else {
                                const double ln = 0.5 * (1.0 + sqrt(1.0 + 4.0 * lf * lf));
                                bt = (lf - 1.0) / ln;
                                lf = ln;
                            }
                        }
                        s_sc[10] = bt;
                        S_.bt_att = bt;
                        if (sizeof(T) == 4) {
                            const FF bf2 = ff_from_double(bt);
                            C_.bt_h = bf2.h;
                            C_.bt_l = bf2.l;
                        }
                        s_si[4] = na; s_si[5] = nx; s_si[6] = stop;
                        s_si[9] = low;
                        s_si[13] = retry;
                    }
                }
                pf_wait();  // this thread's copies have landed; the barrier below publishes them
                __syncthreads();
                lowB = s_si[9] != 0;
                if (s_si[6]) break;
                X btX;
                if constexpr (sizeof(T) == 4) btX = FF{C_.bt_h, C_.bt_l};
                else btX = s_sc[10];
                if (ADAPT && s_si[13]) {
                    // ---- (B') the step that produced x_{t-1} failed its acceptance test: redo it from the same
                    // base point and correlations with the new step constant (TwIST: as the plain shrinkage
                    // step), at the same positions; atoms screened by the test of t-1 stay out of the lists
                    X* const xR = xbuf(iO);
                    X* const uR = ubuf(iO);
                    int nz_base = 0;
                    for (int base = 0; base < n_own; base += kThreads) {
                        const int k = base + tid;
                        int cnt = 0, gid = 0, lo_a = 0, sz = 0, td = 0;
                        if (k < n_own && __ldcg(W.keep + g_lo + k)) {
                            gid = __ldcg(W.act[cur] + g_lo + k);
                            lo_a = is_grp ? __ldcg(W.aoff[cur] + g_lo + k) : a_lo0 + k;
                            sz = is_grp ? P.goff[gid + 1] - P.goff[gid] : 1;
                            td = f32_sphere ? __float_as_int(__ldcg(W.thrc[cur] + g_lo + k)) : gid;
                            X f = it_from(T(1), (X*)nullptr);
                            if (is_grp) {
                                // group soft threshold: max(0, (||v_g|| - t w_g) / ||v_g||) v_g
                                Acc vq;
                                for (int q = 0; q < sz; q++)
                                    acc_sq(vq, it_grad_step(ldcg_x(W.bS + lo_a + q), __ldcg(W.zS + lo_a + q), invL));
                                const double nv = sqrt(vq.value());
                                f = it_cast(nv > 0.0 ? fmax(0.0, (nv - thrL * P.w[gid]) / nv) : 0.0, (X*)nullptr);
                            }
                            for (int q = 0; q < sz; q++) {
                                const X v = it_grad_step(ldcg_x(W.bS + lo_a + q), __ldcg(W.zS + lo_a + q), invL);
                                const X xv = is_grp ? it_scale(v, f) : it_soft(v, thrX);
                                const X pq = ldcg_x(W.pS + lo_a + q);
                                const X uv = SM == 3 ? pq : (fista ? it_momentum(xv, pq, btX) : xv);
                                xR[lo_a + q] = xv;
                                uR[lo_a + q] = uv;
                                cnt += (it_nz(xv) || (SM < 2 && it_nz(uv))) ? 1 : 0;
                            }
                        }
                        int totc;
                        const int pc = block_exclusive_scan(cnt, s_tmp, &totc);
                        if (cnt) {
                            const int c0 = is_grp ? P.goff[gid] : gid;
                            int e = a_lo0 + nz_base + pc;
                            for (int q = 0; q < sz; q++) {
                                const X xv = xR[lo_a + q];
                                const X uv = SM >= 2 ? xv : uR[lo_a + q];
                                if (it_nz(xv) || it_nz(uv)) {
                                    W.nz_col[e] = c0 + q;
                                    W.nz_u[e] = uv;
                                    W.nz_x[e] = xv;
                                    W.nz_t[e] = td;
                                    e++;
                                }
                            }
                        }
                        nz_base += totc;
                    }
                    if (tid == 0) W.c_nz[b] = nz_base;
                    ok = grid_sync(bar, G, gen);
                    if (!ok) return false;
                    t--;  // the same iteration again: the test of t-1 and the synthesis of the redone step
                    continue;
                }
                if (tid == 0) {
                    cols_corr += s_si[4];
                    if (lowB) cols_lowp += s_si[4];
                    if (SM) {
                        // the step was accepted: theta_t's Lemma 8 terms take effect, theta_t is the accepted theta
                        alpha = S_.n_alpha;
                        beta = S_.n_beta;
                        C_.m2a = S_.n_m2a;
                        s_unc = S_.n_s_unc;
                        sqrt_beta = S_.n_sqrt_beta;
                        C_.s_unc_f = S_.n_s_unc_f;
                        C_.sqb_f = S_.n_sqb_f;
                        T* const th = C_.thA;
                        C_.thA = C_.thN;
                        C_.thN = th;
                    }
                }

                // rounds of the slice's live groups (whole groups, at most RA atoms): the survivors of
                // the test of t-1 move to their compacted positions (list nxt, iterate buffers iO ^ 1),
                // z = D_A^T theta_t, x_t = prox(u_{t-1} - z / L), u_t = FISTA extrapolation, nonzero list
                const int nxt = cur ^ 1, iW = iO ^ 1;
                X* const xW = xbuf(iW);
                X* const uW = ubuf(iW);
                const X* const xO = xbuf(iO);
                const X* const uO = ubuf(iO);
                int* const opos_s = cols_s + P.RA;
                // Group-Lasso: the round's old iterates u and x, staged in shared memory (and the steps after them)
                X* const rs_u = reinterpret_cast<X*>((reinterpret_cast<uintptr_t>(opos_s + P.RA) + 7) & ~uintptr_t(7));
                X* const rs_x = rs_u + P.RA;
                // Lasso slice in which the last test screened nothing: positions stay, no list copy
                const bool same = !is_grp && s_si[12] == n_own;
                T mloc = T(0);
                int kg_run = 0, ka_run = 0, nz_base = 0;
                int k0 = 0;
                while (k0 < n_own) {
                    const int k = k0 + tid;  // one old live group per thread
                    int sz = 0, gid = 0, kp = 0, lo_o = 0;
                    float thf = 0.f;
                    if (!is_grp) {
                        if (k < n_own && tid < P.RA) {
                            sz = 1;
                            const bool first = k0 == 0;
                            kp = first ? s_pf_i0[tid] : __ldcg(W.keep + g_lo + k);
                            gid = first ? s_pf_i1[tid] : __ldcg(W.act[cur] + g_lo + k);
                            thf = f32_sphere ? (first ? s_pf_f0[tid] : __ldcg(W.thrc[cur] + g_lo + k)) : 0.f;
                            lo_o = a_lo0 + k;
                        }
                    } else if (k < n_own) {
                        const bool first = k0 == 0;  // k < n0: prefetched
                        kp = first ? s_pf_i0[tid] : __ldcg(W.keep + g_lo + k);
                        gid = first ? s_pf_i1[tid] : __ldcg(W.act[cur] + g_lo + k);
                        if (f32_sphere) thf = first ? s_pf_f0[tid] : __ldcg(W.thrc[cur] + g_lo + k);
                        lo_o = first ? s_pf_i2[tid] : __ldcg(W.aoff[cur] + g_lo + k);
                        sz = P.goff[gid + 1] - P.goff[gid];
                    }
                    int k1;
                    if (!is_grp) {
                        k1 = min(n_own, k0 + P.RA);
                    } else {
                        // whole groups while the atoms fit in RA
                        int tot_sz;
                        const int ex_sz = block_exclusive_scan(sz, s_tmp, &tot_sz);
                        const int in_round = (k < n_own && ex_sz + sz <= P.RA) ? 1 : 0;
                        k1 = k0 + __syncthreads_count(in_round);
                        if (k >= k1) { kp = 0; sz = 0; }
                    }
                    const int kept = (kp && k < k1) ? 1 : 0;
                    int r_a, natoms, ngr;  // first atom of the group within the round; round totals
                    if (same) {
                        r_a = tid;
                        natoms = ngr = k1 - k0;
                        if (kept) {
                            cols_s[r_a] = gid;
                            opos_s[r_a] = lo_o;
                        }
                    } else {
                        int tot;
                        const int pre = block_exclusive_scan(kept ? ((1 << 16) | sz) : 0, s_tmp, &tot);
                        r_a = pre & 0xffff;
                        natoms = tot & 0xffff;
                        ngr = tot >> 16;
                        if (kept) {
                            const int ng = kg_run + (pre >> 16);
                            W.act[nxt][g_lo + ng] = gid;
                            if (is_grp) W.aoff[nxt][g_lo + ng] = a_lo0 + ka_run + r_a;
                            if (f32_sphere) W.thrc[nxt][g_lo + ng] = thf;
                            const int c0 = is_grp ? P.goff[gid] : gid;
                            for (int q = 0; q < sz; q++) {
                                cols_s[r_a + q] = c0 + q;
                                opos_s[r_a + q] = lo_o + q;
                            }
                        }
                    }
                    __syncthreads();
                    if (is_grp) {
                        // the round's old iterates, fetched into shared memory while the correlation runs: the
                        // owner of a group then reads its atoms there instead of one L2 trip after another
                        for (int r = tid; r < natoms; r += kThreads) {
                            pf8(&rs_u[r], uO + opos_s[r]);
                            pf8(&rs_x[r], xO + opos_s[r]);
                        }
                    }
                    // z = D_A^T theta_t: items (atom, row chunk)
                    const int nchunk = P.nchunk;
                    if constexpr (sizeof(T) == 4) {
                        if (lowB && P.lo_kind == 1)
                            gemv_lowp<1, 4>(P.Dlo, P.ld_lo, P.lo_scale, reinterpret_cast<const float*>(th_s),
                                            reinterpret_cast<float*>(zpart), cols_s, natoms, nchunk, lane, warp, nw);
                        else if (lowB)
                            gemv_lowp<2, 8>(P.Dlo, P.ld_lo, P.lo_scale, reinterpret_cast<const float*>(th_s),
                                            reinterpret_cast<float*>(zpart), cols_s, natoms, nchunk, lane, warp, nw);
                        else
                            gemv_f32<4>(P.D, ld, th_s, zpart, cols_s, natoms, nchunk, lane, warp, nw);
                    } else {
                        const V* thv = reinterpret_cast<const V*>(th_s);
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
                            for (int q = 0; q < kU; q++) {
                                const int v0 = c0 * (32 * kU) + q * 32 + lane;
                                const int v1 = c1 * (32 * kU) + q * 32 + lane;
                                d0[q] = v0 < ldv ? __ldg(col0 + v0) : v4zero((V*)nullptr);
                                d1[q] = (h1 && v1 < ldv) ? __ldg(col1 + v1) : v4zero((V*)nullptr);
                            }
                            T s0 = T(0), s1 = T(0);
#pragma unroll
                            for (int q = 0; q < kU; q++) {
                                s0 = vdot(d0[q], thv[c0 * (32 * kU) + q * 32 + lane], s0);
                                s1 = vdot(d1[q], thv[c1 * (32 * kU) + q * 32 + lane], s1);
                            }
                            s0 = warp_sum(s0);
                            s1 = warp_sum(s1);
                            if (lane == 0) {
                                zpart[a0 * nchunk + c0] = s0;
                                if (h1) zpart[a1 * nchunk + c1] = s1;
                            }
                        }
                    }
                    if (is_grp) pf_wait();  // this thread's staged iterates; the barrier publishes them
                    __syncthreads();
                    int totc;  // entries of this round in the nonzero list of (u_t, x_t)
                    if (!is_grp) {
                        // proximal step (Table 1), x_t = prox_{lambda/L Omega}(u_{t-1} - z / L), and the FISTA
                        // extrapolation u_t = x_t + bt (x_t - x_{t-1}), by the thread that owns the atom
                        int cnt = 0;
                        X lx = it_zero((X*)nullptr), lu = lx;  // x_t, u_t of the thread's atom, for the list
                        if (kept) {
                            const int an = a_lo0 + ka_run + r_a;  // new position of the atom
                            T z = T(0);
                            for (int c = 0; c < nchunk; c++) z += zpart[r_a * nchunk + c];
                            const bool first = k0 == 0;
                            const X uo = first ? s_pf_u[tid] : ldcg_x(uO + lo_o);
                            const X xo = first ? s_pf_x[tid] : ldcg_x(xO + lo_o);
                            // gradient step from ubar_{t-1} (ISTA, FISTA) or x_{t-1} (CP, SpaRSA, TwIST)
                            const X bpt = (cp || SM >= 2) ? xo : uo;
                            X xv = it_soft(it_grad_step(bpt, z, invL), thrX);
                            // TwIST after its first step: (1 - a) x_{t-2} + (a - b) x_{t-1} + b prox(...), with
                            // x_{t-2} kept in the u buffer
                            if (SM == 3 && t > 1) xv = it_twist(uo, xo, xv, P.tw_a, P.tw_b);
                            const X uv = SM == 3 ? xo : (ista ? xv : it_momentum(xv, xo, btX));
                            xW[an] = xv;
                            uW[an] = uv;
                            lx = xv;
                            lu = uv;
                            if (SM) {
                                // what a redone step needs: z_t, the base point and x_{t-1}
                                W.zS[an] = z;
                                W.bS[an] = bpt;
                                W.pS[an] = xo;
                            }
                            mloc = fmax(mloc, fabs(z));
                            cnt = (it_nz(SM >= 2 ? xv : uv) || it_nz(xv)) ? 1 : 0;
                        }
                        // nonzero list of (u_t, x_t), with the atom's test data
                        const int pc = block_exclusive_scan(cnt, s_tmp, &totc);
                        if (cnt) {
                            const int e = a_lo0 + nz_base + pc;
                            W.nz_col[e] = gid;
                            W.nz_u[e] = SM >= 2 ? lx : lu;
                            W.nz_x[e] = lx;
                            W.nz_t[e] = f32_sphere ? __float_as_int(thf) : gid;
                        }
                    } else {
                        // Group-Lasso prox (Table 1, group soft threshold) in three steps over the round's atoms,
                        // which sit at 0 .. natoms-1 group after group: (1) thread r: z_r and the gradient step
                        // v_r of atom r; (2) the owner of a group: ||v_g||, the group's threshold factor and
                        // ||z_g|| / w_g; (3) thread r: x_t, u_t and the nonzero-list entry of atom r
                        X* const rs_f = rs_x + P.RA;  // per atom: v_r, then its group's factor
                        const int r = tid;
                        const bool ra_in = r < natoms;
                        T z_r = T(0);
                        X v_r = it_zero((X*)nullptr), xo = v_r, uo = v_r;
                        if (ra_in) {
                            for (int c = 0; c < nchunk; c++) z_r += zpart[r * nchunk + c];
                            xo = rs_x[r];
                            uo = rs_u[r];
                            // gradient step from ubar_{t-1} (ISTA, FISTA) or x_{t-1} (CP, SpaRSA, TwIST)
                            v_r = it_grad_step((cp || SM >= 2) ? xo : uo, z_r, invL);
                            zpart[r * nchunk] = z_r;
                            rs_f[r] = v_r;
                        }
                        __syncthreads();
                        if (kept) {
                            Acc zq, vq;
                            for (int q = 0; q < sz; q++) {
                                const T z = zpart[(r_a + q) * nchunk];
                                zq.add(z, z);
                                acc_sq(vq, rs_f[r_a + q]);
                            }
                            const double wg = P.w[gid];
                            const double nv = fast_sqrt(vq.value());
                            // group soft threshold: max(0, (||v_g|| - t w_g) / ||v_g||) v_g
                            const X f = it_cast(nv > 0.0 ? fmax(0.0, (nv - thrL * wg) * fast_rcp(nv)) : 0.0, (X*)nullptr);
                            const int td = f32_sphere ? __float_as_int(thf) : gid;
                            for (int q = 0; q < sz; q++) {
                                rs_f[r_a + q] = f;
                                opos_s[r_a + q] = td;  // the group's test data, for the list (positions are read)
                            }
                            mloc = fmax(mloc, group_zmax(zq, wg));
                        }
                        __syncthreads();
                        int nzf = 0;
                        X xv = v_r, uv = v_r;
                        if (ra_in) {
                            const int an = a_lo0 + ka_run + r;  // new position of atom r
                            xv = it_scale(v_r, rs_f[r]);
                            // TwIST after its first step: (1 - a) x_{t-2} + (a - b) x_{t-1} + b prox(...), with
                            // x_{t-2} kept in the u buffer
                            if (SM == 3 && t > 1) xv = it_twist(uo, xo, xv, P.tw_a, P.tw_b);
                            uv = SM == 3 ? xo : (ista ? xv : it_momentum(xv, xo, btX));
                            xW[an] = xv;
                            uW[an] = uv;
                            if (SM) {
                                // what a redone step needs: z_t, the base point and x_{t-1}
                                W.zS[an] = z_r;
                                W.bS[an] = (cp || SM >= 2) ? xo : uo;
                                W.pS[an] = xo;
                            }
                            nzf = (it_nz(SM >= 2 ? xv : uv) || it_nz(xv)) ? 1 : 0;
                        }
                        // nonzero list: one entry per nonzero atom, in atom order (the groups' order)
                        const int pc = block_exclusive_scan(nzf, s_tmp, &totc);
                        if (nzf) {
                            const int e = a_lo0 + nz_base + pc;
                            W.nz_col[e] = cols_s[r];
                            W.nz_u[e] = SM >= 2 ? xv : uv;
                            W.nz_x[e] = xv;
                            W.nz_t[e] = opos_s[r];
                        }
                    }
                    kg_run += ngr;
                    ka_run += natoms;
                    nz_base += totc;
                    k0 = k1;
                }
                n_own = kg_run;
                na_own = ka_run;
                if (!same) cur = nxt;
                iO = iW;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mloc = fmax(mloc, __shfl_xor_sync(0xffffffffu, mloc, o));
                T* const s_mw = reinterpret_cast<T*>(s_dred);  // per-warp maxima, in the type of z
                if (lane == 0) s_mw[warp] = mloc;
                __syncthreads();
                if (tid == 0) {
                    T m = T(0);
                    for (int k = 0; k < nw; k++) m = fmax(m, s_mw[k]);
                    W.p_m[b] = m;
                    W.c_nz[b] = nz_base;
                }
            }
            ok = grid_sync(bar, G, gen);
            if (!ok) return false;
        }

        // ------------------------------------------------------------ output
        // x_{t-1} restricted to the survivors of the test of iteration t-1 (Algorithm 3), zero elsewhere
        for (int i = a_lo0 + tid; i < a_hi0; i += kThreads) xout[i] = T(0);
        __syncthreads();
        for (int k = tid; k < n_own; k += kThreads) {
            if (!__ldcg(W.keep + g_lo + k)) continue;
            const int gid = __ldcg(W.act[cur] + g_lo + k);
            const int lo_a = is_grp ? __ldcg(W.aoff[cur] + g_lo + k) : a_lo0 + k;
            const int c0 = is_grp ? P.goff[gid] : gid;
            const int sz = is_grp ? P.goff[gid + 1] - P.goff[gid] : 1;
            for (int q = 0; q < sz; q++) xout[c0 + q] = (T)it_round(ldcg_x(xbuf(iO) + lo_a + q));
        }
        if (b == 0 && tid == 0) {
            R->iters = iters;
            R->status = (P.tol > 0.0 && !(gap <= P.tol * 0.5 * yy)) ? kDevNotConverged : kDevOk;
            R->n_active = s_si[4];  // active atoms and nonzeros of the returned iterate
            R->nnz = s_si[5];
            R->gap = gap;
            R->primal = primal;
            R->dual = primal - gap;
            R->lambda = lam;
            R->lambda_max = lstar;
            R->cols_corr = cols_corr;
            R->cols_synth = cols_synth;
            R->cols_lowp = cols_lowp;
        }
        __syncthreads();
    }
    return true;
}

// ------------------------------------------------------------ host helpers

// Launch geometry of a solve: GEMV row chunks, padded N, atoms per round, grid, shared memory.
struct Geometry {
    int nchunk, npad, RA, G;
    size_t smem;
};

template <typename T>
inline ds_status geometry(const DictDesc& dd, int num_sms, size_t smem_optin, Geometry* g)
{
    using X = typename IterT<T>::type;
    constexpr int EV = 16 / sizeof(T);
    const int chunk = 32 * EV * kU;
    g->nchunk = (dd.N + chunk - 1) / chunk;
    g->npad = g->nchunk * chunk;
    g->G = std::min(num_sms, kMaxG);  // one CTA per SM, within the fixed-size reductions
    // shared memory: theta, then per atom of a round its z chunks, column and old position (Group-Lasso
    // also its old iterates u and x and its step v, 8-byte aligned), and room for n (hi/lo) in the precompute
    const size_t fixed = g->npad * sizeof(T) + 8;
    const size_t per_atom = g->nchunk * sizeof(T) + 8 + (dd.is_group ? 3 * sizeof(X) : 0);
    const size_t budget = smem_optin > 48 * 1024 ? smem_optin - 40 * 1024 : 48 * 1024;
    if (fixed + 64 * per_atom > budget) return DS_ERR_UNSUPPORTED;
    g->RA = (int)std::min<size_t>(512, (budget - fixed) / per_atom);
    if (dd.is_group && g->RA < dd.max_gsize) return DS_ERR_UNSUPPORTED;
    g->smem = std::max(fixed + (size_t)g->RA * per_atom, (size_t)g->npad * 8);
    if (g->smem > budget) return DS_ERR_UNSUPPORTED;
    return DS_OK;
}

// Carves the solve workspace out of `base` (nullptr: only measures it).
template <typename T>
inline size_t layout(char* base, const DictDesc& dd, const Geometry& g, int n_lambda, Ws<T>* w, double** lam_dev,
              DevResult** res_dev, double** colnorm_w)
{
    using X = typename IterT<T>::type;
    const int N = dd.N, K = dd.K, nG = dd.nG, G = g.G;
    Bump bp{base, 0};
    w->bar = bp.take<GridBarrier>(1);
    w->theta = bp.take<T>(g.npad);
    w->b = bp.take<double>(K);
    w->tv = bp.take<double>(K);
    w->thr = bp.take<double>(nG);
    w->nvec = bp.take<double>(N);
    for (int k = 0; k < 2; k++) {
        w->act[k] = bp.take<int>(nG);
        w->aoff[k] = bp.take<int>(nG + 1);
        w->thrc[k] = bp.take<float>(nG);
        w->xc[k] = bp.take<X>(K);
        w->uc[k] = bp.take<X>(K);
    }
    w->keep = bp.take<int>(nG);
    w->domef = bp.take<float4>(dd.is_group ? 0 : K);
    w->nz_col = bp.take<int>(K);
    w->nz_u = bp.take<X>(K);
    w->nz_x = bp.take<X>(K);
    w->nz_t = bp.take<int>(K);
    w->c_ka = bp.take<int>(G);
    w->c_nz = bp.take<int>(G);
    w->c_nnzx = bp.take<int>(G);
    w->p_m = bp.take<T>(G);
    w->p_l1 = bp.take<X>(G);
    w->p_a = bp.take<X>(G);
    w->p_b = bp.take<X>(G);
    w->p_r = bp.take<X>(G);
    w->p_v = bp.take<double>(G);
    w->p_i = bp.take<int>(G);
    w->p_cn = bp.take<double>(G);
    w->theta2 = bp.take<T>(g.npad);
    w->zS = bp.take<T>(K);
    w->bS = bp.take<X>(K);
    w->pS = bp.take<X>(K);
    w->p_sq = bp.take<X>(G);
    w->p_dq = bp.take<X>(G);
    *lam_dev = bp.take<double>(std::max(n_lambda, 1));
    *res_dev = bp.take<DevResult>(std::max(n_lambda, 1));
    *colnorm_w = dd.norms_in_kernel ? bp.take<double>(K) : nullptr;
    return bp.off + 256;
}


// Dictionary, options and geometry fields of a solve's parameters (the caller
// sets the problem data: y, x0, lambdas, outputs, workspace).
template <typename T>
inline void fill_params(SolveP<T>& P, const DictDesc& dd, const Geometry& g, const ds_options* opt)
{
    constexpr int EV = 16 / sizeof(T);
    P.D = reinterpret_cast<const T*>(dd.D);
    P.N = dd.N; P.K = dd.K; P.ld = dd.ld; P.nG = dd.nG; P.is_group = dd.is_group;
    P.goff = dd.goff; P.w = dd.w; P.spec = dd.spec; P.colnorm = dd.colnorm;
    P.fmax = dd.fmax;
    P.Dff = sizeof(T) == 8 ? dd.Dff : nullptr;
    P.lam0 = 0.0;
    {
        // worst-case rounding of the FP GEMV: each product goes through at most
        // kU*EV FMAs in a lane, 5 shuffle additions and nchunk chunk additions
        const double u = sizeof(T) == 4 ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53);
        const double k = kU * EV + 5 + g.nchunk;
        P.gamma = 1.01 * k * u / (1.0 - k * u);
    }
    P.eps_test = sizeof(T) == 4 ? 1e-9 : 1e-11;
    P.lambda_rel = opt ? opt->lambda_rel : 0;
    P.alg = opt ? opt->alg : 1;
    P.test = opt ? opt->test : 0;
    P.dynamic = opt ? opt->dynamic : 1;
    P.warm_start = opt ? opt->warm_start : 0;
    P.max_iter = opt ? opt->max_iter : 1;
    P.tol = opt ? opt->tol_gap_rel : 0.0;
    P.L = (opt && opt->L > 0) ? opt->L : dd.L;
    // Chambolle-Pock steps: tau_0 sigma_0 ||D||^2 < 1 by default (0.99 / sqrt(L) each)
    P.cp_tau0 = (opt && opt->cp_tau > 0.0) ? opt->cp_tau : 0.99 / std::sqrt(P.L);
    P.cp_sigma0 = (opt && opt->cp_sigma > 0.0) ? opt->cp_sigma : 0.99 / std::sqrt(P.L);
    P.cp_gamma = (opt && opt->cp_gamma > 0.0) ? opt->cp_gamma : 0.0;
    P.step_mode = 0;
    if (opt && opt->alg == DS_SPARSA) P.step_mode = 2;
    else if (opt && opt->alg == DS_TWIST) P.step_mode = 3;
    else if (opt && opt->step_backtracking && (opt->alg == DS_ISTA || opt->alg == DS_FISTA)) P.step_mode = 1;
    P.bt_L0 = (opt && opt->bt_L0 > 0.0) ? opt->bt_L0 : 1.0;
    {
        // TwIST (Bioucas-Dias, Figueiredo): alpha = rho^2 + 1, beta = 2 alpha / (xi_1 + xi_m) with
        // rho = (1 - sqrt(k)) / (1 + sqrt(k)), k = xi_1 / xi_m, for the eigenvalues of D^T D / L in [xi_1, 1]
        const double xi1 = (opt && opt->twist_xi1 > 0.0) ? opt->twist_xi1 : 1e-4;
        const double rho = (1.0 - std::sqrt(xi1)) / (1.0 + std::sqrt(xi1));
        P.tw_a = rho * rho + 1.0;
        P.tw_b = 2.0 * P.tw_a / (1.0 + xi1);
    }
    P.gap_every = (opt && opt->gap_every > 1) ? opt->gap_every : 1;
    P.RA = g.RA;
    P.nchunk = g.nchunk;
    P.npad = g.npad;
    P.syn_cap = (int)(g.smem / (sizeof(int) + 2 * sizeof(typename IterT<T>::type))) & ~15;
    P.hist = nullptr;
    P.hist_rows = 0;
    P.scr_log = nullptr;
    P.scr_rows = 0;
    P.x0 = nullptr;
    P.colnorm_w = nullptr;
    P.fista = nullptr;
    P.fista_n = 0;
    P.abort_flag = nullptr;
    P.Dlo = dd.Dlo;
    P.lo_kind = sizeof(T) == 4 ? dd.lo_kind : 0;
    P.ld_lo = dd.ld_lo;
    P.lo_scale = dd.lo_scale;
    P.emax = dd.emax;
    {
        // rounding of the copy's FP32 accumulation: 16 FMAs a lane, 5 shuffles, the chunks, the FP8 scale
        const double u = std::ldexp(1.0, -24);
        const double k = 16 + 5 + g.nchunk + 1;
        P.gamma_lo = 1.01 * k * u / (1.0 - k * u);
    }
    // default: leave the copy once the nominal gap is below 1e-3 (or the tolerance, if coarser); the
    // FP32 iterations restart FISTA from there, which also acts as a restart of the momentum
    P.lo_switch = (opt && opt->lowp_switch > 0.0) ? opt->lowp_switch
                                                   : std::max(1e-3, (opt && opt->tol_gap_rel > 0.0) ? opt->tol_gap_rel : 0.0);
}

}  // namespace ds
