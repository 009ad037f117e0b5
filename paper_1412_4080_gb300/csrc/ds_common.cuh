// ds_common.cuh -- device helpers shared by the dscreen kernels: the bounded
// grid barrier of the persistent cooperative kernels, compensated dot-product
// accumulation, fixed-order reductions and vector load helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ds {

constexpr int kWarp = 32;

// ----------------------------------------------------------- grid barrier
//
// Barrier for a cooperative grid (all CTAs co-resident) on a monotonic
// counter: the k-th barrier of a launch waits until the counter reaches
// k * gridDim.x.  Arrival is one release-ordered atomic add; waiting is an
// acquire-ordered poll with an iteration limit.  A wait that exceeds the limit
// sets `err` and returns false; every CTA then leaves its loop, so a lost CTA
// can never hang the GPU.  The counter is zeroed before each launch.
struct GridBarrier {
    unsigned int count;
    unsigned int gen;  // unused by the counter barrier, kept for layout
    unsigned int err;
    unsigned int pad;
};

constexpr unsigned long long kSpinLimit = 1ull << 25;  // backstop on the number of polls
constexpr unsigned long long kWaitNs = 2000000000ull;  // a barrier wait gives up after 2 s

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned int* p, unsigned int v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

// Returns true when every CTA arrived; false when the barrier (now or earlier)
// failed or the wait exceeded limit_ns.  `target` is the CTA's private running
// target (advanced by gridDim.x).
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned int nblocks, unsigned int& target,
                                          unsigned long long limit_ns = kWaitNs)
{
    __shared__ int s_ok;
    if (nblocks == 1) {  // a team of one CTA: the block barrier is enough
        __syncthreads();
        return true;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        target += nblocks;
        // the release add orders every write of the CTA (made before the block
        // barrier above) before the arrival; no separate fence is needed
        red_release_add_u32(&bar->count, 1u);
        unsigned long long spins = 0, t0 = 0;
        while (ld_acquire_u32(&bar->count) < target) {
            ++spins;
            bool give_up = spins > kSpinLimit || ((spins & 1023) == 0 && ld_volatile_u32(&bar->err));
            if ((spins & 63) == 1) {  // the clock, every 64 polls
                const unsigned long long now = global_ns();
                if (spins == 1) t0 = now;
                else if (now - t0 > limit_ns) give_up = true;
            }
            if (give_up) {
                atomicExch(&bar->err, 1u);
                ok = 0;
                break;
            }
            if (spins > 2048) __nanosleep(spins > 65536 ? 512 : 64);
        }
        // a CTA that gave up raised `err` and left; the others notice it while they poll at
        // their next barrier, so a completed wait needs no further load here
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// -------------------------------------------------- compensated dot product
//
// Dot2 (Ogita, Rump, Oishi, "Accurate sum and dot product", 2005): the FP32
// product error is recovered exactly with an FMA (TwoProduct) and the sum
// error with Knuth's TwoSum; the result is as accurate as a dot product
// computed in twice the working precision.  Used by the precompute passes
// (D^T y, D^T d_*, norms) whose values enter the screening thresholds.
struct Dot2f {
    float s, c;
    __device__ __forceinline__ Dot2f() : s(0.f), c(0.f) {}
    __device__ __forceinline__ void add(float a, float b)
    {
        float p = a * b;
        float pe = fmaf(a, b, -p);
        float t = s + p;
        float bb = t - s;
        float e = (s - (t - bb)) + (p - bb);
        s = t;
        c += e + pe;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Error-free accumulation of another (s, c) pair.
__device__ __forceinline__ void dot2_merge(Dot2f& a, float s2, float c2)
{
    float t = a.s + s2;
    float bb = t - a.s;
    float e = (a.s - (t - bb)) + (s2 - bb);
    a.s = t;
    a.c += e + c2;
}
__device__ __forceinline__ Dot2f dot2_warp_reduce(Dot2f a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float s2 = __shfl_xor_sync(0xffffffffu, a.s, o);
        float c2 = __shfl_xor_sync(0xffffffffu, a.c, o);
        dot2_merge(a, s2, c2);
    }
    return a;
}
__device__ __forceinline__ double dot2_warp_sum(Dot2f a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float s2 = __shfl_xor_sync(0xffffffffu, a.s, o);
        float c2 = __shfl_xor_sync(0xffffffffu, a.c, o);
        dot2_merge(a, s2, c2);
    }
    return a.value();
}

struct Dot2d {  // FP64 dictionaries: plain FP64 accumulation is already accurate enough
    double s;
    __device__ __forceinline__ Dot2d() : s(0.0) {}
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};

template <typename T> struct Dot2;
template <> struct Dot2<float> { using type = Dot2f; };
template <> struct Dot2<double> { using type = Dot2d; };

// ----------------------------------------------------------- warp reductions

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum of n doubles in a fixed order (lane-strided partial sums, then a fixed
// xor tree), evaluated by one full warp; every warp of every CTA that calls it
// on the same data gets the same bits.
__device__ __forceinline__ double warp_sum_fixed(const double* p, int n, int lane)
{
    double s = 0.0;
    for (int i = lane; i < n; i += kWarp) s += __ldcg(p + i);
    return warp_sum(s);
}
__device__ __forceinline__ double warp_max_fixed(const double* p, int n, int lane)
{
    double s = 0.0;
    for (int i = lane; i < n; i += kWarp) s = fmax(s, __ldcg(p + i));
    return warp_max(s);
}
__device__ __forceinline__ long long warp_sum_fixed(const int* p, int n, int lane)
{
    long long s = 0;
    for (int i = lane; i < n; i += kWarp) s += __ldcg(p + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Block-wide exclusive scan of one int per thread (any blockDim multiple of 32,
// up to 1024).  `tmp` holds 32 ints of shared memory.  Returns the exclusive
// prefix; *total receives the block sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int* tmp, int* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int t = lane < nw ? tmp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        tmp[lane] = t;  // inclusive prefix of warp totals
    }
    __syncthreads();
    int base = wid ? tmp[wid - 1] : 0;
    int tot = tmp[nw - 1];
    __syncthreads();
    *total = tot;
    return base + x - v;
}

// ------------------------------------------------------ float-float numbers
//
// An FF value is the unevaluated sum h + l of two floats with |l| <= ulp(h)/2
// (about 48 significant bits).  The operations below are built from the
// error-free transformations TwoSum (Knuth) and TwoProduct via FMA, in the
// manner of Dekker's double-length arithmetic ("A floating-point technique
// for extending the available precision", 1971).  They carry the solver's
// iterates and reductions on the FP32 pipes: GB300 executes FP64 at a small
// fraction of the FP32 rate, so per-atom and per-row FP64 arithmetic would
// dominate an iteration.
struct FF {
    float h, l;
};

__device__ __forceinline__ FF ff_two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return FF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b)  // requires |a| >= |b| or a == 0
{
    const float s = a + b;
    return FF{s, b - (s - a)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    FF s = ff_two_sum(a.h, b.h);
    const FF t = ff_two_sum(a.l, b.l);
    s.l += t.h;
    s = ff_fast_two_sum(s.h, s.l);
    s.l += t.l;
    return ff_fast_two_sum(s.h, s.l);
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.h, -a.l}; }
__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ FF ff_prod(float a, float b)
{
    const float p = a * b;
    return FF{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.h + (double)a.l; }
__host__ __device__ __forceinline__ FF ff_from_double(double d)
{
    const float h = (float)d;
    return FF{h, (float)(d - (double)h)};
}

// ------------------------------------------- FP64 reciprocal and square root
//
// GB300 runs FP64 divide and square root as long instruction sequences on its
// narrow FP64 pipe.  On the solver's serial path they are replaced by Newton's
// iteration seeded with the correctly rounded FP32 result: for the reciprocal
// r <- r + r (1 - a r), for the reciprocal square root r <- r + (r/2)(1 - a r^2).
// Each step squares the relative error (quadratic convergence), so two steps
// from a seed within 2^-23 reach the FP64 rounding level; the self-test entry
// point compares them with CUDA's own division and square root.
__device__ __forceinline__ double fast_rcp(double a)
{
    const float af = fabsf((float)a);
    if (!(af > 1e-30f && af < 1e30f)) return 1.0 / a;  // outside the FP32 seed's range
    double r = (double)__frcp_rn((float)a);
    double e = fma(-a, r, 1.0);
    r = fma(r, e, r);
    e = fma(-a, r, 1.0);
    return fma(r, e, r);
}
__device__ __forceinline__ double fast_sqrt(double a)  // a >= 0
{
    if (!(a > 0.0)) return 0.0;
    if (!(a > 1e-30 && a < 1e30)) return sqrt(a);  // outside the FP32 seed's range
    double r = (double)rsqrtf((float)a);
    double e = fma(-a * r, r, 1.0);
    r = fma(0.5 * r, e, r);
    e = fma(-a * r, r, 1.0);
    r = fma(0.5 * r, e, r);
    return a * r;
}

// ------------------------------------------------------------ small helpers

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double2; };  // 16 bytes as well

__device__ __forceinline__ float4 ldg_nc(const float4* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_nc(const double2* p) { return __ldg(p); }

}  // namespace ds
