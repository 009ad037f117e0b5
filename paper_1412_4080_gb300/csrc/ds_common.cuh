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
// Sense-counting barrier for a cooperative grid (all CTAs co-resident).  The
// last CTA to arrive resets the counter and bumps the generation; the others
// spin on the generation with an iteration limit.  A wait that exceeds the
// limit sets `err` and returns false; every CTA then leaves its loop, so a
// lost CTA can never hang the GPU.
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    unsigned int err;
    unsigned int pad;
};

constexpr unsigned long long kSpinLimit = 1ull << 25;  // ~2 s with the backoff below

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

// Returns true when every CTA arrived; false when the barrier (now or earlier)
// failed.  `gen` is the CTA's private copy of the generation counter.
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned int nblocks, unsigned int& gen)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned int g = gen;
        __threadfence();
        unsigned int arrived = atomicAdd(&bar->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (ld_acquire_u32(&bar->gen) == g) {
                if (++spins > kSpinLimit || ld_volatile_u32(&bar->err)) {
                    atomicExch(&bar->err, 1u);
                    ok = 0;
                    break;
                }
                if (spins > 64) __nanosleep(spins > 4096 ? 256 : 32);
            }
        }
        __threadfence();
        if (ld_volatile_u32(&bar->err)) ok = 0;
        gen = g + 1;
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

// ------------------------------------------------------------ small helpers

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double2; };  // 16 bytes as well

__device__ __forceinline__ float4 ldg_nc(const float4* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg_nc(const double2* p) { return __ldg(p); }

}  // namespace ds
