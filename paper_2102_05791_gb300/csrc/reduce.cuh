// Deterministic block reductions and the last-block-done pattern.
//
// Every reduction writes one partial per block; the block that finishes
// last (integer ticket, so the result does not depend on arrival order)
// sums the partials in index order.  Sums therefore come out bit-identical
// from run to run.
//
// FP32 variants serve the mixed-precision CG loop: GB300 executes FP64 at
// 1/64 of the FP32 rate, so the FP32 kernels keep their block sums in FP32
// and the one-block reductions of their partials use compensated FP32
// summation (TwoSum, Knuth), which carries each rounding error forward and
// loses nothing to a plain FP64 sum of the same partials in practice.
#pragma once

#include <cuda_runtime.h>

namespace softsim {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// FP32 sum over the block; the result is valid in thread 0.
__device__ __forceinline__ float block_sum(float v)
{
    __shared__ float redf[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) redf[w] = v;
    __syncthreads();
    float r = 0.0f;
    if (w == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? redf[lane] : 0.0f;
        r = warp_sum(r);
    }
    return r;
}

// s + e == a + b exactly (six FP32 additions; no multiplication, so no FMA
// contraction can change it).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) + (h2, l2), renormalised.
__device__ __forceinline__ void ds_merge(float &hi, float &lo, float h2, float l2)
{
    float s, e;
    two_sum(hi, h2, s, e);
    e += lo + l2;
    two_sum(s, e, hi, lo);
}

// Running sum of one thread's terms: compensated (TwoSum, error carried in
// lo) in FP32, plain in FP64.
template <typename T>
struct CompSum;
template <>
struct CompSum<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        float s, e;
        two_sum(hi, x, s, e);
        hi = s;
        lo += e;
    }
};
template <>
struct CompSum<double> {
    double hi = 0.0, lo = 0.0;
    __device__ __forceinline__ void add(double x) { hi += x; }
};

// Compensated FP32 sum over the block of per-thread (hi, lo) pairs, merged
// in a fixed order; the renormalised pair is valid in thread 0.
__device__ __forceinline__ float2 block_sum_comp(float hi, float lo)
{
    __shared__ float rh[32], rl[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o), l2 = __shfl_down_sync(0xffffffffu, lo, o);
        ds_merge(hi, lo, h2, l2);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        rh[w] = hi;
        rl[w] = lo;
    }
    __syncthreads();
    float2 r = make_float2(0.0f, 0.0f);
    if (w == 0) {
        const bool in = lane < (int)(blockDim.x >> 5);
        hi = in ? rh[lane] : 0.0f;
        lo = in ? rl[lane] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_down_sync(0xffffffffu, hi, o), l2 = __shfl_down_sync(0xffffffffu, lo, o);
            ds_merge(hi, lo, h2, l2);
        }
        r = make_float2(hi, lo);
    }
    return r;
}

// Fixed-order compensated sum of n (hi, lo) FP32 partial pairs; valid (as
// FP64, hi + lo) in thread 0.
__device__ __forceinline__ double sum_partials(const float2 *p, int n)
{
    float hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
    const int bd = blockDim.x;
    int i = threadIdx.x;
    for (; i + 3 * bd < n; i += 4 * bd) {
        float2 v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = __ldcg(p + i + k * bd);
#pragma unroll
        for (int k = 0; k < 4; ++k) ds_merge(hi[k], lo[k], v[k].x, v[k].y);
    }
    for (; i < n; i += bd) {
        const float2 v = __ldcg(p + i);
        ds_merge(hi[0], lo[0], v.x, v.y);
    }
#pragma unroll
    for (int k = 1; k < 4; ++k) ds_merge(hi[0], lo[0], hi[k], lo[k]);
    const float2 r = block_sum_comp(hi[0], lo[0]);
    return (double)r.x + (double)r.y;
}

// Fixed-order compensated sum of n FP32 partials; valid (as FP64) in thread 0.
__device__ __forceinline__ double sum_partials(const float *p, int n)
{
    float hi[8] = {0, 0, 0, 0, 0, 0, 0, 0}, lo[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int bd = blockDim.x;
    int i = threadIdx.x;
    for (; i + 7 * bd < n; i += 8 * bd) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __ldcg(p + i + k * bd);
#pragma unroll
        for (int k = 0; k < 8; ++k) ds_merge(hi[k], lo[k], v[k], 0.0f);
    }
    for (; i < n; i += bd) ds_merge(hi[0], lo[0], __ldcg(p + i), 0.0f);
#pragma unroll
    for (int k = 1; k < 8; ++k) ds_merge(hi[0], lo[0], hi[k], lo[k]);
    float h = hi[0], l = lo[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, h, o), l2 = __shfl_down_sync(0xffffffffu, l, o);
        ds_merge(h, l, h2, l2);
    }
    __shared__ float rh[32], rl[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        rh[w] = h;
        rl[w] = l;
    }
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        const bool in = lane < (int)(blockDim.x >> 5);
        h = in ? rh[lane] : 0.0f;
        l = in ? rl[lane] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_down_sync(0xffffffffu, h, o), l2 = __shfl_down_sync(0xffffffffu, l, o);
            ds_merge(h, l, h2, l2);
        }
        r = (double)h + (double)l;
    }
    return r;
}

// Sum over the block; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

__device__ __forceinline__ double block_min(double v)
{
    __shared__ double red[32];
    v = warp_min(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = INFINITY;
    if (w == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? red[lane] : INFINITY;
        r = warp_min(r);
    }
    return r;
}

// Block partial of a per-thread running sum into *slot (thread 0): a
// compensated (hi, lo) pair in FP32, stored as one float2 in the 8-byte
// slot, or a double in FP64.
template <typename T>
__device__ __forceinline__ void store_block_partial(const CompSum<T> &acc, double *slot)
{
    if constexpr (sizeof(T) == 4) {
        const float2 r = block_sum_comp(acc.hi, acc.lo);
        if (threadIdx.x == 0) *reinterpret_cast<float2 *>(slot) = r;
    } else {
        const double r = block_sum(acc.hi);
        if (threadIdx.x == 0) *slot = r;
    }
}

// Call after thread 0 has written this block's partial(s).  Returns true in
// every thread of the block that arrives last; that block resets the ticket.
// Only the partials (written by thread 0) must be visible to the last block,
// so only thread 0 fences before taking its ticket.
__device__ __forceinline__ bool last_block(unsigned int *ticket, unsigned int n_blocks)
{
    __shared__ bool is_last;
    if (threadIdx.x == 0) {
        __threadfence();
        is_last = (atomicAdd(ticket, 1u) == n_blocks - 1);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        if (threadIdx.x == 0) *ticket = 0u;
    }
    return is_last;
}

// Fixed-order sum of n partials (bypassing L1: they were written by other
// blocks); valid in thread 0.  Each thread keeps 8 loads in flight with 8
// accumulators that always take the same indices, so the result does not
// depend on timing.
__device__ __forceinline__ double sum_partials(const double *p, int n)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int bd = blockDim.x;
    int i = threadIdx.x;
    for (; i + 7 * bd < n; i += 8 * bd) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __ldcg(p + i + k * bd);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += v[k];
    }
    for (; i < n; i += bd) acc[0] += __ldcg(p + i);
    const double s = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    return block_sum(s);
}

// Fixed-order sum of n block partials written by store_block_partial<T>.
template <typename T>
__device__ __forceinline__ double sum_block_partials(const double *p, int n)
{
    if constexpr (sizeof(T) == 4)
        return sum_partials(reinterpret_cast<const float2 *>(p), n);
    else
        return sum_partials(p, n);
}

__device__ __forceinline__ double min_partials(const double *p, int n)
{
    double acc[8] = {INFINITY, INFINITY, INFINITY, INFINITY, INFINITY, INFINITY, INFINITY, INFINITY};
    const int bd = blockDim.x;
    int i = threadIdx.x;
    for (; i + 7 * bd < n; i += 8 * bd) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = __ldcg(p + i + k * bd);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = fmin(acc[k], v[k]);
    }
    for (; i < n; i += bd) acc[0] = fmin(acc[0], __ldcg(p + i));
    double s = acc[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) s = fmin(s, acc[k]);
    return block_min(s);
}

}  // namespace softsim
