// sv_device.cuh -- device-side helpers shared by the kernels (complex types,
// deterministic block reductions, bit helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace svk {

template <typename R> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename R> using cplx = typename cplx_t<R>::type;

template <typename R> __device__ __forceinline__ cplx<R> mk(R x, R y) { cplx<R> c; c.x = x; c.y = y; return c; }

// Insert a zero bit at position p of k (bits >= p move up by one).
__device__ __forceinline__ uint32_t insert_zero(uint32_t k, int p) {
    uint32_t low = k & ((1u << p) - 1u);
    return ((k >> p) << (p + 1)) | low;
}

// Sum over a warp in a fixed shuffle tree; the total is valid in lane 0.
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Threads per block used by every reduction kernel.
constexpr int kThreads = 256;

// Deterministic sum of one double per thread over a block of kThreads threads:
// a fixed shuffle tree inside each warp, then warp sums in warp order.  The result
// is valid in thread 0.  `red` must hold kThreads/32 doubles.
__device__ __forceinline__ double block_sum(double v, double *red) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        #pragma unroll
        for (int i = 0; i < kThreads / 32; ++i) s += red[i];
    }
    __syncthreads();
    return s;
}

// Two sums at once (same order as block_sum).
__device__ __forceinline__ void block_sum2(double &a, double &b, double *red) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[w] = a; red[kThreads / 32 + w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        #pragma unroll
        for (int i = 0; i < kThreads / 32; ++i) { sa += red[i]; sb += red[kThreads / 32 + i]; }
        a = sa; b = sb;
    }
    __syncthreads();
}

}  // namespace svk
