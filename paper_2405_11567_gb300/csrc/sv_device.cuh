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

// Amplitude types of a state: complex (float2 / double2, interleaved re, im) or
// real (float / double: the real-amplitude states SV_R32 / SV_R64).  Kernels that
// serve both are written against these helpers; for a real type every imaginary
// part is the constant 0 and drops out at compile time.
template <typename A> struct AmpT;
template <> struct AmpT<float2> { using R = float; static constexpr bool kCplx = true; };
template <> struct AmpT<double2> { using R = double; static constexpr bool kCplx = true; };
template <> struct AmpT<float> { using R = float; static constexpr bool kCplx = false; };
template <> struct AmpT<double> { using R = double; static constexpr bool kCplx = false; };
template <typename A> using real_of = typename AmpT<A>::R;

__device__ __forceinline__ float re(float2 a) { return a.x; }
__device__ __forceinline__ double re(double2 a) { return a.x; }
__device__ __forceinline__ float re(float a) { return a; }
__device__ __forceinline__ double re(double a) { return a; }
__device__ __forceinline__ float im(float2 a) { return a.y; }
__device__ __forceinline__ double im(double2 a) { return a.y; }
__device__ __forceinline__ float im(float) { return 0.f; }
__device__ __forceinline__ double im(double) { return 0.0; }

// The amplitude x + i y (y dropped for a real type).
template <typename A> __device__ __forceinline__ A mka(real_of<A> x, real_of<A> y);
template <> __device__ __forceinline__ float2 mka<float2>(float x, float y) { return make_float2(x, y); }
template <> __device__ __forceinline__ double2 mka<double2>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float mka<float>(float x, float) { return x; }
template <> __device__ __forceinline__ double mka<double>(double x, double) { return x; }

// s a + t b, component by component.
template <typename A>
__device__ __forceinline__ A lin2(real_of<A> s, A a, real_of<A> t, A b) {
    return mka<A>(s * re(a) + t * re(b), s * im(a) + t * im(b));
}
// acc += v c (v real).
template <typename A>
__device__ __forceinline__ void axpy(A &acc, real_of<A> v, A c) {
    acc = mka<A>(re(acc) + v * re(c), im(acc) + v * im(c));
}
// v c and a + b.
template <typename A> __device__ __forceinline__ A scale_a(real_of<A> v, A c) { return mka<A>(v * re(c), v * im(c)); }
template <typename A> __device__ __forceinline__ A add_a(A a, A b) { return mka<A>(re(a) + re(b), im(a) + im(b)); }
// acc += w0 c0 + w1 c1 as two chained multiply-adds per component (no separate product:
// float64 states are FP64-pipe bound on GB300).
__device__ __forceinline__ void acc2(float2 &a, float w0, float2 c0, float w1, float2 c1) {
    a.x = fmaf(w1, c1.x, fmaf(w0, c0.x, a.x));
    a.y = fmaf(w1, c1.y, fmaf(w0, c0.y, a.y));
}
__device__ __forceinline__ void acc2(double2 &a, double w0, double2 c0, double w1, double2 c1) {
    a.x = fma(w1, c1.x, fma(w0, c0.x, a.x));
    a.y = fma(w1, c1.y, fma(w0, c0.y, a.y));
}
__device__ __forceinline__ void acc2(float &a, float w0, float c0, float w1, float c1) { a = fmaf(w1, c1, fmaf(w0, c0, a)); }
__device__ __forceinline__ void acc2(double &a, double w0, double c0, double w1, double c1) { a = fma(w1, c1, fma(w0, c0, a)); }
// Re(conj(u) v) in float64.
template <typename A>
__device__ __forceinline__ double dre_dot(A u, A v) {
    if constexpr (AmpT<A>::kCplx) return (double)re(u) * (double)re(v) + (double)im(u) * (double)im(v);
    else return (double)u * (double)v;
}
// Re(conj(u) v) and Im(conj(u) v).
template <typename A> __device__ __forceinline__ real_of<A> re_dot(A u, A v) { return re(u) * re(v) + im(u) * im(v); }
template <typename A> __device__ __forceinline__ real_of<A> im_dot(A u, A v) { return re(u) * im(v) - im(u) * re(v); }

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

// block_sum / block_sum2 for a block of NT threads (NT a multiple of 32, <= 1024);
// `red` must hold NT/32 (block_sum_nt) or 2 NT/32 (block_sum2_nt) doubles.
template <int NT>
__device__ __forceinline__ double block_sum_nt(double v, double *red) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        #pragma unroll
        for (int i = 0; i < NT / 32; ++i) s += red[i];
    }
    __syncthreads();
    return s;
}

template <int NT>
__device__ __forceinline__ void block_sum2_nt(double &a, double &b, double *red) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[w] = a; red[NT / 32 + w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        #pragma unroll
        for (int i = 0; i < NT / 32; ++i) { sa += red[i]; sb += red[NT / 32 + i]; }
        a = sa; b = sb;
    }
    __syncthreads();
}

}  // namespace svk
