// sv_ff.cuh -- float-float arithmetic: a float64 value held as the unevaluated sum
// of two float32 words, hi + lo with |lo| <= ulp(hi) / 2 (a 48-bit significand), for
// the expectation of float64 states on the FP32 pipe (GB300's FP64 pipe is about 1/64
// of its FP32 rate).  The operations are the classical error-free transformations:
//   two_sum(a, b)  = (s, e) with s = fl(a + b) and a + b = s + e exactly (Knuth),
//   fast_two_sum   the same when |a| >= |b| (Dekker),
//   two_prod(a, b) = (p, e) with p = fl(a b), a b = p + e exactly, e = fma(a, b, -p),
// combined into an addition and a multiply-add whose relative error is a few units of
// 2^-48 (Dekker 1971; Bailey's double-double library uses the same steps).  The values
// here -- amplitudes, integrals and sums of at most a few thousand products of them --
// stay far inside float32's exponent range; anything below about 1e-38 in magnitude is
// flushed to zero, an absolute error far below the float64 tolerances.
#pragma once

#include <cuda_runtime.h>

#include "sv_device.cuh"

namespace svk {

struct __align__(8) ff {
    float hi, lo;
    ff() = default;
    __host__ __device__ constexpr ff(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr ff(int v) : hi((float)v), lo(0.f) {}  // small integers: exact
    __device__ explicit ff(double v);                                      // nearest float-float
};
struct __align__(16) ffc {
    ff x, y;  // real and imaginary parts
};

template <> struct AmpT<ffc> { using R = ff; static constexpr bool kCplx = true; };
template <> struct AmpT<ff> { using R = ff; static constexpr bool kCplx = false; };

__device__ __forceinline__ ff ff_make(float hi, float lo) { return ff(hi, lo); }

// nearest float-float of a float64 value (float64 operations: used where values enter)
__device__ __forceinline__ ff ff_from(double x) {
    const float h = __double2float_rn(x);
    return ff(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ ff::ff(double v) : hi(0.f), lo(0.f) { *this = ff_from(v); }
__device__ __forceinline__ double ff_to(ff a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e += a.lo + b.lo;
    fast_two_sum(s, e, s, e);
    return ff_make(s, e);
}
__device__ __forceinline__ ff operator-(ff a) { return ff_make(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff &operator+=(ff &a, ff b) { a = a + b; return a; }
__device__ __forceinline__ ff operator*(ff a, ff b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    float s;
    fast_two_sum(p, e, s, e);
    return ff_make(s, e);
}
// acc + a b in one step: the exact product (p, e) added to acc with one two_sum
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff acc) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    float s, t;
    two_sum(acc.hi, p, s, t);
    t += e + acc.lo;
    fast_two_sum(s, t, s, t);
    return ff_make(s, t);
}

// the amplitude helpers of sv_device.cuh for the float-float types
__device__ __forceinline__ ff re(ffc a) { return a.x; }
__device__ __forceinline__ ff im(ffc a) { return a.y; }
__device__ __forceinline__ ff re(ff a) { return a; }
__device__ __forceinline__ ff im(ff) { return ff_make(0.f, 0.f); }
template <> __device__ __forceinline__ ffc mka<ffc>(ff x, ff y) { ffc c; c.x = x; c.y = y; return c; }
template <> __device__ __forceinline__ ff mka<ff>(ff x, ff) { return x; }

__device__ __forceinline__ void axpy(ffc &acc, ff v, ffc c) {
    acc.x = ff_fma(v, c.x, acc.x);
    acc.y = ff_fma(v, c.y, acc.y);
}
__device__ __forceinline__ void axpy(ff &acc, ff v, ff c) { acc = ff_fma(v, c, acc); }
__device__ __forceinline__ void acc2(ffc &a, ff w0, ffc c0, ff w1, ffc c1) {
    a.x = ff_fma(w1, c1.x, ff_fma(w0, c0.x, a.x));
    a.y = ff_fma(w1, c1.y, ff_fma(w0, c0.y, a.y));
}
__device__ __forceinline__ void acc2(ff &a, ff w0, ff c0, ff w1, ff c1) { a = ff_fma(w1, c1, ff_fma(w0, c0, a)); }

template <> __device__ __forceinline__ double dre_dot<ffc>(ffc u, ffc v) {
    return ff_to(u.x) * ff_to(v.x) + ff_to(u.y) * ff_to(v.y);
}
template <> __device__ __forceinline__ double dre_dot<ff>(ff u, ff v) { return ff_to(u) * ff_to(v); }

// a value with its sign flipped when bit is 1 (both words: sign-bit operations)
__device__ __forceinline__ ff ff_flip(ff v, uint32_t bit) {
    const int m = (int)(bit << 31);
    return ff_make(__int_as_float(__float_as_int(v.hi) ^ m), __int_as_float(__float_as_int(v.lo) ^ m));
}

}  // namespace svk
