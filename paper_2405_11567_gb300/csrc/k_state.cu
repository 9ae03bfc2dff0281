// k_state.cu -- state preparation, the excitation-rotation kernel (forward
// sweep) and the fused adjoint step (reverse sweep), plus the fixed-order
// row reduction used by every reduction.
//
// Rotation (one launch per excitation, Methodology "Computational Details":
// ADAPT-VQE ansatz of fermionic excitations).  For excitation T with flip mask m,
// every basis index x whose mask bits equal `from` is paired with x' = x ^ m,
// T|x> = s|x'> with s = (-1)^popc(x & sm), and U = exp(theta (T - T^dagger)) acts
// on the pair as
//     psi'[x]  = c psi[x]  - s sn psi[x']
//     psi'[x'] = c psi[x'] + s sn psi[x]
// (c = cos theta, sn = sin theta, from the host in float64).  Every other
// amplitude is left alone.  The kernel streams the 2 * 2^(n - nbits) touched
// amplitudes once (read + write): HBM-bound.
//
// Adjoint step: with psi_k and lambda_k (lambda = (H - c) psi_L carried back
// through the gates), g_k = 2 Re <lambda_k| G_k psi_k> where
// (G psi)[x] = -s psi[x'], (G psi)[x'] = s psi[x]; then both vectors are
// rotated by U_k^dagger = exp(-theta G_k).  One pass over the touched pairs of
// both vectors; the per-block float64 partial sums are reduced afterwards in a
// fixed order (bit-identical reruns).
#include "sv_device.cuh"
#include "sv_internal.h"

namespace svk {

struct OpArgs {
    uint32_t m, from, sm;
    int pos0, pos1, pos2, pos3;
    double c, s;
    double t;    // tan(theta / 2) = s / (1 + c), for the shear form
    int shear;   // 1 when c > 0 (|t| < 1): float64 amplitudes rotate by three shears
};

static OpArgs to_args(const OpDesc &d) {
    OpArgs a;
    a.m = d.m; a.from = d.from; a.sm = d.sm;
    a.pos0 = d.pos[0]; a.pos1 = d.pos[1]; a.pos2 = d.pos[2]; a.pos3 = d.pos[3];
    a.c = d.c; a.s = d.s;
    a.shear = d.c > 0.0;
    a.t = a.shear ? d.s / (1.0 + d.c) : 0.0;
    return a;
}

// (p, q) <- (c p - s q, s p + c q), the rotation [[c, -s], [s, c]], as three shears
// (Paeth's decomposition, valid for c > -1 with t = tan of the half angle):
// p1 = p - t q, q' = q + s p1, p' = p1 - t q'.  Three multiply-adds per component
// instead of four: the float64 kernels are bound by GB300's FP64 pipe, not by HBM, so
// this is what moves them.  Rounding differs from the direct form only in the last
// bits; a quarter turn (t = 1, s = 1) still maps basis states exactly.
// x or -x by flipping the sign bit (an integer operation: keeps the FP64 pipe free).
__device__ __forceinline__ double neg_if(double x, bool neg) {
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)neg << 63));
}
__device__ __forceinline__ float neg_if(float x, bool neg) {
    return __int_as_float(__float_as_int(x) ^ ((int)neg << 31));
}

template <typename R>
__device__ __forceinline__ void shear3(R &p, R &q, R t, R s) {
    const R p1 = fma(-t, q, p);
    q = fma(s, p1, q);
    p = fma(-t, q, p1);
}
__device__ __forceinline__ void rot_shear(double2 &p, double2 &q, double t, double s) {
    shear3(p.x, q.x, t, s);
    shear3(p.y, q.y, t, s);
}
__device__ __forceinline__ void rot_shear(double &p, double &q, double t, double s) { shear3(p, q, t, s); }

template <int NB>
__device__ __forceinline__ uint32_t pair_index(uint32_t k, const OpArgs &a) {
    uint32_t x = insert_zero(k, a.pos0);
    x = insert_zero(x, a.pos1);
    if (NB == 4) {
        x = insert_zero(x, a.pos2);
        x = insert_zero(x, a.pos3);
    }
    return x | a.from;
}

// ---------------------------------------------------------------- preparation

template <typename A>
__global__ void k_set_basis(A *psi, uint32_t x) {
    psi[x] = mka<A>(real_of<A>(1), real_of<A>(0));
}

// ---------------------------------------------------------------- vector access

// V consecutive amplitudes starting at a V-aligned index, moved as 16-byte words
// (complex64: V = 2 or 4 -> one or two float4; complex128: one double2 each).
template <typename R, int V> struct VecIO;

template <int V> struct VecIO<float, V> {
    static __device__ __forceinline__ void ld(const float2 *__restrict__ p, float2 (&v)[V]) {
        if constexpr (V == 1) {
            v[0] = p[0];
        } else {
            #pragma unroll
            for (int i = 0; i < V / 2; ++i) {
                float4 f = reinterpret_cast<const float4 *>(p)[i];
                v[2 * i] = make_float2(f.x, f.y);
                v[2 * i + 1] = make_float2(f.z, f.w);
            }
        }
    }
    static __device__ __forceinline__ void st(float2 *__restrict__ p, const float2 (&v)[V]) {
        if constexpr (V == 1) {
            p[0] = v[0];
        } else {
            #pragma unroll
            for (int i = 0; i < V / 2; ++i)
                reinterpret_cast<float4 *>(p)[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
        }
    }
};

template <int V> struct VecIO<double, V> {
    static __device__ __forceinline__ void ld(const double2 *__restrict__ p, double2 (&v)[V]) {
        #pragma unroll
        for (int i = 0; i < V; ++i) v[i] = p[i];
    }
    static __device__ __forceinline__ void st(double2 *__restrict__ p, const double2 (&v)[V]) {
        #pragma unroll
        for (int i = 0; i < V; ++i) p[i] = v[i];
    }
};

// Real amplitudes: V floats as one float2 / float4, V doubles as double2 words.
template <int V> struct VecIOr;
template <> struct VecIOr<1> {
    template <typename T> static __device__ __forceinline__ void ld(const T *__restrict__ p, T (&v)[1]) { v[0] = p[0]; }
    template <typename T> static __device__ __forceinline__ void st(T *__restrict__ p, const T (&v)[1]) { p[0] = v[0]; }
};
template <> struct VecIOr<2> {
    static __device__ __forceinline__ void ld(const float *__restrict__ p, float (&v)[2]) {
        const float2 f = *reinterpret_cast<const float2 *>(p);
        v[0] = f.x; v[1] = f.y;
    }
    static __device__ __forceinline__ void st(float *__restrict__ p, const float (&v)[2]) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    }
    static __device__ __forceinline__ void ld(const double *__restrict__ p, double (&v)[2]) {
        const double2 f = *reinterpret_cast<const double2 *>(p);
        v[0] = f.x; v[1] = f.y;
    }
    static __device__ __forceinline__ void st(double *__restrict__ p, const double (&v)[2]) {
        *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    }
};
template <> struct VecIOr<4> {
    static __device__ __forceinline__ void ld(const float *__restrict__ p, float (&v)[4]) {
        const float4 f = *reinterpret_cast<const float4 *>(p);
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
    }
    static __device__ __forceinline__ void st(float *__restrict__ p, const float (&v)[4]) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    static __device__ __forceinline__ void ld(const double *__restrict__ p, double (&v)[4]) {
        const double2 f = reinterpret_cast<const double2 *>(p)[0], g = reinterpret_cast<const double2 *>(p)[1];
        v[0] = f.x; v[1] = f.y; v[2] = g.x; v[3] = g.y;
    }
    static __device__ __forceinline__ void st(double *__restrict__ p, const double (&v)[4]) {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
};

template <> struct VecIOr<8> {
    static __device__ __forceinline__ void ld(const float *__restrict__ p, float (&v)[8]) {
        const float4 f = reinterpret_cast<const float4 *>(p)[0], g = reinterpret_cast<const float4 *>(p)[1];
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w; v[4] = g.x; v[5] = g.y; v[6] = g.z; v[7] = g.w;
    }
    static __device__ __forceinline__ void st(float *__restrict__ p, const float (&v)[8]) {
        reinterpret_cast<float4 *>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4 *>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
};

template <int V> __device__ __forceinline__ void ld_vec(const float2 *__restrict__ p, float2 (&v)[V]) { VecIO<float, V>::ld(p, v); }
template <int V> __device__ __forceinline__ void ld_vec(const double2 *__restrict__ p, double2 (&v)[V]) { VecIO<double, V>::ld(p, v); }
template <int V> __device__ __forceinline__ void ld_vec(const float *__restrict__ p, float (&v)[V]) { VecIOr<V>::ld(p, v); }
template <int V> __device__ __forceinline__ void ld_vec(const double *__restrict__ p, double (&v)[V]) { VecIOr<V>::ld(p, v); }
template <int V> __device__ __forceinline__ void st_vec(float2 *__restrict__ p, const float2 (&v)[V]) { VecIO<float, V>::st(p, v); }
template <int V> __device__ __forceinline__ void st_vec(double2 *__restrict__ p, const double2 (&v)[V]) { VecIO<double, V>::st(p, v); }
template <int V> __device__ __forceinline__ void st_vec(float *__restrict__ p, const float (&v)[V]) { VecIOr<V>::st(p, v); }
template <int V> __device__ __forceinline__ void st_vec(double *__restrict__ p, const double (&v)[V]) { VecIOr<V>::st(p, v); }

// ---------------------------------------------------------------- forward rotation

// Each thread owns groups of V consecutive pair indices; the lowest mask position is
// >= log2(V), so a group maps to V consecutive amplitudes on each side of the pair
// and the sign is the same across the group only if no sign-mask bit lies below
// log2(V) -- it is therefore evaluated per amplitude.  Two groups per iteration keep
// four independent vector loads in flight per thread.
// psi'[x] = c psi[x] - s sn psi[x'], psi'[x'] = c psi[x'] + s sn psi[x] on one pair
// (s = -1 when neg); float64 amplitudes use the shear form when the op allows it.
template <typename A>
__device__ __forceinline__ void rotate_pair(A &p, A &q, bool neg, real_of<A> c, real_of<A> sn, real_of<A> th,
                                            bool shear) {
    using R = real_of<A>;
    if constexpr (sizeof(R) == 8) {
        const R ss = neg_if(sn, neg);
        if (shear) {
            rot_shear(p, q, neg_if(th, neg), ss);
            return;
        }
        const A p0 = p, q0 = q;
        p = lin2<A>(c, p0, -ss, q0);
        q = lin2<A>(c, q0, ss, p0);
        return;
    }
    const R ss = neg ? -sn : sn;
    const A p0 = p, q0 = q;
    p = lin2<A>(c, p0, -ss, q0);
    q = lin2<A>(c, q0, ss, p0);
}

template <typename A, int NB, int V>
__global__ void __launch_bounds__(kThreads) k_rotate(A *__restrict__ psi, uint32_t ngroups, OpArgs a) {
    using R = real_of<A>;
    const R c = (R)a.c, sn = (R)a.s, th = (R)a.t;
    const bool shear = a.shear != 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += 2 * stride) {
        const uint32_t g2 = g + stride;
        const bool two = g2 < ngroups;
        const uint32_t x = pair_index<NB>(g * V, a), x2 = two ? pair_index<NB>(g2 * V, a) : x;
        A u[V], v[V], u2[V], v2[V];
        ld_vec<V>(psi + x, u);
        ld_vec<V>(psi + (x ^ a.m), v);
        if (two) {
            ld_vec<V>(psi + x2, u2);
            ld_vec<V>(psi + (x2 ^ a.m), v2);
        }
        #pragma unroll
        for (int i = 0; i < V; ++i) rotate_pair<A>(u[i], v[i], (__popc((x + i) & a.sm) & 1) != 0, c, sn, th, shear);
        st_vec<V>(psi + x, u);
        st_vec<V>(psi + (x ^ a.m), v);
        if (two) {
            #pragma unroll
            for (int i = 0; i < V; ++i)
                rotate_pair<A>(u2[i], v2[i], (__popc((x2 + i) & a.sm) & 1) != 0, c, sn, th, shear);
            st_vec<V>(psi + x2, u2);
            st_vec<V>(psi + (x2 ^ a.m), v2);
        }
    }
}

// ---------------------------------------------------------------- adjoint step

// One pair of the adjoint step: adds the pair's term of Re <lambda|G psi> to t and
// applies U^dagger to (u, v) (psi) and (lu, lv) (lambda).  <lambda|G psi> on the pair:
// conj(lu) (-s v) + conj(lv) (s u), real part.  U^dagger: psi'[x] = c u + s sn v,
// psi'[x'] = c v - s sn u (lambda alike), the forward rotation with the sign of the
// angle flipped.
template <typename A>
__device__ __forceinline__ void adjoint_pair(A &u, A &v, A &lu, A &lv, bool neg, real_of<A> c, real_of<A> sn,
                                             real_of<A> th, bool shear, real_of<A> &t) {
    using R = real_of<A>;
    if constexpr (sizeof(R) == 8) {
        // float64: the product terms chained into t by multiply-adds (sign on the
        // lambda operand), four per complex pair instead of six
        t = fma(neg_if(re(lv), neg), re(u), t);
        t = fma(neg_if(re(lu), !neg), re(v), t);
        if constexpr (AmpT<A>::kCplx) {
            t = fma(neg_if(im(lv), neg), im(u), t);
            t = fma(neg_if(im(lu), !neg), im(v), t);
        }
    } else {
        const R ti = re_dot(lv, u) - re_dot(lu, v);
        t += neg ? -ti : ti;
    }
    rotate_pair<A>(u, v, !neg, c, sn, th, shear);
    rotate_pair<A>(lu, lv, !neg, c, sn, th, shear);
}

template <typename A, int NB, int V>
__global__ void __launch_bounds__(kThreads) k_adjoint(A *__restrict__ psi, A *__restrict__ lam,
                                                      uint32_t ngroups, OpArgs a, double *__restrict__ partial) {
    using R = real_of<A>;
    __shared__ double red[kThreads / 32];
    const R c = (R)a.c, sn = (R)a.s, th = (R)a.t;
    const bool shear = a.shear != 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    double acc = 0.0;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
        const uint32_t x = pair_index<NB>(g * V, a), xp = x ^ a.m;
        A u[V], v[V], lu[V], lv[V];
        ld_vec<V>(psi + x, u);
        ld_vec<V>(psi + xp, v);
        ld_vec<V>(lam + x, lu);
        ld_vec<V>(lam + xp, lv);
        R t = 0;
        #pragma unroll
        for (int i = 0; i < V; ++i)
            adjoint_pair<A>(u[i], v[i], lu[i], lv[i], (__popc((x + i) & a.sm) & 1) != 0, c, sn, th, shear, t);
        acc += (double)t;
        st_vec<V>(psi + x, u);
        st_vec<V>(psi + xp, v);
        st_vec<V>(lam + x, lu);
        st_vec<V>(lam + xp, lv);
    }
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// ---------------------------------------------------------------- adjoint step, interleaved

// The same step on one buffer holding psi and lambda interleaved by amplitude,
// cl[2x] = psi[x], cl[2x + 1] = lambda[x].  A touched run of 2^b amplitudes is then
// one run of 2^(b+1) words instead of one run of 2^b in each of two vectors, so an
// excitation whose lowest address bit is b moves runs twice as long: HBM moves
// 32-byte sectors, runs of 8 or 16 bytes use half of each, and runs of 128 bytes or
// more stream at about the copy rate.  Two groups of V pairs per iteration (four
// vector loads in flight per thread).
template <typename A, int NB, int V>
__global__ void __launch_bounds__(kThreads) k_adjoint_i(A *__restrict__ cl, uint32_t ngroups, OpArgs a,
                                                        double *__restrict__ partial) {
    using R = real_of<A>;
    __shared__ double red[kThreads / 32];
    const R c = (R)a.c, sn = (R)a.s, th = (R)a.t;
    const bool shear = a.shear != 0;
    const uint32_t stride = gridDim.x * blockDim.x;
    double acc = 0.0;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += 2 * stride) {
        const uint32_t g2 = g + stride;
        const bool two = g2 < ngroups;
        const uint32_t x = pair_index<NB>(g * V, a), x2 = two ? pair_index<NB>(g2 * V, a) : x;
        A *const p = cl + 2 * (size_t)x, *const q = cl + 2 * (size_t)(x ^ a.m);
        A *const p2 = cl + 2 * (size_t)x2, *const q2 = cl + 2 * (size_t)(x2 ^ a.m);
        A u[2 * V], v[2 * V], u2[2 * V], v2[2 * V];
        ld_vec<2 * V>(p, u);
        ld_vec<2 * V>(q, v);
        if (two) {
            ld_vec<2 * V>(p2, u2);
            ld_vec<2 * V>(q2, v2);
        }
        R t = 0;
        #pragma unroll
        for (int i = 0; i < V; ++i)
            adjoint_pair<A>(u[2 * i], v[2 * i], u[2 * i + 1], v[2 * i + 1], (__popc((x + i) & a.sm) & 1) != 0, c,
                            sn, th, shear, t);
        acc += (double)t;
        st_vec<2 * V>(p, u);
        st_vec<2 * V>(q, v);
        if (two) {
            R t2 = 0;
            #pragma unroll
            for (int i = 0; i < V; ++i)
                adjoint_pair<A>(u2[2 * i], v2[2 * i], u2[2 * i + 1], v2[2 * i + 1],
                                (__popc((x2 + i) & a.sm) & 1) != 0, c, sn, th, shear, t2);
            acc += (double)t2;
            st_vec<2 * V>(p2, u2);
            st_vec<2 * V>(q2, v2);
        }
    }
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// cl[2x] = psi[x], cl[2x + 1] = 0 for every x (two amplitudes per thread and step:
// one 16- or 32-byte load, one 32- or 64-byte store).
template <typename A>
__global__ void __launch_bounds__(kThreads) k_interleave_zero(const A *__restrict__ psi, A *__restrict__ cl,
                                                              uint64_t pairs) {
    const A z = mka<A>(real_of<A>(0), real_of<A>(0));
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < pairs;
         t += (uint64_t)gridDim.x * blockDim.x) {
        A u[2], w[4];
        ld_vec<2>(psi + 2 * t, u);
        w[0] = u[0]; w[1] = z; w[2] = u[1]; w[3] = z;
        st_vec<4>(cl + 4 * t, w);
    }
}

// The odd words of the interleaved buffer at the sector's storage addresses:
// cl[2 (sa_s[a] | sb_s[b]) + 1] = lamc[b Da + a] (one block per beta string).
template <typename A>
__global__ void __launch_bounds__(kThreads) k_scatter_odd(const A *__restrict__ lamc, A *__restrict__ cl,
                                                          const uint32_t *__restrict__ sa_s,
                                                          const uint32_t *__restrict__ sb_s, int Da, int Db) {
    for (int Ib = blockIdx.x; Ib < Db; Ib += gridDim.x) {
        const uint32_t xb = sb_s[Ib];
        const A *row = lamc + (size_t)Ib * Da;
        for (int Ia = threadIdx.x; Ia < Da; Ia += blockDim.x) cl[2 * (size_t)(sa_s[Ia] | xb) + 1] = row[Ia];
    }
}

// ---------------------------------------------------------------- layout change

// out[sigma(x)] = in[x]: sigma moves address bit j to address bit sg[j].
struct PermArgs {
    int sg[32];
    int n;
};

template <typename A>
__global__ void __launch_bounds__(kThreads) k_permute(const A *__restrict__ in, A *__restrict__ out,
                                                      uint64_t dim, PermArgs p) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < dim; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)t;
        uint32_t y = 0;
        for (int j = 0; j < p.n; ++j) y |= ((v >> j) & 1u) << p.sg[j];
        out[y] = in[t];
    }
}

cudaError_t launch_permute(const void *in, void *out, int dtype, int n, const int *sg, int sm_count, cudaStream_t st) {
    PermArgs p;
    for (int j = 0; j < 32; ++j) p.sg[j] = j < n ? sg[j] : j;
    p.n = n;
    uint64_t dim = 1ull << n;
    uint64_t want = (dim + kThreads - 1) / kThreads, cap = (uint64_t)sm_count * 16;
    int grid = (int)(want < cap ? want : cap);
    SV_DISPATCH_AMP(dtype, k_permute<A><<<grid, kThreads, 0, st>>>((const A *)in, (A *)out, dim, p));
    return cudaGetLastError();
}

// ---------------------------------------------------------------- sampling

// out[i] = psi[addr[i]] (addresses already in the storage layout)
template <typename A>
__global__ void __launch_bounds__(kThreads) k_gather(const A *__restrict__ psi, const uint32_t *__restrict__ addr,
                                                     int count, A *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) out[i] = psi[addr[i]];
}

cudaError_t launch_gather(const void *psi, int dtype, const uint32_t *addr, int count, void *out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    int grid = (count + kThreads - 1) / kThreads;
    if (grid > 1024) grid = 1024;
    SV_DISPATCH_AMP(dtype, k_gather<A><<<grid, kThreads, 0, st>>>((const A *)psi, addr, count, (A *)out));
    return cudaGetLastError();
}

// ---------------------------------------------------------------- reductions

// out[r] = sum_c partials[r * cols + c], fixed order (one block per row).
__global__ void __launch_bounds__(kThreads) k_reduce_rows(const double *__restrict__ partials, int cols,
                                                          double *__restrict__ out) {
    __shared__ double red[kThreads / 32];
    const double *row = partials + (size_t)blockIdx.x * cols;
    double acc = 0.0;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) acc += row[c];
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// ---------------------------------------------------------------- launchers

// Blocks for a grid-stride launch over npairs items: enough for one item per thread,
// at most bps blocks per SM (8 unless sv_autotune / SV_OPT_ROT_BLOCKS_PER_SM chose).
int rotate_grid(uint64_t npairs, int sm_count, int bps) {
    uint64_t want = (npairs + kThreads - 1) / kThreads;
    uint64_t cap = (uint64_t)sm_count * (uint64_t)(bps > 0 ? bps : 8);
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

cudaError_t launch_set_basis(void *psi, int dtype, uint32_t x, cudaStream_t st) {
    SV_DISPATCH_AMP(dtype, k_set_basis<A><<<1, 1, 0, st>>>((A *)psi, x));
    return cudaGetLastError();
}

// Vector width: as many consecutive amplitudes as fit in 32 bytes, limited by the
// lowest mask position (the pairs of a group must be consecutive on both sides).
static int vec_log2(int dtype, const OpDesc &d, int n) {
    int vmax = dtype == SV_C128 ? 1 : 2;  // 32-byte words (16 for real floats)
    int v = d.pos[0] < vmax ? d.pos[0] : vmax;
    while (v > 0 && (n - d.nbits) < v) --v;
    return v;
}

template <typename A, int NB>
static void rot_v(void *psi, int v, uint32_t npairs, OpArgs a, int sm_count, int bps, cudaStream_t st) {
    uint32_t ng = npairs >> v;
    int grid = rotate_grid((ng + 1) / 2, sm_count, bps);
    if (v == 0) k_rotate<A, NB, 1><<<grid, kThreads, 0, st>>>((A *)psi, ng, a);
    else if (v == 1) k_rotate<A, NB, 2><<<grid, kThreads, 0, st>>>((A *)psi, ng, a);
    else k_rotate<A, NB, 4><<<grid, kThreads, 0, st>>>((A *)psi, ng, a);
}

cudaError_t launch_rotate(void *psi, int dtype, int n, const OpDesc &d, int sm_count, int bps, cudaStream_t st) {
    OpArgs a = to_args(d);
    uint32_t npairs = (uint32_t)(1ull << (n - d.nbits));
    int v = vec_log2(dtype, d, n);
    SV_DISPATCH_AMP(dtype, if (d.nbits == 2) rot_v<A, 2>(psi, v, npairs, a, sm_count, bps, st);
                           else rot_v<A, 4>(psi, v, npairs, a, sm_count, bps, st));
    return cudaGetLastError();
}

template <typename A, int NB>
static void adj_v(void *psi, void *lam, int v, uint32_t npairs, OpArgs a, int grid, double *partial,
                  cudaStream_t st) {
    uint32_t ng = npairs >> v;
    if (v == 0) k_adjoint<A, NB, 1><<<grid, kThreads, 0, st>>>((A *)psi, (A *)lam, ng, a, partial);
    else if (v == 1) k_adjoint<A, NB, 2><<<grid, kThreads, 0, st>>>((A *)psi, (A *)lam, ng, a, partial);
    else k_adjoint<A, NB, 4><<<grid, kThreads, 0, st>>>((A *)psi, (A *)lam, ng, a, partial);
}

// `grid` blocks write partial[0 .. grid); the caller gives every op the same grid.
cudaError_t launch_adjoint(void *psi, void *lam, int dtype, int n, const OpDesc &d, int grid,
                           double *partial, cudaStream_t st) {
    OpArgs a = to_args(d);
    uint32_t npairs = (uint32_t)(1ull << (n - d.nbits));
    int v = vec_log2(dtype, d, n);
    SV_DISPATCH_AMP(dtype, if (d.nbits == 2) adj_v<A, 2>(psi, lam, v, npairs, a, grid, partial, st);
                           else adj_v<A, 4>(psi, lam, v, npairs, a, grid, partial, st));
    return cudaGetLastError();
}

// Interleaved adjoint step: V elements (psi, lambda pairs) per vector access, at most
// 32 bytes, limited as for the separate vectors by the lowest mask position.
static int vec_log2_i(int dtype, const OpDesc &d, int n) {
    const int ebytes = 2 * (int)amp_size(dtype);
    int vmax = ebytes >= 32 ? 0 : ebytes == 16 ? 1 : 2;
    int v = d.pos[0] < vmax ? d.pos[0] : vmax;
    while (v > 0 && (n - d.nbits) < v) --v;
    return v;
}

template <typename A, int NB>
static void adj_i_v(void *cl, int v, uint32_t npairs, OpArgs a, int grid, double *partial, cudaStream_t st) {
    uint32_t ng = npairs >> v;
    if (v == 0) k_adjoint_i<A, NB, 1><<<grid, kThreads, 0, st>>>((A *)cl, ng, a, partial);
    else if (v == 1) k_adjoint_i<A, NB, 2><<<grid, kThreads, 0, st>>>((A *)cl, ng, a, partial);
    else {
        if constexpr (sizeof(A) == 4) k_adjoint_i<A, NB, 4><<<grid, kThreads, 0, st>>>((A *)cl, ng, a, partial);
    }
}

// `grid` blocks write partial[0 .. grid); the caller gives every op the same grid.
cudaError_t launch_adjoint_i(void *cl, int dtype, int n, const OpDesc &d, int grid, double *partial,
                             cudaStream_t st) {
    OpArgs a = to_args(d);
    uint32_t npairs = (uint32_t)(1ull << (n - d.nbits));
    int v = vec_log2_i(dtype, d, n);
    SV_DISPATCH_AMP(dtype, if (d.nbits == 2) adj_i_v<A, 2>(cl, v, npairs, a, grid, partial, st);
                           else adj_i_v<A, 4>(cl, v, npairs, a, grid, partial, st));
    return cudaGetLastError();
}

cudaError_t launch_interleave_zero(const void *psi, void *cl, int dtype, int n, int sm_count, cudaStream_t st) {
    const uint64_t pairs = 1ull << (n - 1);
    uint64_t want = (pairs + kThreads - 1) / kThreads, cap = (uint64_t)sm_count * 16;
    const int grid = (int)(want < cap ? want : cap);
    SV_DISPATCH_AMP(dtype, k_interleave_zero<A><<<grid, kThreads, 0, st>>>((const A *)psi, (A *)cl, pairs));
    return cudaGetLastError();
}

cudaError_t launch_scatter_odd(const void *lamc, void *cl, int dtype, const uint32_t *sa_s, const uint32_t *sb_s,
                               int Da, int Db, int sm_count, cudaStream_t st) {
    if (Da <= 0 || Db <= 0) return cudaSuccess;
    const int grid = Db < sm_count * 8 ? Db : sm_count * 8;
    SV_DISPATCH_AMP(dtype, k_scatter_odd<A><<<grid, kThreads, 0, st>>>((const A *)lamc, (A *)cl, sa_s, sb_s, Da, Db));
    return cudaGetLastError();
}

cudaError_t launch_reduce_rows(const double *partials, int rows, int cols, double *out, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    k_reduce_rows<<<rows, kThreads, 0, st>>>(partials, cols, out);
    return cudaGetLastError();
}

}  // namespace svk
