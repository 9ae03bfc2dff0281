// k_pool.cu -- ADAPT-VQE operator screening ("Computational Details": ADAPT-VQE
// grows the ansatz one pool operator at a time): for the current state psi and
// every pool operator G_k = T_k - T_k^dagger, the energy gradient of appending
// exp(theta G_k) at theta = 0,
//     g_k = 2 Re <psi| H G_k |psi> = 2 Re <lambda| G_k psi>,  lambda = (H - c) psi
// (c drops out: Re <psi|G_k psi> = 0 for anti-Hermitian G_k).
//
// Both psi and lambda are read from the compact string-row matrices
// C[rank(b)][rank(a)] (L2-resident), so one block per pool operator visits the
// operator's "from" determinants row by row: a warp takes a beta string whose bits
// on the operator's beta mask equal its "from" pattern, its lanes take the alpha
// strings that match on the alpha mask, and each pair (x, x') adds
// s(x) (Re conj(lambda[x']) psi[x] - Re conj(lambda[x]) psi[x']) in float64, reduced
// in a fixed order per block (k_pool_grad, the string scan).  k_pool_grad_l visits
// the same pairs from per-operator pair lists, reading psi and lambda interleaved.
#include "sv_check.cuh"
#include "sv_internal.h"
#include "sv_sigma.cuh"

namespace svk {

struct PoolOp {
    uint32_t sm;          // sign mask (qubit space); 0 for qubit excitations
    uint16_t ma, fa;      // alpha-string flip mask and "from" pattern
    uint16_t mb, fb;      // beta-string flip mask and "from" pattern
};

template <typename A>
__global__ void __launch_bounds__(kThreads)
k_pool_grad(const A *__restrict__ C, const A *__restrict__ L, const PoolOp *__restrict__ ops,
            const uint32_t *__restrict__ sa, const uint32_t *__restrict__ sb, const uint16_t *__restrict__ stra,
            const uint16_t *__restrict__ strb, const uint16_t *__restrict__ ra, const uint16_t *__restrict__ rb,
            int Da, int Db, double *__restrict__ out) {
    using R = real_of<A>;
    __shared__ double red[kThreads / 32];
    const PoolOp op = ops[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double acc = 0.0;
    for (int Ib = warp; Ib < Db; Ib += nw) {
        const uint32_t b = strb[Ib];
        if ((b & op.mb) != op.fb) continue;
        const int Jb = rb[b ^ op.mb];
        const uint32_t xb = sb[Ib];
        R t = 0;
        for (int Ia = lane; Ia < Da; Ia += 32) {
            const uint32_t a = stra[Ia];
            if ((a & op.ma) != op.fa) continue;
            const int Ja = ra[a ^ op.ma];
            const size_t I = (size_t)Ib * Da + Ia, J = (size_t)Jb * Da + Ja;
            const A u = C[I], v = C[J], lu = L[I], lv = L[J];
            const R ti = re_dot(lv, u) - re_dot(lu, v);
            t += par((sa[Ia] | xb) & op.sm) ? -ti : ti;
        }
        acc += (double)t;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// Interleaved compact amplitudes and sigma: CL[2 i] = C[i], CL[2 i + 1] = L[i], so one
// aligned load of 2 sizeof(A) bytes (one 32-byte sector at most) reads both at a
// determinant.
template <typename A>
__device__ __forceinline__ void ld_pair(const A *p, A &c, A &l) {
    c = p[0];
    l = p[1];
}
template <>
__device__ __forceinline__ void ld_pair<float2>(const float2 *p, float2 &c, float2 &l) {
    const float4 v = *(const float4 *)p;
    c = make_float2(v.x, v.y);
    l = make_float2(v.z, v.w);
}
template <>
__device__ __forceinline__ void ld_pair<float>(const float *p, float &c, float &l) {
    const float2 v = *(const float2 *)p;
    c = v.x;
    l = v.y;
}
template <>
__device__ __forceinline__ void ld_pair<double>(const double *p, double &c, double &l) {
    const double2 v = *(const double2 *)p;
    c = v.x;
    l = v.y;
}

template <typename A>
__global__ void __launch_bounds__(kThreads) k_interleave(const A *__restrict__ C, const A *__restrict__ L,
                                                         A *__restrict__ CL, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        CL[2 * i] = C[i];
        CL[2 * i + 1] = L[i];
    }
}

// Screening over the pool's pair lists (the lists the sector rotations use, built
// once per pool by k_build_lists): block k takes operator k's pairs (beta entry r,
// alpha entry i) in the flattened order r na + i, thread t the pairs t, t + T, ...
// (T = blockDim.x), four at a time so that their loads are in flight together.  Each
// thread sums kPoolFlush pairs in the state precision before adding them to its
// float64 sum; then a fixed-order block reduction.  Only the pairs of the operator
// are visited (C(N - |m|, n - |f|) per spin), not every string.
constexpr int kPoolFlush = 32;

template <typename A>
__global__ void __launch_bounds__(kThreads) k_pool_grad_l(const A *__restrict__ CL, const uint32_t *__restrict__ lists,
                                                          const int4 *__restrict__ info, int Da, int Db,
                                                          double *__restrict__ out) {
    using R = real_of<A>;
    __shared__ double red[kThreads / 32];
    const int4 li = info[blockIdx.x];  // alpha offset, alpha length, beta offset, beta length
    const uint32_t *al = lists + li.x, *bl = lists + li.z;
    const int na = li.y, nb = li.w;
    double acc = 0.0;
    if (na > 0 && nb > 0) {
        const int dr = (int)blockDim.x / na, di = (int)blockDim.x % na;
        int r = (int)threadIdx.x / na, i = (int)threadIdx.x % na;
        while (r < nb) {
            R t = 0;
            #pragma unroll 1
            for (int u = 0; u < kPoolFlush / 4 && r < nb; ++u) {
                size_t I[4], J[4];
                uint32_t neg[4];
                bool ok[4];
                #pragma unroll
                for (int v = 0; v < 4; ++v) {
                    ok[v] = r < nb;
                    const uint32_t eb = ok[v] ? bl[r] : 0u, ea = ok[v] ? al[i] : 0u;  // 0: rank 0, in bounds
                    I[v] = (size_t)(eb & 0x7FFFu) * Da + (ea & 0x7FFFu);
                    J[v] = (size_t)(eb >> 16) * Da + (ea >> 16);
                    neg[v] = (ea ^ eb) & 0x8000u;
                    if (!(SV_IN_RANGE(I[v], (size_t)Da * Db, kChkPair) && SV_IN_RANGE(J[v], (size_t)Da * Db, kChkPair))) {
                        ok[v] = false;  // checked build: skip the pair
                        I[v] = J[v] = 0;
                    }
                    r += dr;
                    i += di;
                    if (i >= na) {
                        i -= na;
                        ++r;
                    }
                }
                A c0[4], l0[4], c1[4], l1[4];
                #pragma unroll
                for (int v = 0; v < 4; ++v) {
                    ld_pair<A>(CL + 2 * I[v], c0[v], l0[v]);
                    ld_pair<A>(CL + 2 * J[v], c1[v], l1[v]);
                }
                #pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const R ti = re_dot(l1[v], c0[v]) - re_dot(l0[v], c1[v]);
                    if (ok[v]) t += neg[v] ? -ti : ti;
                }
            }
            acc += (double)t;
        }
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// Host descriptor of a pool operator from its qubit-space masks.
void pool_op_from(const OpDesc &d, int N, void *dst) {
    PoolOp p;
    p.sm = d.sm;
    uint32_t ma = 0, fa = 0, mb = 0, fb = 0;
    for (int q = 0; q < N; ++q) {
        if ((d.m >> (2 * q)) & 1u) ma |= 1u << q;
        if ((d.from >> (2 * q)) & 1u) fa |= 1u << q;
        if ((d.m >> (2 * q + 1)) & 1u) mb |= 1u << q;
        if ((d.from >> (2 * q + 1)) & 1u) fb |= 1u << q;
    }
    p.ma = (uint16_t)ma; p.fa = (uint16_t)fa; p.mb = (uint16_t)mb; p.fb = (uint16_t)fb;
    *(PoolOp *)dst = p;
}

size_t pool_op_bytes() { return sizeof(PoolOp); }

cudaError_t launch_pool_grad(const void *C, const void *L, int dtype, const void *ops, int n_ops, const uint32_t *sa,
                             const uint32_t *sb, const uint16_t *stra, const uint16_t *strb, const uint16_t *ra,
                             const uint16_t *rb, int Da, int Db, double *out, cudaStream_t st) {
    if (n_ops <= 0) return cudaSuccess;
    SV_DISPATCH_AMP(dtype, k_pool_grad<A><<<n_ops, kThreads, 0, st>>>((const A *)C, (const A *)L, (const PoolOp *)ops,
                                                                      sa, sb, stra, strb, ra, rb, Da, Db, out));
    return cudaGetLastError();
}

// CL: 2 count amplitudes.
cudaError_t launch_interleave(const void *C, const void *L, int dtype, void *CL, size_t count, int sm_count,
                              cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    size_t grid = (count + kThreads - 1) / kThreads;
    if (grid > (size_t)sm_count * 8) grid = (size_t)sm_count * 8;
    SV_DISPATCH_AMP(dtype, k_interleave<A><<<(unsigned)grid, kThreads, 0, st>>>((const A *)C, (const A *)L, (A *)CL,
                                                                               count));
    return cudaGetLastError();
}

// info: n_ops int4 records (alpha offset, alpha length, beta offset, beta length) into lists.
cudaError_t launch_pool_grad_l(const void *CL, int dtype, const uint32_t *lists, const int *info, int n_ops, int Da,
                               int Db, double *out, cudaStream_t st) {
    if (n_ops <= 0) return cudaSuccess;
    SV_DISPATCH_AMP(dtype, k_pool_grad_l<A><<<n_ops, kThreads, 0, st>>>((const A *)CL, lists, (const int4 *)info, Da,
                                                                         Db, out));
    return cudaGetLastError();
}

// This unit's check word (checked build), for sv_check_status.
SV_CHECK_READER(check_word_pool)

}  // namespace svk
