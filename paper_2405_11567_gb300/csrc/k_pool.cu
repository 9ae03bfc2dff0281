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
// in a fixed order per block.
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

}  // namespace svk
