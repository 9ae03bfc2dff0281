// k_sector.cu -- kernels for sector storage: the state held as only the
// amplitudes of its (N_alpha, N_beta) sector, in the string-row order
// C[rank(b)][rank(a)] (x = spread_alpha(a) | spread_beta(b)); 9,018,009 amplitudes
// (72 MB in complex64) at 30 qubits and 10 electrons instead of 2^30.  Every
// operator of the method conserves both electron numbers, so nothing outside the
// sector is ever needed.
//
// An excitation (or a density-matrix element a+_p a_q) acts on the determinants
// whose alpha string matches its alpha "from" pattern and whose beta string
// matches its beta pattern; its partner is found through the string ranks.  The
// kernels below give each block one beta string (row) and its threads the alpha
// strings of that row, so a launch touches only the pairs it rotates:
//   k_rotate_c   psi'[x] = c psi[x] - s sn psi[x'],  psi'[x'] = c psi[x'] + s sn psi[x]
//   k_adjoint_c  g += s (Re conj(lam[x']) psi[x] - Re conj(lam[x]) psi[x']), then U^dagger
//                on psi and lambda (float64 per block, fixed-order sums)
//   k_rdm_rows   one block per beta string: every density-matrix element's share
// with s = (-1)^popc(x & sm), the Jordan-Wigner sign (sm = 0 for qubit
// excitations).
#include <cstring>
#include <vector>

#include "sv_internal.h"
#include "sv_sigma.cuh"

namespace svk {

struct SectOp {
    uint32_t sm;
    uint32_t ma, fa, mb, fb;  // alpha / beta string flip masks and "from" patterns
    double c, s;
};

struct SectTabs {
    const uint32_t *sa, *sb;       // qubit-space spreads
    const uint16_t *stra, *strb;   // strings
    const uint16_t *ra, *rb;       // ranks
    int Da, Db;
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_rotate_c(cplx<R> *__restrict__ psi, SectOp op, SectTabs T) {
    const R c = (R)op.c, sn = (R)op.s;
    for (int Ib = blockIdx.x; Ib < T.Db; Ib += gridDim.x) {
        const uint32_t b = T.strb[Ib];
        if ((b & op.mb) != op.fb) continue;
        const size_t rowI = (size_t)Ib * T.Da, rowJ = (size_t)T.rb[b ^ op.mb] * T.Da;
        const uint32_t xb = T.sb[Ib];
        for (int Ia = threadIdx.x; Ia < T.Da; Ia += blockDim.x) {
            const uint32_t a = T.stra[Ia];
            if ((a & op.ma) != op.fa) continue;
            const size_t I = rowI + Ia, J = rowJ + T.ra[a ^ op.ma];
            const R ss = par((T.sa[Ia] | xb) & op.sm) ? -sn : sn;
            const cplx<R> u = psi[I], v = psi[J];
            psi[I] = mk<R>(c * u.x - ss * v.x, c * u.y - ss * v.y);
            psi[J] = mk<R>(c * v.x + ss * u.x, c * v.y + ss * u.y);
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_adjoint_c(cplx<R> *__restrict__ psi, cplx<R> *__restrict__ lam, SectOp op,
                                                        SectTabs T, double *__restrict__ partial) {
    __shared__ double red[kThreads / 32];
    const R c = (R)op.c, sn = (R)op.s;
    double acc = 0.0;
    for (int Ib = blockIdx.x; Ib < T.Db; Ib += gridDim.x) {
        const uint32_t b = T.strb[Ib];
        if ((b & op.mb) != op.fb) continue;
        const size_t rowI = (size_t)Ib * T.Da, rowJ = (size_t)T.rb[b ^ op.mb] * T.Da;
        const uint32_t xb = T.sb[Ib];
        R t = 0;
        for (int Ia = threadIdx.x; Ia < T.Da; Ia += blockDim.x) {
            const uint32_t a = T.stra[Ia];
            if ((a & op.ma) != op.fa) continue;
            const size_t I = rowI + Ia, J = rowJ + T.ra[a ^ op.ma];
            const bool neg = par((T.sa[Ia] | xb) & op.sm);
            const cplx<R> u = psi[I], v = psi[J], lu = lam[I], lv = lam[J];
            const R ti = (lv.x * u.x + lv.y * u.y) - (lu.x * v.x + lu.y * v.y);
            t += neg ? -ti : ti;
            const R ss = neg ? -sn : sn;
            psi[I] = mk<R>(c * u.x + ss * v.x, c * u.y + ss * v.y);
            psi[J] = mk<R>(c * v.x - ss * u.x, c * v.y - ss * u.y);
            lam[I] = mk<R>(c * lu.x + ss * lv.x, c * lu.y + ss * lv.y);
            lam[J] = mk<R>(c * lv.x - ss * lu.x, c * lv.y - ss * lu.y);
        }
        acc += (double)t;
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Density matrix by rows: a block takes beta strings (rows) Ib = blockIdx.x,
// blockIdx.x + gridDim.x, ...; for each row its warps sum, in the state precision,
//   norm and alpha occupations   sum_a |C[b][a]|^2 (a_p)
//   beta occupations             the row norm when b holds p
//   alpha pairs p < q            sum over a with q in a, p not in a of
//                                conj(C[b][a']) C[b][a] (-1)^popc(x & between(2p, 2q)), a' = a - q + p
//   beta pairs p < q (b holds q, not p)
//                                sum_a conj(C[b'][a]) C[b][a] (-1)^popc(x & between(2p+1, 2q+1))
// (x = spread(a) | spread(b)), in the element order norm, n occupations
// (j = 2p + sigma), alpha pairs, beta pairs.  Each warp's sum goes to its own
// shared slot; after each row the block adds the slots in warp order into float64
// running sums, written to partial[e][blockIdx.x] at the end: fixed-order sums.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_rdm_rows(const cplx<R> *__restrict__ C, SectTabs T, int N,
                                                       double *__restrict__ partial) {
    extern __shared__ double rdm_s[];  // [2 n_el] running sums, then [kThreads/32][2 n_el] warp slots
    const int n = 2 * N, npair = N * (N - 1) / 2, n_el = 1 + n + 2 * npair, W = 2 * n_el;
    double *acc = rdm_s, *slot = rdm_s + W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *my = slot + warp * W;
    for (int i = threadIdx.x; i < W; i += blockDim.x) acc[i] = 0.0;
    const uint32_t maskN = (1u << N) - 1u;
    for (int Ib = blockIdx.x; Ib < T.Db; Ib += gridDim.x) {
        const uint32_t b = T.strb[Ib], xb = T.sb[Ib];
        const cplx<R> *row = C + (size_t)Ib * T.Da;
        // norm and alpha occupations
        R nrm = 0, occ[16];
        #pragma unroll
        for (int p = 0; p < 16; ++p) occ[p] = 0;
        for (int Ia = threadIdx.x; Ia < T.Da; Ia += blockDim.x) {
            const cplx<R> c = row[Ia];
            const R w = c.x * c.x + c.y * c.y;
            const uint32_t a = T.stra[Ia];
            nrm += w;
            #pragma unroll
            for (int p = 0; p < 16; ++p)
                if ((a >> p) & 1u) occ[p] += w;
        }
        nrm = warp_sum(nrm);
        if (lane == 0) {
            my[0] = (double)nrm;
            my[1] = 0.0;
        }
        #pragma unroll
        for (int p = 0; p < 16; ++p) {
            if (p >= N) break;
            const R s = warp_sum(occ[p]);
            if (lane == 0) {
                my[2 * (1 + 2 * p)] = (double)s;
                my[2 * (1 + 2 * p) + 1] = 0.0;
                my[2 * (2 + 2 * p)] = ((b >> p) & 1u) ? (double)nrm : 0.0;
                my[2 * (2 + 2 * p) + 1] = 0.0;
            }
        }
        // alpha pairs (same row) and beta pairs (row b')
        int e = 1 + n;
        for (int s = 0; s < 2; ++s)
            for (int p = 0; p < N; ++p)
                for (int q = p + 1; q < N; ++q, ++e) {
                    const uint32_t m = (1u << p) | (1u << q), f = 1u << q;
                    const uint32_t bm = between(2 * p + s, 2 * q + s);
                    R re = 0, im = 0;
                    if (s == 0) {
                        for (int Ia = threadIdx.x; Ia < T.Da; Ia += blockDim.x) {
                            const uint32_t a = T.stra[Ia];
                            if ((a & m) != f) continue;
                            const cplx<R> u = row[Ia], v = row[T.ra[a ^ m]];
                            R ar = v.x * u.x + v.y * u.y, ai = v.x * u.y - v.y * u.x;  // conj(v) u
                            if (par((T.sa[Ia] | xb) & bm)) { ar = -ar; ai = -ai; }
                            re += ar;
                            im += ai;
                        }
                    } else if ((b & m) == f) {
                        const cplx<R> *row2 = C + (size_t)T.rb[b ^ m] * T.Da;
                        for (int Ia = threadIdx.x; Ia < T.Da; Ia += blockDim.x) {
                            const cplx<R> u = row[Ia], v = row2[Ia];
                            R ar = v.x * u.x + v.y * u.y, ai = v.x * u.y - v.y * u.x;
                            if (par((T.sa[Ia] | xb) & bm)) { ar = -ar; ai = -ai; }
                            re += ar;
                            im += ai;
                        }
                    }
                    re = warp_sum(re);
                    im = warp_sum(im);
                    if (lane == 0) {
                        my[2 * e] = (double)re;
                        my[2 * e + 1] = (double)im;
                    }
                }
        (void)maskN;
        __syncthreads();
        for (int i = threadIdx.x; i < W; i += blockDim.x) {
            double t = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) t += slot[w * W + i];
            acc[i] += t;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < W; i += blockDim.x) partial[(size_t)i * gridDim.x + blockIdx.x] = acc[i];
}

// out[i] = C[idx[i]] or 0 when idx[i] is 0xFFFFFFFF (a basis state outside the sector)
template <typename R>
__global__ void k_gather_c(const cplx<R> *__restrict__ psi, const uint32_t *__restrict__ idx, int count,
                           cplx<R> *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        out[i] = idx[i] == 0xFFFFFFFFu ? mk<R>(0, 0) : psi[idx[i]];
}

// ---------------------------------------------------------------- launchers

static SectTabs tabs(const uint32_t *sa, const uint32_t *sb, const uint16_t *stra, const uint16_t *strb,
                     const uint16_t *ra, const uint16_t *rb, int Da, int Db) {
    SectTabs t;
    t.sa = sa; t.sb = sb; t.stra = stra; t.strb = strb; t.ra = ra; t.rb = rb; t.Da = Da; t.Db = Db;
    return t;
}

// Alpha / beta string parts of a qubit-space op.
void sect_op_from(const OpDesc &d, int N, void *dst) {
    SectOp o;
    o.sm = d.sm;
    o.ma = o.fa = o.mb = o.fb = 0;
    for (int q = 0; q < N; ++q) {
        if ((d.m >> (2 * q)) & 1u) o.ma |= 1u << q;
        if ((d.from >> (2 * q)) & 1u) o.fa |= 1u << q;
        if ((d.m >> (2 * q + 1)) & 1u) o.mb |= 1u << q;
        if ((d.from >> (2 * q + 1)) & 1u) o.fb |= 1u << q;
    }
    o.c = d.c;
    o.s = d.s;
    *(SectOp *)dst = o;
}

size_t sect_op_bytes() { return sizeof(SectOp); }

int sector_grid(int Db, int sm_count) { return Db < sm_count * 8 ? Db : sm_count * 8; }

cudaError_t launch_rotate_c(void *psi, int dtype, const void *op, const uint32_t *sa, const uint32_t *sb,
                            const uint16_t *stra, const uint16_t *strb, const uint16_t *ra, const uint16_t *rb, int Da,
                            int Db, int grid, cudaStream_t st) {
    SectTabs T = tabs(sa, sb, stra, strb, ra, rb, Da, Db);
    const SectOp o = *(const SectOp *)op;
    if (dtype == SV_C64) k_rotate_c<float><<<grid, kThreads, 0, st>>>((float2 *)psi, o, T);
    else k_rotate_c<double><<<grid, kThreads, 0, st>>>((double2 *)psi, o, T);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_c(void *psi, void *lam, int dtype, const void *op, const uint32_t *sa, const uint32_t *sb,
                             const uint16_t *stra, const uint16_t *strb, const uint16_t *ra, const uint16_t *rb,
                             int Da, int Db, int grid, double *partial, cudaStream_t st) {
    SectTabs T = tabs(sa, sb, stra, strb, ra, rb, Da, Db);
    const SectOp o = *(const SectOp *)op;
    if (dtype == SV_C64) k_adjoint_c<float><<<grid, kThreads, 0, st>>>((float2 *)psi, (float2 *)lam, o, T, partial);
    else k_adjoint_c<double><<<grid, kThreads, 0, st>>>((double2 *)psi, (double2 *)lam, o, T, partial);
    return cudaGetLastError();
}

int rdm_rows_elements(int n) { return 1 + n + (n / 2) * (n / 2 - 1); }

int rdm_rows_grid(int Db, int sm_count) { return Db < 4 * sm_count ? Db : 4 * sm_count; }

// partial: [2 n_el][grid] doubles (n_el = rdm_rows_elements(n)), reduced by launch_reduce_rows.
cudaError_t launch_rdm_rows(const void *C, int dtype, int n, const uint32_t *sa, const uint32_t *sb,
                            const uint16_t *stra, const uint16_t *strb, const uint16_t *ra, const uint16_t *rb, int Da,
                            int Db, int grid, double *partial, cudaStream_t st) {
    SectTabs T = tabs(sa, sb, stra, strb, ra, rb, Da, Db);
    const size_t smem = sizeof(double) * 2 * rdm_rows_elements(n) * (1 + kThreads / 32);
    cudaError_t e;
    if (dtype == SV_C64) {
        e = cudaFuncSetAttribute(k_rdm_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_rdm_rows<float><<<grid, kThreads, smem, st>>>((const float2 *)C, T, n / 2, partial);
    } else {
        e = cudaFuncSetAttribute(k_rdm_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_rdm_rows<double><<<grid, kThreads, smem, st>>>((const double2 *)C, T, n / 2, partial);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather_c(const void *psi, int dtype, const uint32_t *idx, int count, void *out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    int grid = (count + kThreads - 1) / kThreads;
    if (grid > 1024) grid = 1024;
    if (dtype == SV_C64) k_gather_c<float><<<grid, kThreads, 0, st>>>((const float2 *)psi, idx, count, (float2 *)out);
    else k_gather_c<double><<<grid, kThreads, 0, st>>>((const double2 *)psi, idx, count, (double2 *)out);
    return cudaGetLastError();
}

}  // namespace svk
