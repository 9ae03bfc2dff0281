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
//   k_rdm_c      one block per density-matrix element
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

// Density-matrix elements.  kind 0: norm; kind 1: occupation of one spin-orbital
// (alpha string bit ma or beta string bit mb); kind 2: <psi|a+_P a_Q|psi> for a
// same-spin pair, from determinants with Q occupied and P empty.
struct SectElem {
    int kind;
    uint32_t sm;
    uint32_t ma, fa, mb, fb;
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_rdm_c(const cplx<R> *__restrict__ psi, const SectElem *__restrict__ el,
                                                    SectTabs T, double *__restrict__ out) {
    __shared__ double red[2 * kThreads / 32];
    const SectElem E = el[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double re = 0.0, im = 0.0;
    for (int Ib = warp; Ib < T.Db; Ib += nw) {
        const uint32_t b = T.strb[Ib];
        if ((b & E.mb) != E.fb) continue;
        const size_t rowI = (size_t)Ib * T.Da;
        const size_t rowJ = E.kind == 2 ? (size_t)T.rb[b ^ E.mb] * T.Da : rowI;
        const uint32_t xb = T.sb[Ib];
        R r = 0, i = 0;
        for (int Ia = lane; Ia < T.Da; Ia += 32) {
            const uint32_t a = T.stra[Ia];
            if ((a & E.ma) != E.fa) continue;
            const cplx<R> u = psi[rowI + Ia];
            if (E.kind != 2) {
                r += u.x * u.x + u.y * u.y;
                continue;
            }
            const cplx<R> p = psi[rowJ + T.ra[a ^ E.ma]];
            R ar = p.x * u.x + p.y * u.y, ai = p.x * u.y - p.y * u.x;  // conj(p) u
            if (par((T.sa[Ia] | xb) & E.sm)) { ar = -ar; ai = -ai; }
            r += ar;
            i += ai;
        }
        re += (double)r;
        im += (double)i;
    }
    block_sum2(re, im, red);
    if (threadIdx.x == 0) {
        out[2 * blockIdx.x] = re;
        out[2 * blockIdx.x + 1] = im;
    }
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

// Elements in the order norm, n occupations (spin-orbital j = 2p + sigma), then p<q pairs
// for alpha then beta -- the order sv_rdm1 unpacks.
int sect_rdm_elements(int n, std::vector<uint8_t> &out) {
    const int N = n / 2;
    std::vector<SectElem> el;
    el.push_back(SectElem{0, 0u, 0u, 0u, 0u, 0u});
    for (int j = 0; j < n; ++j) {
        const uint32_t bit = 1u << (j >> 1);
        if (j & 1) el.push_back(SectElem{1, 0u, 0u, 0u, bit, bit});
        else el.push_back(SectElem{1, 0u, bit, bit, 0u, 0u});
    }
    for (int s = 0; s < 2; ++s)
        for (int p = 0; p < N; ++p)
            for (int q = p + 1; q < N; ++q) {
                const int P = 2 * p + s, Q = 2 * q + s;
                const uint32_t m = (1u << p) | (1u << q), f = 1u << q;  // Q occupied, P empty
                SectElem e{2, bits_between(P, Q), 0u, 0u, 0u, 0u};
                if (s == 0) { e.ma = m; e.fa = f; } else { e.mb = m; e.fb = f; }
                el.push_back(e);
            }
    out.resize(el.size() * sizeof(SectElem));
    memcpy(out.data(), el.data(), out.size());
    return (int)el.size();
}

cudaError_t launch_rdm_c(const void *psi, int dtype, const void *elems, int n_el, const uint32_t *sa,
                         const uint32_t *sb, const uint16_t *stra, const uint16_t *strb, const uint16_t *ra,
                         const uint16_t *rb, int Da, int Db, double *out, cudaStream_t st) {
    SectTabs T = tabs(sa, sb, stra, strb, ra, rb, Da, Db);
    if (dtype == SV_C64) k_rdm_c<float><<<n_el, kThreads, 0, st>>>((const float2 *)psi, (const SectElem *)elems, T, out);
    else k_rdm_c<double><<<n_el, kThreads, 0, st>>>((const double2 *)psi, (const SectElem *)elems, T, out);
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
