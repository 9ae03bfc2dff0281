// k_expect.cu -- expectation value <psi|H|psi> and sigma = (H - c) psi.
//
// The energy of the second-quantised Hamiltonian (Fig. 1: the QPU/GPU returns
// <H>; Methodology, FCI energy functional) is evaluated group by group: the
// Pauli strings of the Jordan-Wigner Hamiltonian are grouped by their X-part
// (flip mask m), and the whole group is evaluated at a basis index x in closed
// form (sv_tables.cpp), so one pass over the masks serves every string of every
// group.
//
// Record-scan variant (this file, k_expect_gather): one thread per basis index
// of the (N_alpha, N_beta) sector list (every other amplitude of the state is
// identically zero: the reference and every excitation conserve both numbers).
// For its x the thread sums the diagonal element and every single and double
// mask group connected to x, gathering psi[x ^ m] from global memory.  The mask
// records are staged through shared memory in chunks shared by the block; each
// thread carries XPT basis indices so every staged record is used XPT times.
// Accumulation over masks is in the state precision; the energy and norm sums
// are float64, reduced per block and then in a fixed order.  Indices and masks
// are in the storage layout (the per-spin-orbital diagonal tables too).
//
// The default variant, string rows, lives in k_rows.cu.
#include "sv_device.cuh"
#include "sv_internal.h"

namespace svk {

template <typename R>
__device__ __forceinline__ double diag_shifted(uint32_t x, int n, const double *__restrict__ hdiag,
                                               const double *__restrict__ Jp, double e_shift) {
    double d = e_shift;
    for (uint32_t b = x; b; b &= b - 1u) {
        int k = __ffs(b) - 1;
        d += hdiag[k];
        for (uint32_t b2 = b & (b - 1u); b2; b2 &= b2 - 1u) {
            int l = __ffs(b2) - 1;
            d += Jp[k * n + l];
        }
    }
    return d;
}

// Value of a double-mask group at x (0 when x is not connected through it).
template <typename R>
__device__ __forceinline__ R double_value(uint32_t x, const DoubleRec<R> &r) {
    uint32_t t = x & r.m;
    if (__popc(t) != 2) return (R)0;
    uint32_t u = (t & r.b0) ? t : (r.m ^ t);  // the pair that contains q0
    uint32_t o = u ^ r.b0;
    R v = (o == r.b1) ? r.v[0] : ((o == r.b2) ? r.v[1] : r.v[2]);
    return (__popc(x & r.sm) & 1) ? -v : v;
}

constexpr int kChunk = 256;  // mask records staged per chunk

template <typename R, int XPT>
__global__ void __launch_bounds__(kThreads)
k_expect_gather(const cplx<R> *__restrict__ psi, cplx<R> *__restrict__ sigma,
                const uint32_t *__restrict__ sector, uint32_t count,
                const DoubleRec<R> *__restrict__ dbl, int n_dbl,
                const SingleRec<R> *__restrict__ sgl, int n_sgl, const R *__restrict__ W, int n,
                const double *__restrict__ hdiag, const double *__restrict__ Jp, double e_shift,
                double *__restrict__ partial) {
    __shared__ DoubleRec<R> s_rec[kChunk];
    __shared__ double red[2 * kThreads / 32];
    double e_acc = 0.0, n_acc = 0.0;
    const uint32_t per_block = kThreads * XPT;
    for (uint32_t base = blockIdx.x * per_block; base < count; base += gridDim.x * per_block) {
        uint32_t x[XPT];
        bool ok[XPT];
        cplx<R> px[XPT], acc[XPT];
        #pragma unroll
        for (int t = 0; t < XPT; ++t) {
            uint32_t r = base + t * kThreads + threadIdx.x;
            ok[t] = r < count;
            x[t] = ok[t] ? sector[r] : 0u;
            px[t] = ok[t] ? psi[x[t]] : mk<R>(0, 0);
            R d = ok[t] ? (R)diag_shifted<R>(x[t], n, hdiag, Jp, e_shift) : (R)0;
            acc[t] = mk<R>(d * px[t].x, d * px[t].y);
        }
        // single-excitation groups
        for (int i = 0; i < n_sgl; ++i) {
            const SingleRec<R> r = sgl[i];
            const R *w = W + (size_t)i * n;
            #pragma unroll
            for (int t = 0; t < XPT; ++t) {
                if (!ok[t] || __popc(x[t] & r.m) != 1) continue;
                R v = r.h;
                for (uint32_t b = x[t]; b; b &= b - 1u) v += w[__ffs(b) - 1];
                if (__popc(x[t] & r.sm) & 1) v = -v;
                cplx<R> p = psi[x[t] ^ r.m];
                acc[t].x += v * p.x;
                acc[t].y += v * p.y;
            }
        }
        // double-excitation groups, staged through shared memory
        for (int c0 = 0; c0 < n_dbl; c0 += kChunk) {
            int cn = min(kChunk, n_dbl - c0);
            __syncthreads();
            for (int i = threadIdx.x; i < cn; i += kThreads) s_rec[i] = dbl[c0 + i];
            __syncthreads();
            for (int i = 0; i < cn; ++i) {
                const DoubleRec<R> r = s_rec[i];
                #pragma unroll
                for (int t = 0; t < XPT; ++t) {
                    R v = double_value<R>(x[t], r);
                    if (!ok[t] || v == (R)0) continue;
                    cplx<R> p = psi[x[t] ^ r.m];
                    acc[t].x += v * p.x;
                    acc[t].y += v * p.y;
                }
            }
        }
        #pragma unroll
        for (int t = 0; t < XPT; ++t) {
            if (!ok[t]) continue;
            if (sigma) sigma[x[t]] = acc[t];
            e_acc += (double)px[t].x * (double)acc[t].x + (double)px[t].y * (double)acc[t].y;
            n_acc += (double)px[t].x * (double)px[t].x + (double)px[t].y * (double)px[t].y;
        }
    }
    block_sum2(e_acc, n_acc, red);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = e_acc;
        partial[gridDim.x + blockIdx.x] = n_acc;
    }
}

constexpr int kXptGather = 4;

int expect_gather_grid(uint64_t count, int sm_count) {
    uint64_t per_block = (uint64_t)kThreads * kXptGather;
    uint64_t want = (count + per_block - 1) / per_block;
    uint64_t cap = (uint64_t)sm_count * 4;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

// partial must hold 2 * grid doubles: [0, grid) energy parts, [grid, 2 grid) norm parts.
cudaError_t launch_expect_gather(const void *psi, void *sigma, int dtype, int n, const uint32_t *sector,
                                 uint64_t count, const DevTables &T, double e_shift, int grid,
                                 double *partial, cudaStream_t st) {
    if (dtype == SV_C64) {
        k_expect_gather<float, kXptGather><<<grid, kThreads, 0, st>>>(
            (const float2 *)psi, (float2 *)sigma, sector, (uint32_t)count,
            (const DoubleRec<float> *)T.dbl, T.n_dbl, (const SingleRec<float> *)T.sgl, T.n_sgl,
            (const float *)T.W, n, T.hdiag_s, T.Jp_s, e_shift, partial);
    } else {
        k_expect_gather<double, kXptGather><<<grid, kThreads, 0, st>>>(
            (const double2 *)psi, (double2 *)sigma, sector, (uint32_t)count,
            (const DoubleRec<double> *)T.dbl, T.n_dbl, (const SingleRec<double> *)T.sgl, T.n_sgl,
            (const double *)T.W, n, T.hdiag_s, T.Jp_s, e_shift, partial);
    }
    return cudaGetLastError();
}

}  // namespace svk
