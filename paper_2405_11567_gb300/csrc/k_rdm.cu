// k_rdm.cu -- spin-resolved one-particle density matrix
//     n_{pq,sigma} = <psi| a+_{p sigma} a_{q sigma} |psi>
// (Methodology, Strategy 2, equation for n_{pq,sigma}; Jordan-Wigner mapping of
// a+_{p sigma} a_{q sigma}).
//
// Elements (host list, one float64 (re, im) sum each):
//   kind 0  norm       sum_x |psi[x]|^2
//   kind 1  diagonal   sum_x |psi[x]|^2 x_P                     (P = 2p + sigma)
//   kind 2  p < q      sum_x conj(psi[x ^ m]) (-1)^popc(x & sm) psi[x] over x with Q
//                      occupied and P empty, m = {P, Q}, sm = bits strictly between
//                      P and Q (Jordan-Wigner sign of a+_P a_Q on x);
//                      n_{qp} = conj(n_{pq}).
// Sector-gather variant: one thread per XPT basis indices of the sector list;
// each element's per-thread sum is reduced across the warp with shuffles (in the
// state precision: at most 32 * XPT terms) and added in float64 by lane 0 into the
// warp's own shared-memory slot (no atomics), and the block adds its warps in a
// fixed order at the end: bit-identical reruns.
#include <cstring>
#include <vector>

#include "sv_device.cuh"
#include "sv_internal.h"

namespace svk {

struct RdmElem {
    uint32_t m, sm, want;  // contribute when (x & m) == want
    int kind;
};

template <typename R, int XPT>
__global__ void __launch_bounds__(kThreads)
k_rdm_gather(const cplx<R> *__restrict__ psi, const uint32_t *__restrict__ sector, uint32_t count,
             const RdmElem *__restrict__ el, int n_el, double *__restrict__ partial) {
    extern __shared__ double s_acc[];  // [kThreads/32][2 * n_el]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < (kThreads / 32) * 2 * n_el; i += kThreads) s_acc[i] = 0.0;
    __syncthreads();
    const uint32_t per_block = kThreads * XPT;
    for (uint32_t base = blockIdx.x * per_block; base < count; base += gridDim.x * per_block) {
        uint32_t x[XPT];
        bool ok[XPT];
        cplx<R> px[XPT];
        #pragma unroll
        for (int t = 0; t < XPT; ++t) {
            uint32_t r = base + t * kThreads + threadIdx.x;
            ok[t] = r < count;
            x[t] = ok[t] ? sector[r] : 0u;
            px[t] = ok[t] ? psi[x[t]] : mk<R>(0, 0);
        }
        for (int e = 0; e < n_el; ++e) {
            const RdmElem E = el[e];
            R re = 0, im = 0;
            #pragma unroll
            for (int t = 0; t < XPT; ++t) {
                if (!ok[t]) continue;
                if (E.kind == 2) {
                    if ((x[t] & E.m) != E.want) continue;
                    cplx<R> p = psi[x[t] ^ E.m];
                    R a = p.x * px[t].x + p.y * px[t].y;  // Re conj(p) psi_x
                    R b = p.x * px[t].y - p.y * px[t].x;  // Im conj(p) psi_x
                    if (__popc(x[t] & E.sm) & 1) { a = -a; b = -b; }
                    re += a;
                    im += b;
                } else if ((x[t] & E.m) == E.want) {
                    re += px[t].x * px[t].x + px[t].y * px[t].y;
                }
            }
            // warp sum in the state precision (32 x XPT terms), then float64 per warp
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                re += __shfl_down_sync(0xffffffffu, re, o);
                im += __shfl_down_sync(0xffffffffu, im, o);
            }
            if (lane == 0) {
                s_acc[warp * 2 * n_el + 2 * e] += (double)re;
                s_acc[warp * 2 * n_el + 2 * e + 1] += (double)im;
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * n_el; i += kThreads) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += s_acc[w * 2 * n_el + i];
        partial[(size_t)i * gridDim.x + blockIdx.x] = s;
    }
}

constexpr int kXptRdm = 8;

int rdm_gather_grid(uint64_t count, int sm_count) {
    uint64_t per_block = (uint64_t)kThreads * kXptRdm;
    uint64_t want = (count + per_block - 1) / per_block;
    uint64_t cap = (uint64_t)sm_count * 2;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

// Host list of elements for an n-qubit register (norm, n diagonals, then p<q pairs
// for alpha then beta).  Returns the count.
// Masks are mapped to the storage layout `perm`.
int rdm_elements(int n, const int *perm, std::vector<RdmElem> &out) {
    out.clear();
    out.push_back(RdmElem{0u, 0u, 0u, 0});
    for (int j = 0; j < n; ++j) out.push_back(RdmElem{1u << perm[j], 0u, 1u << perm[j], 1});
    const int N = n / 2;
    for (int s = 0; s < 2; ++s)
        for (int p = 0; p < N; ++p)
            for (int q = p + 1; q < N; ++q) {
                int P = 2 * p + s, Q = 2 * q + s;
                out.push_back(RdmElem{map_bits((1u << P) | (1u << Q), perm), map_bits(bits_between(P, Q), perm),
                                      1u << perm[Q], 2});
            }
    return (int)out.size();
}

// The element list serialised for upload.
int rdm_elements_bytes(int n, const int *perm, std::vector<uint8_t> &out) {
    std::vector<RdmElem> el;
    int cnt = rdm_elements(n, perm, el);
    out.resize(el.size() * sizeof(RdmElem));
    memcpy(out.data(), el.data(), out.size());
    return cnt;
}

// partial must hold 2 * n_el * grid doubles; layout [2 n_el][grid].
cudaError_t launch_rdm_gather(const void *psi, int dtype, const uint32_t *sector, uint64_t count,
                              const void *elems, int n_el, int grid, double *partial, cudaStream_t st) {
    size_t smem = sizeof(double) * (kThreads / 32) * 2 * n_el;
    if (dtype == SV_C64) {
        k_rdm_gather<float, kXptRdm><<<grid, kThreads, smem, st>>>(
            (const float2 *)psi, sector, (uint32_t)count, (const RdmElem *)elems, n_el, partial);
    } else {
        k_rdm_gather<double, kXptRdm><<<grid, kThreads, smem, st>>>(
            (const double2 *)psi, sector, (uint32_t)count, (const RdmElem *)elems, n_el, partial);
    }
    return cudaGetLastError();
}

}  // namespace svk
