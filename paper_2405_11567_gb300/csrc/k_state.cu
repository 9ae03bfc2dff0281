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
};

static OpArgs to_args(const OpDesc &d) {
    OpArgs a;
    a.m = d.m; a.from = d.from; a.sm = d.sm;
    a.pos0 = d.pos[0]; a.pos1 = d.pos[1]; a.pos2 = d.pos[2]; a.pos3 = d.pos[3];
    a.c = d.c; a.s = d.s;
    return a;
}

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

template <typename R>
__global__ void k_set_basis(cplx<R> *psi, uint32_t x) {
    psi[x] = mk<R>(R(1), R(0));
}

// ---------------------------------------------------------------- forward rotation

template <typename R, int NB>
__global__ void __launch_bounds__(kThreads) k_rotate(cplx<R> *__restrict__ psi, uint32_t npairs, OpArgs a) {
    const R c = (R)a.c, sn = (R)a.s;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < npairs; k += stride) {
        uint32_t x = pair_index<NB>(k, a);
        uint32_t xp = x ^ a.m;
        R ss = (__popc(x & a.sm) & 1) ? -sn : sn;
        cplx<R> u = psi[x], v = psi[xp];
        psi[x] = mk<R>(c * u.x - ss * v.x, c * u.y - ss * v.y);
        psi[xp] = mk<R>(c * v.x + ss * u.x, c * v.y + ss * u.y);
    }
}

// ---------------------------------------------------------------- adjoint step

template <typename R, int NB>
__global__ void __launch_bounds__(kThreads) k_adjoint(cplx<R> *__restrict__ psi, cplx<R> *__restrict__ lam,
                                                      uint32_t npairs, OpArgs a, double *__restrict__ partial) {
    __shared__ double red[kThreads / 32];
    const R c = (R)a.c, sn = (R)a.s;
    const uint32_t stride = gridDim.x * blockDim.x;
    double acc = 0.0;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < npairs; k += stride) {
        uint32_t x = pair_index<NB>(k, a);
        uint32_t xp = x ^ a.m;
        const bool neg = __popc(x & a.sm) & 1;
        cplx<R> u = psi[x], v = psi[xp], lu = lam[x], lv = lam[xp];
        // <lambda|G psi> on the pair: conj(lu) * (-s v) + conj(lv) * (s u); real part
        R t = (lv.x * u.x + lv.y * u.y) - (lu.x * v.x + lu.y * v.y);
        acc += (double)(neg ? -t : t);
        // U^dagger: psi'[x] = c u + s sn v ; psi'[x'] = c v - s sn u
        R ss = neg ? -sn : sn;
        psi[x] = mk<R>(c * u.x + ss * v.x, c * u.y + ss * v.y);
        psi[xp] = mk<R>(c * v.x - ss * u.x, c * v.y - ss * u.y);
        lam[x] = mk<R>(c * lu.x + ss * lv.x, c * lu.y + ss * lv.y);
        lam[xp] = mk<R>(c * lv.x - ss * lu.x, c * lv.y - ss * lu.y);
    }
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
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

int rotate_grid(uint64_t npairs, int sm_count) {
    uint64_t want = (npairs + kThreads - 1) / kThreads;
    uint64_t cap = (uint64_t)sm_count * 8;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

cudaError_t launch_set_basis(void *psi, int dtype, uint32_t x, cudaStream_t st) {
    if (dtype == SV_C64) k_set_basis<float><<<1, 1, 0, st>>>((float2 *)psi, x);
    else k_set_basis<double><<<1, 1, 0, st>>>((double2 *)psi, x);
    return cudaGetLastError();
}

cudaError_t launch_rotate(void *psi, int dtype, int n, const OpDesc &d, int sm_count, cudaStream_t st) {
    OpArgs a = to_args(d);
    uint32_t npairs = (uint32_t)(1ull << (n - d.nbits));
    int grid = rotate_grid(npairs, sm_count);
    if (dtype == SV_C64) {
        if (d.nbits == 2) k_rotate<float, 2><<<grid, kThreads, 0, st>>>((float2 *)psi, npairs, a);
        else k_rotate<float, 4><<<grid, kThreads, 0, st>>>((float2 *)psi, npairs, a);
    } else {
        if (d.nbits == 2) k_rotate<double, 2><<<grid, kThreads, 0, st>>>((double2 *)psi, npairs, a);
        else k_rotate<double, 4><<<grid, kThreads, 0, st>>>((double2 *)psi, npairs, a);
    }
    return cudaGetLastError();
}

int adjoint_grid(int n, const OpDesc &d, int sm_count) {
    return rotate_grid(1ull << (n - d.nbits), sm_count);
}

cudaError_t launch_adjoint(void *psi, void *lam, int dtype, int n, const OpDesc &d, int grid,
                           double *partial, cudaStream_t st) {
    OpArgs a = to_args(d);
    uint32_t npairs = (uint32_t)(1ull << (n - d.nbits));
    if (dtype == SV_C64) {
        if (d.nbits == 2) k_adjoint<float, 2><<<grid, kThreads, 0, st>>>((float2 *)psi, (float2 *)lam, npairs, a, partial);
        else k_adjoint<float, 4><<<grid, kThreads, 0, st>>>((float2 *)psi, (float2 *)lam, npairs, a, partial);
    } else {
        if (d.nbits == 2) k_adjoint<double, 2><<<grid, kThreads, 0, st>>>((double2 *)psi, (double2 *)lam, npairs, a, partial);
        else k_adjoint<double, 4><<<grid, kThreads, 0, st>>>((double2 *)psi, (double2 *)lam, npairs, a, partial);
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce_rows(const double *partials, int rows, int cols, double *out, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    k_reduce_rows<<<rows, kThreads, 0, st>>>(partials, cols, out);
    return cudaGetLastError();
}

}  // namespace svk
