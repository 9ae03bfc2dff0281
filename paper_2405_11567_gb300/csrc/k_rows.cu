// k_rows.cu -- expectation value and sigma = (H - c) psi on the string-row view
// of the (N_alpha, N_beta) sector.
//
// Every basis index of the sector factorises into an alpha string a (the even
// bits) and a beta string b (the odd bits): x = spread_alpha(a) | spread_beta(b).
// The sector amplitudes are first gathered into a compact matrix
// C[rank(b)][rank(a)] (k_compact; 72 MB at 30 qubits in complex64, so it stays in
// L2), then one block per beta string ("row") and one thread per alpha string
// evaluates
//   sigma[x] = sum over the mask groups of H connected to x of <x^m|H|x> psi[x^m]
// with the groups taken by their flip pattern (the Jordan-Wigner Pauli strings of
// one X-mask summed in closed form, Methodology "Computational Details"):
//   diagonal          m = 0
//   alpha singles and alpha-alpha doubles   partner in the same row  (C[row][a'])
//   beta singles and beta-beta doubles      partner in another row, same column
//   alpha-beta doubles                      partner in another row at an
//                                           alpha-excited column
// Values: <x'|H|x> = v * <x'|T|x> with, for a single i->a,
// v = h_ai + sum_{k occupied} ([ai|kk] - [ak|ki]) and for a double (i<j -> a<b)
// v = [ai|bj] - [aj|bi]; [PQ|RS] = (pq|rs) delta(sP,sQ) delta(sR,sS).  The
// Jordan-Wigner signs are popcounts of x over the bits strictly between the
// indices: a single i->a gives (-1)^popc(x & between(i,a)); a double
// T = a+_a a+_b a_j a_i = -(a+_a a_j)(a+_b a_i) gives minus the product of the
// two single signs taken in that order.
//
// The energy and norm are float64 sums per row, reduced in a fixed order; the
// accumulation over the groups of one amplitude is in the state precision.
#include "sv_internal.h"
#include "sv_sigma.cuh"

namespace svk {

constexpr int kRowThreads = kThreads;

template <typename R>
struct RowArgs {
    SigmaTables<R> T;
    const cplx<R> *C;       // [Db][Da] compact sector amplitudes
    cplx<R> *lam;           // dense sigma output (nullable)
    const uint32_t *sa_s;   // [Da] alpha spread in the storage layout: addresses
    const uint32_t *sb_s;   // [Db]
    double *partial;        // [2][Db]
    int Db;
};

template <typename R>
__global__ void __launch_bounds__(kRowThreads) k_sigma_rows(RowArgs<R> A) {
    __shared__ double red[2 * kThreads / 32];
    const int Ib = blockIdx.x;
    const cplx<R> *row = A.C + (size_t)Ib * A.T.Da;
    double e_acc = 0.0, n_acc = 0.0;
    for (int Ia = threadIdx.x; Ia < A.T.Da; Ia += blockDim.x) {
        const cplx<R> c0 = row[Ia];
        const cplx<R> acc = sigma_at<R>(A.T, A.C, Ia, Ib, c0);
        if (A.lam) A.lam[A.sa_s[Ia] | A.sb_s[Ib]] = acc;
        e_acc += (double)c0.x * (double)acc.x + (double)c0.y * (double)acc.y;
        n_acc += (double)c0.x * (double)c0.x + (double)c0.y * (double)c0.y;
    }
    block_sum2(e_acc, n_acc, red);
    if (threadIdx.x == 0) {
        A.partial[Ib] = e_acc;
        A.partial[A.Db + Ib] = n_acc;
    }
}

// C[Ib][Ia] = psi[sa[Ia] | sb[Ib]]
template <typename R>
__global__ void __launch_bounds__(kThreads) k_compact(const cplx<R> *__restrict__ psi, cplx<R> *__restrict__ C,
                                                      const uint32_t *__restrict__ sa, const uint32_t *__restrict__ sb,
                                                      int Da, uint64_t total) {
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const int Ib = (int)(t / Da), Ia = (int)(t % Da);
        C[t] = psi[sa[Ia] | sb[Ib]];
    }
}

cudaError_t launch_compact(const void *psi, void *C, int dtype, const uint32_t *sa, const uint32_t *sb, int Da,
                           int Db, int sm_count, cudaStream_t st) {
    uint64_t total = (uint64_t)Da * Db;
    uint64_t want = (total + kThreads - 1) / kThreads;
    uint64_t cap = (uint64_t)sm_count * 16;
    int grid = (int)(want < cap ? (want ? want : 1) : cap);
    if (dtype == SV_C64)
        k_compact<float><<<grid, kThreads, 0, st>>>((const float2 *)psi, (float2 *)C, sa, sb, Da, total);
    else
        k_compact<double><<<grid, kThreads, 0, st>>>((const double2 *)psi, (double2 *)C, sa, sb, Da, total);
    return cudaGetLastError();
}

// Device pointers of the string-row tables (built by the host in sv_api.cu).
struct RowTables {
    const uint32_t *sa, *sb, *sa_s, *sb_s;
    const uint16_t *stra, *strb, *ra, *rb;
    const void *eri, *hm, *Dt, *Jt;
    int N, Da, Db;
};

template <typename R>
static RowArgs<R> row_args(const void *C, void *lam, int n, const RowTables &T, const double *hdiag, const double *Jp,
                           double e_shift, double *partial) {
    RowArgs<R> A;
    A.T.sa = T.sa; A.T.sb = T.sb; A.T.stra = T.stra; A.T.strb = T.strb; A.T.ra = T.ra; A.T.rb = T.rb;
    A.T.eri = (const R *)T.eri; A.T.hm = (const R *)T.hm; A.T.Dt = (const R *)T.Dt; A.T.Jt = (const R *)T.Jt;
    A.T.hdiag = hdiag; A.T.Jp = Jp; A.T.e_shift = e_shift;
    A.T.N = T.N; A.T.n = n; A.T.Da = T.Da; A.T.maskN = (1u << T.N) - 1u;
    A.C = (const cplx<R> *)C; A.lam = (cplx<R> *)lam; A.sa_s = T.sa_s; A.sb_s = T.sb_s;
    A.partial = partial; A.Db = T.Db;
    return A;
}

cudaError_t launch_sigma_rows(const void *C, void *lam, int dtype, int n, const RowTables &T, const double *hdiag,
                              const double *Jp, double e_shift, double *partial, cudaStream_t st) {
    if (dtype == SV_C64) {
        k_sigma_rows<float><<<T.Db, kRowThreads, 0, st>>>(row_args<float>(C, lam, n, T, hdiag, Jp, e_shift, partial));
    } else {
        k_sigma_rows<double><<<T.Db, kRowThreads, 0, st>>>(row_args<double>(C, lam, n, T, hdiag, Jp, e_shift, partial));
    }
    return cudaGetLastError();
}

}  // namespace svk
