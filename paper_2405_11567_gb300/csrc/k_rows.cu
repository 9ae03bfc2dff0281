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
#include "sv_device.cuh"
#include "sv_internal.h"

namespace svk {

constexpr int kRowThreads = kThreads;

__device__ __forceinline__ uint32_t between(int a, int b) {
    int lo = min(a, b), hi = max(a, b);
    return ((1u << hi) - 1u) & ~((2u << lo) - 1u);
}

__device__ __forceinline__ int par(uint32_t v) { return __popc(v) & 1; }

template <typename R>
struct RowArgs {
    const cplx<R> *C;       // [Db][Da] compact sector amplitudes
    cplx<R> *lam;           // dense sigma output (nullable)
    const uint32_t *sa;     // [Da] alpha spread (even bits)
    const uint32_t *sb;     // [Db] beta spread (odd bits)
    const uint16_t *stra;   // [Da] alpha strings
    const uint16_t *strb;   // [Db] beta strings
    const uint16_t *ra;     // [2^N] rank of an alpha string (valid strings only)
    const uint16_t *rb;     // [2^N] rank of a beta string
    const R *eri;           // [N^4] spatial (pq|rs)
    const R *hm;            // [N^2] spatial h_pq
    const R *Dt;            // [N^3] (qp|kk) - (qk|kp): same-spin occupied k
    const R *Jt;            // [N^3] (qp|kk): opposite-spin occupied k
    const double *hdiag;    // [n] h_kk per spin-orbital
    const double *Jp;       // [n][n] [kk|ll] - [kl|lk]
    double e_shift;         // E_nuc - c
    double *partial;        // [2][Db]
    int N, n, Da, Db;
    uint32_t maskN;
};

// v for a single p->q of one spin with same-spin string `own` and opposite-spin
// string `other`: h_qp + sum_{k in own} ((qp|kk) - (qk|kp)) + sum_{k in other} (qp|kk).
template <typename R>
__device__ __forceinline__ R single_value(const RowArgs<R> &A, int p, int q, uint32_t own, uint32_t other) {
    const int N = A.N;
    const R *dt = A.Dt + (q * N + p) * N;
    const R *jt = A.Jt + (q * N + p) * N;
    R v = A.hm[q * N + p];
    for (uint32_t o = own; o; o &= o - 1u) v += dt[__ffs(o) - 1];
    for (uint32_t o = other; o; o &= o - 1u) v += jt[__ffs(o) - 1];
    return v;
}

template <typename R>
__device__ __forceinline__ R eri4(const RowArgs<R> &A, int p, int q, int r, int s) {
    const int N = A.N;
    return A.eri[((p * N + q) * N + r) * N + s];
}

template <typename R>
__device__ __forceinline__ void fma_c(cplx<R> &acc, R v, const cplx<R> &c) {
    acc.x += v * c.x;
    acc.y += v * c.y;
}

template <typename R>
__global__ void __launch_bounds__(kRowThreads) k_sigma_rows(RowArgs<R> A) {
    __shared__ double red[2 * kThreads / 32];
    const int Ib = blockIdx.x;
    const int N = A.N, Da = A.Da;
    const uint32_t b = A.strb[Ib], xb = A.sb[Ib];
    const uint32_t eb = ~b & A.maskN;
    const cplx<R> *row = A.C + (size_t)Ib * Da;
    double e_acc = 0.0, n_acc = 0.0;
    for (int Ia = threadIdx.x; Ia < Da; Ia += blockDim.x) {
        const uint32_t a = A.stra[Ia], xa = A.sa[Ia], x = xa | xb;
        const uint32_t ea = ~a & A.maskN;
        const cplx<R> c0 = row[Ia];
        // diagonal (float64), including E_nuc - c
        double d = A.e_shift;
        for (uint32_t o = x; o; o &= o - 1u) {
            int k = __ffs(o) - 1;
            d += A.hdiag[k];
            for (uint32_t o2 = o & (o - 1u); o2; o2 &= o2 - 1u) d += A.Jp[k * A.n + __ffs(o2) - 1];
        }
        cplx<R> acc = mk<R>((R)d * c0.x, (R)d * c0.y);
        // alpha singles p -> q (partner in this row)
        for (uint32_t o = a; o; o &= o - 1u) {
            const int p = __ffs(o) - 1;
            for (uint32_t e = ea; e; e &= e - 1u) {
                const int q = __ffs(e) - 1;
                R v = single_value<R>(A, p, q, a, b);
                if (par(x & between(2 * p, 2 * q))) v = -v;
                fma_c<R>(acc, v, row[A.ra[a ^ (1u << p) ^ (1u << q)]]);
            }
        }
        // alpha-alpha doubles (p1<p2 occupied -> q1<q2 empty), partner in this row
        for (uint32_t o = a; o; o &= o - 1u) {
            const int p1 = __ffs(o) - 1;
            for (uint32_t o2 = o & (o - 1u); o2; o2 &= o2 - 1u) {
                const int p2 = __ffs(o2) - 1;
                for (uint32_t e = ea; e; e &= e - 1u) {
                    const int q1 = __ffs(e) - 1;
                    for (uint32_t e2 = e & (e - 1u); e2; e2 &= e2 - 1u) {
                        const int q2 = __ffs(e2) - 1;
                        R v = eri4<R>(A, q1, p1, q2, p2) - eri4<R>(A, q1, p2, q2, p1);
                        // T = a+_a a+_b a_j a_i, i=2p1, j=2p2, a=2q1, b=2q2: -(a+_a a_j)(a+_b a_i)
                        const int i = 2 * p1, j = 2 * p2, aa = 2 * q1, bb = 2 * q2;
                        const uint32_t x1 = x ^ (1u << i) ^ (1u << bb);
                        const int s = 1 ^ par(x & between(i, bb)) ^ par(x1 & between(j, aa));
                        if (s) v = -v;
                        fma_c<R>(acc, v, row[A.ra[a ^ (1u << p1) ^ (1u << p2) ^ (1u << q1) ^ (1u << q2)]]);
                    }
                }
            }
        }
        // beta singles r -> s (partner row, same column)
        for (uint32_t o = b; o; o &= o - 1u) {
            const int r = __ffs(o) - 1;
            for (uint32_t e = eb; e; e &= e - 1u) {
                const int s = __ffs(e) - 1;
                const int Jb = A.rb[b ^ (1u << r) ^ (1u << s)];
                R v = single_value<R>(A, r, s, b, a);
                if (par(x & between(2 * r + 1, 2 * s + 1))) v = -v;
                fma_c<R>(acc, v, A.C[(size_t)Jb * Da + Ia]);
            }
        }
        // beta-beta doubles
        for (uint32_t o = b; o; o &= o - 1u) {
            const int r1 = __ffs(o) - 1;
            for (uint32_t o2 = o & (o - 1u); o2; o2 &= o2 - 1u) {
                const int r2 = __ffs(o2) - 1;
                for (uint32_t e = eb; e; e &= e - 1u) {
                    const int s1 = __ffs(e) - 1;
                    for (uint32_t e2 = e & (e - 1u); e2; e2 &= e2 - 1u) {
                        const int s2 = __ffs(e2) - 1;
                        R v = eri4<R>(A, s1, r1, s2, r2) - eri4<R>(A, s1, r2, s2, r1);
                        const int i = 2 * r1 + 1, j = 2 * r2 + 1, aa = 2 * s1 + 1, bb = 2 * s2 + 1;
                        const uint32_t x1 = x ^ (1u << i) ^ (1u << bb);
                        const int sg = 1 ^ par(x & between(i, bb)) ^ par(x1 & between(j, aa));
                        if (sg) v = -v;
                        const int Jb = A.rb[b ^ (1u << r1) ^ (1u << r2) ^ (1u << s1) ^ (1u << s2)];
                        fma_c<R>(acc, v, A.C[(size_t)Jb * Da + Ia]);
                    }
                }
            }
        }
        // alpha-beta doubles: beta r -> s and alpha p -> q, value (qp|sr);
        // <x'|(a+_q a_p)(a+_s a_r)|x>: beta single on x, then alpha single on x_beta
        for (uint32_t o = b; o; o &= o - 1u) {
            const int r = __ffs(o) - 1;
            for (uint32_t e = eb; e; e &= e - 1u) {
                const int s = __ffs(e) - 1;
                const int Jb = A.rb[b ^ (1u << r) ^ (1u << s)];
                const cplx<R> *prow = A.C + (size_t)Jb * Da;
                const int sb_ = par(x & between(2 * r + 1, 2 * s + 1));
                const uint32_t xbeta = x ^ (1u << (2 * r + 1)) ^ (1u << (2 * s + 1));
                for (uint32_t oa = a; oa; oa &= oa - 1u) {
                    const int p = __ffs(oa) - 1;
                    for (uint32_t ee = ea; ee; ee &= ee - 1u) {
                        const int q = __ffs(ee) - 1;
                        R v = eri4<R>(A, q, p, s, r);
                        if (sb_ ^ par(xbeta & between(2 * p, 2 * q))) v = -v;
                        fma_c<R>(acc, v, prow[A.ra[a ^ (1u << p) ^ (1u << q)]]);
                    }
                }
            }
        }
        if (A.lam) A.lam[x] = acc;
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
    const uint32_t *sa, *sb;
    const uint16_t *stra, *strb, *ra, *rb;
    const void *eri, *hm, *Dt, *Jt;
    int N, Da, Db;
};

cudaError_t launch_sigma_rows(const void *C, void *lam, int dtype, int n, const RowTables &T, const double *hdiag,
                              const double *Jp, double e_shift, double *partial, cudaStream_t st) {
    if (dtype == SV_C64) {
        RowArgs<float> A;
        A.C = (const float2 *)C; A.lam = (float2 *)lam;
        A.sa = T.sa; A.sb = T.sb; A.stra = T.stra; A.strb = T.strb; A.ra = T.ra; A.rb = T.rb;
        A.eri = (const float *)T.eri; A.hm = (const float *)T.hm; A.Dt = (const float *)T.Dt;
        A.Jt = (const float *)T.Jt; A.hdiag = hdiag; A.Jp = Jp; A.e_shift = e_shift; A.partial = partial;
        A.N = T.N; A.n = n; A.Da = T.Da; A.Db = T.Db; A.maskN = (1u << T.N) - 1u;
        k_sigma_rows<float><<<T.Db, kRowThreads, 0, st>>>(A);
    } else {
        RowArgs<double> A;
        A.C = (const double2 *)C; A.lam = (double2 *)lam;
        A.sa = T.sa; A.sb = T.sb; A.stra = T.stra; A.strb = T.strb; A.ra = T.ra; A.rb = T.rb;
        A.eri = (const double *)T.eri; A.hm = (const double *)T.hm; A.Dt = (const double *)T.Dt;
        A.Jt = (const double *)T.Jt; A.hdiag = hdiag; A.Jp = Jp; A.e_shift = e_shift; A.partial = partial;
        A.N = T.N; A.n = n; A.Da = T.Da; A.Db = T.Db; A.maskN = (1u << T.N) - 1u;
        k_sigma_rows<double><<<T.Db, kRowThreads, 0, st>>>(A);
    }
    return cudaGetLastError();
}

}  // namespace svk
