// sv_sigma.cuh -- one element of sigma = (H - c) psi on the string-row view of a
// sector, shared by the string-row expectation kernel (k_rows.cu) and the batched
// persistent kernel (k_batch.cu).
//
// A sector determinant is x = spread_alpha(a) | spread_beta(b); C[rank(b)][rank(a)]
// holds the amplitudes.  The element at (a, b) sums the diagonal and every X-mask
// group connected to x (Slater-Condon closed forms; Jordan-Wigner signs as
// popcount parities over the bits strictly between the indices, a double
// T = a+_a a+_b a_j a_i taken as -(a+_a a_j)(a+_b a_i)):
//   alpha singles, alpha-alpha doubles      partner C[rank(b)][rank(a')]
//   beta singles, beta-beta doubles         partner C[rank(b')][rank(a)]
//   alpha-beta doubles (value (qp|sr))      partner C[rank(b')][rank(a')]
#pragma once

#include "sv_device.cuh"

namespace svk {

__device__ __forceinline__ uint32_t between(int a, int b) {
    int lo = min(a, b), hi = max(a, b);
    return ((1u << hi) - 1u) & ~((2u << lo) - 1u);
}

__device__ __forceinline__ int par(uint32_t v) { return __popc(v) & 1; }

template <typename R>
struct SigmaTables {
    const uint32_t *sa;     // [Da] alpha spread (even bits), qubit space
    const uint32_t *sb;     // [Db] beta spread (odd bits), qubit space
    const uint16_t *stra;   // [Da] alpha strings
    const uint16_t *strb;   // [Db] beta strings
    const uint16_t *ra;     // [2^N] rank of an alpha string (valid strings only)
    const uint16_t *rb;     // [2^N] rank of a beta string
    const R *eri;           // [N^4] spatial (pq|rs)
    const R *hm;            // [N^2] spatial h_pq
    const R *Dt;            // [N^3] (qp|kk) - (qk|kp): same-spin occupied k
    const R *Jt;            // [N^3] (qp|kk): opposite-spin occupied k
    const double *hdiag;    // [n] h_kk per spin-orbital (qubit order)
    const double *Jp;       // [n][n] [kk|ll] - [kl|lk] (qubit order)
    double e_shift;         // E_nuc - c
    int N, n, Da;
    uint32_t maskN;
};

// v for a single p->q of one spin with same-spin string `own` and opposite-spin
// string `other`: h_qp + sum_{k in own} ((qp|kk) - (qk|kp)) + sum_{k in other} (qp|kk).
template <typename R>
__device__ __forceinline__ R single_value(const SigmaTables<R> &A, int p, int q, uint32_t own, uint32_t other) {
    const int N = A.N;
    const R *dt = A.Dt + (q * N + p) * N;
    const R *jt = A.Jt + (q * N + p) * N;
    R v = A.hm[q * N + p];
    for (uint32_t o = own; o; o &= o - 1u) v += dt[__ffs(o) - 1];
    for (uint32_t o = other; o; o &= o - 1u) v += jt[__ffs(o) - 1];
    return v;
}

template <typename R>
__device__ __forceinline__ R eri4(const SigmaTables<R> &A, int p, int q, int r, int s) {
    const int N = A.N;
    return A.eri[((p * N + q) * N + r) * N + s];
}

template <typename R>
__device__ __forceinline__ void fma_c(cplx<R> &acc, R v, const cplx<R> &c) {
    acc.x += v * c.x;
    acc.y += v * c.y;
}

// sigma at (rank a = Ia, rank b = Ib) for amplitudes C ([Db][Da]); c0 = C[Ib][Ia].
template <typename R>
__device__ __forceinline__ cplx<R> sigma_at(const SigmaTables<R> &A, const cplx<R> *__restrict__ C, int Ia, int Ib,
                                            cplx<R> c0) {
    const int N = A.N, Da = A.Da;
    const uint32_t b = A.strb[Ib], xb = A.sb[Ib];
    const uint32_t eb = ~b & A.maskN;
    const cplx<R> *row = C + (size_t)Ib * Da;
    (void)N;
    const uint32_t a = A.stra[Ia], xa = A.sa[Ia], x = xa | xb;
    const uint32_t ea = ~a & A.maskN;
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
            fma_c<R>(acc, v, C[(size_t)Jb * Da + Ia]);
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
                    fma_c<R>(acc, v, C[(size_t)Jb * Da + Ia]);
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
            const cplx<R> *prow = C + (size_t)Jb * Da;
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
    return acc;
}

}  // namespace svk
