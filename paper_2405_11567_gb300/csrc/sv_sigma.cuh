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

// Parity prefix of an orbital string: bit u = parity of the bits of s below u.
__device__ __forceinline__ uint32_t prefix_parity(uint32_t s) {
    uint32_t y = s << 1;
    y ^= y << 1;
    y ^= y << 2;
    y ^= y << 4;
    y ^= y << 8;
    y ^= y << 16;
    return y;
}

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

// Orbital-order part of the Jordan-Wigner sign of a same-spin double p1<p2 -> q1<q2
// taken as -(a+_q1 a_p2)(a+_q2 a_p1): the string-dependent part is the parity of the
// prefix-parity word over the four orbitals.
__device__ __forceinline__ uint32_t double_order_sign(int p1, int p2, int q1, int q2) {
    return (uint32_t)((p1 < q2) ^ (q2 < p2) ^ (p1 < q1) ^ (p2 < q1));
}

// sigma at (rank a = Ia, rank b = Ib) for amplitudes C ([Db][Da]); c0 = C[Ib][Ia].
// Signs from prefix-parity words (bit u = parity of the bits below u): with
// interleaved spin-orbitals the bits of x strictly between 2p and 2q are the alpha
// orbitals strictly between p and q and the beta orbitals in [min, max), so an alpha
// excitation's sign is the parity of pp(a) ^ pp(b) over its orbitals (plus an
// orbital-order term), and a beta excitation's that of pp(b) ^ pp(a) ^ a.
template <typename R>
__device__ __forceinline__ cplx<R> sigma_at(const SigmaTables<R> &A, const cplx<R> *__restrict__ C, int Ia, int Ib,
                                            cplx<R> c0) {
    const int N = A.N, Da = A.Da;
    const uint32_t b = A.strb[Ib], xb = A.sb[Ib];
    const uint32_t eb = ~b & A.maskN;
    const cplx<R> *row = C + (size_t)Ib * Da;
    const uint32_t a = A.stra[Ia], xa = A.sa[Ia], x = xa | xb;
    const uint32_t ea = ~a & A.maskN;
    const uint32_t ppa = prefix_parity(a), ppb = prefix_parity(b);
    const uint32_t PPa = ppa ^ ppb, PPb = ppb ^ ppa ^ a;  // alpha / beta excitation parity words
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
            const uint32_t m = (1u << p) | (1u << q);
            R v = single_value<R>(A, p, q, a, b);
            if ((uint32_t)par(PPa & m) ^ (uint32_t)(p < q)) v = -v;
            fma_c<R>(acc, v, row[A.ra[a ^ m]]);
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
                    const uint32_t m = (1u << p1) | (1u << p2) | (1u << q1) | (1u << q2);
                    R v = eri4<R>(A, q1, p1, q2, p2) - eri4<R>(A, q1, p2, q2, p1);
                    if ((uint32_t)par(PPa & m) ^ double_order_sign(p1, p2, q1, q2)) v = -v;
                    fma_c<R>(acc, v, row[A.ra[a ^ m]]);
                }
            }
        }
    }
    // beta singles r -> s (partner row, same column)
    for (uint32_t o = b; o; o &= o - 1u) {
        const int r = __ffs(o) - 1;
        for (uint32_t e = eb; e; e &= e - 1u) {
            const int s = __ffs(e) - 1;
            const uint32_t m = (1u << r) | (1u << s);
            R v = single_value<R>(A, r, s, b, a);
            if ((uint32_t)par(PPb & m) ^ (uint32_t)(r < s)) v = -v;
            fma_c<R>(acc, v, C[(size_t)A.rb[b ^ m] * Da + Ia]);
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
                    const uint32_t m = (1u << r1) | (1u << r2) | (1u << s1) | (1u << s2);
                    R v = eri4<R>(A, s1, r1, s2, r2) - eri4<R>(A, s1, r2, s2, r1);
                    if ((uint32_t)par(PPb & m) ^ double_order_sign(r1, r2, s1, s2)) v = -v;
                    fma_c<R>(acc, v, C[(size_t)A.rb[b ^ m] * Da + Ia]);
                }
            }
        }
    }
    // alpha-beta doubles: beta r -> s on x, then alpha p -> q on x' (beta string b'),
    // value (qp|sr); alpha partner ranks and signs hoisted out of the beta loop
    for (uint32_t o = b; o; o &= o - 1u) {
        const int r = __ffs(o) - 1;
        for (uint32_t e = eb; e; e &= e - 1u) {
            const int s = __ffs(e) - 1;
            const uint32_t mb = (1u << r) | (1u << s);
            const cplx<R> *prow = C + (size_t)A.rb[b ^ mb] * Da;
            const uint32_t sb = (uint32_t)par(PPb & mb) ^ (uint32_t)(r < s);
            const uint32_t PPx = ppa ^ prefix_parity(b ^ mb);  // alpha parity word on x'
            const R *er = A.eri + s * N + r;                   // (qp|sr) at er[(q N + p) N^2]
            for (uint32_t oa = a; oa; oa &= oa - 1u) {
                const int p = __ffs(oa) - 1;
                for (uint32_t ee = ea; ee; ee &= ee - 1u) {
                    const int q = __ffs(ee) - 1;
                    const uint32_t m = (1u << p) | (1u << q);
                    R v = er[(q * N + p) * N * N];
                    if (sb ^ (uint32_t)par(PPx & m) ^ (uint32_t)(p < q)) v = -v;
                    fma_c<R>(acc, v, prow[A.ra[a ^ m]]);
                }
            }
        }
    }
    return acc;
}

}  // namespace svk
