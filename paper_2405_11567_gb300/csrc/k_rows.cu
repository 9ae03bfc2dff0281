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
//
// Split form (variant 3: float64 states and small sectors, where the rows fit in
// shared memory): the alpha-beta doubles -- 2,500 of the 3,500 connections of an
// amplitude at 30 qubits -- read their partners at scattered columns of 50 other rows,
// which from L2 costs a 32-byte sector per 8-byte amplitude.  k_sigma_ab stages those
// partner rows, K at a time, in shared memory with coalesced loads and sums the
// alpha-beta part of sigma (and its energy share); k_sigma_same then adds every other
// group and completes sigma and the row's energy.  Product forms (variants 4 and 5,
// single-precision states of large sectors): below, "same-spin products", and
// k_abtc.cu for the alpha-beta part.
#include <cuda_bf16.h>

#include "sv_check.cuh"
#include "sv_ff.cuh"
#include "sv_internal.h"
#include "sv_sigma.cuh"

namespace svk {

constexpr int kRowThreads = kThreads;

template <typename A>
struct RowArgs {
    using R = real_of<A>;
    SigmaTables<R> T;
    const A *C;             // [Db][Da] compact sector amplitudes
    A *lam;                 // dense sigma output (nullable)
    A *lamc;                // compact sigma output [Db][Da] (nullable)
    const uint32_t *sa_s;   // [Da] alpha spread in the storage layout: addresses
    const uint32_t *sb_s;   // [Db]
    double *partial;        // [3][Db]: energy, norm, alpha-beta energy share
    const R *W2;            // [NP][NP] same-spin antisymmetrised (q1p1|q2p2) - (q1p2|q2p1), pair-indexed
    int Db;
    int same_gemm;          // 1: k_sigma_ab leaves the string-only parts to the same-spin products
};

// Per-block lists of everything that depends only on the block's beta string b.
template <typename R>
struct BetaSingle {
    int Jb;        // partner row
    int t;         // s * N + r: index of (.. |sr) and of the (sr|kk) row
    uint32_t M;    // bits strictly between 2r+1 and 2s+1
    uint32_t xbf;  // beta spread of b after r -> s
    R vb;          // h_sr + sum_{k in b} ((sr|kk) - (sk|kr))
    int cb;        // parity of the beta bits of b under M
};

template <typename R>
struct BetaDouble {
    int Jb;
    uint32_t M;    // alpha bits that decide the sign: M1 ^ M2
    int c;         // sign contribution of the beta bits
    R v;           // (s1 r1|s2 r2) - (s1 r2|s2 r1)
};

constexpr int kMaxOrb = 16;
constexpr int kMaxPairs = 120;   // C(16, 2)
constexpr int kMaxBS = 65;       // nb (N - nb) <= 8 * 8, plus the row's own slot (variant 4)
constexpr int kMaxBD = 784;      // C(8, 2)^2

template <typename Amp>
__global__ void __launch_bounds__(kRowThreads, 2) k_sigma_rows(RowArgs<Amp> A) {
    using R = real_of<Amp>;
    __shared__ BetaSingle<R> bs[kMaxBS];
    __shared__ BetaDouble<R> bd[kMaxBD];
    __shared__ R JB[kMaxOrb * kMaxOrb];
    __shared__ uint8_t opair[kMaxPairs][2], epair[kMaxPairs][2];
    __shared__ int n_bs, n_op, n_ep;
    __shared__ double red[2 * kThreads / 32];
    const SigmaTables<R> &T = A.T;
    const int Ib = blockIdx.x, N = T.N, Da = T.Da;
    const uint32_t b = T.strb[Ib], xb = T.sb[Ib], eb = ~b & T.maskN;
    if (threadIdx.x == 0) {
        int k = 0;
        for (uint32_t o = b; o; o &= o - 1u) {
            const int r = __ffs(o) - 1;
            for (uint32_t e = eb; e; e &= e - 1u) {
                const int s = __ffs(e) - 1;
                BetaSingle<R> x;
                x.Jb = T.rb[b ^ (1u << r) ^ (1u << s)];
                x.t = s * N + r;
                x.M = between(2 * r + 1, 2 * s + 1);
                x.xbf = xb ^ (1u << (2 * r + 1)) ^ (1u << (2 * s + 1));
                R v = T.hm[s * N + r];
                for (uint32_t o2 = b; o2; o2 &= o2 - 1u) v += T.Dt[(s * N + r) * N + __ffs(o2) - 1];
                x.vb = v;
                x.cb = par(xb & x.M);
                bs[k++] = x;
            }
        }
        n_bs = k;
        int no = 0, ne = 0;
        for (uint32_t o = b; o; o &= o - 1u)
            for (uint32_t o2 = o & (o - 1u); o2; o2 &= o2 - 1u) {
                opair[no][0] = (uint8_t)(__ffs(o) - 1);
                opair[no][1] = (uint8_t)(__ffs(o2) - 1);
                ++no;
            }
        for (uint32_t e = eb; e; e &= e - 1u)
            for (uint32_t e2 = e & (e - 1u); e2; e2 &= e2 - 1u) {
                epair[ne][0] = (uint8_t)(__ffs(e) - 1);
                epair[ne][1] = (uint8_t)(__ffs(e2) - 1);
                ++ne;
            }
        n_op = no;
        n_ep = ne;
    }
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        const R *jt = T.Jt + i * N;  // i = q * N + p
        R v = 0;
        for (uint32_t o = b; o; o &= o - 1u) v += jt[__ffs(o) - 1];
        JB[i] = v;
    }
    __syncthreads();
    const int nbd = n_op * n_ep, nbs = n_bs;
    for (int d = threadIdx.x; d < nbd; d += blockDim.x) {
        const int oi = d / n_ep, ei = d - oi * n_ep;
        const int r1 = opair[oi][0], r2 = opair[oi][1], s1 = epair[ei][0], s2 = epair[ei][1];
        const int i = 2 * r1 + 1, j = 2 * r2 + 1, aa = 2 * s1 + 1, bb = 2 * s2 + 1;
        const uint32_t M1 = between(i, bb), M2 = between(j, aa);
        const uint32_t xb1 = xb ^ (1u << i) ^ (1u << bb);
        BetaDouble<R> x;
        x.Jb = T.rb[b ^ (1u << r1) ^ (1u << r2) ^ (1u << s1) ^ (1u << s2)];
        x.M = M1 ^ M2;
        x.c = 1 ^ par(xb & M1) ^ par(xb1 & M2);  // T = -(a+_a a_j)(a+_b a_i)
        x.v = eri4<R>(T, s1, r1, s2, r2) - eri4<R>(T, s1, r2, s2, r1);
        bd[d] = x;
    }
    __syncthreads();
    const Amp *row = A.C + (size_t)Ib * Da;
    double e_acc = 0.0, n_acc = 0.0;
    for (int Ia = threadIdx.x; Ia < Da; Ia += blockDim.x) {
        const uint32_t a = T.stra[Ia], xa = T.sa[Ia], x = xa | xb;
        const uint32_t ea = ~a & T.maskN;
        const Amp c0 = row[Ia];
        double d = T.e_shift;
        for (uint32_t o = x; o; o &= o - 1u) {
            const int k = __ffs(o) - 1;
            d += T.hdiag[k];
            for (uint32_t o2 = o & (o - 1u); o2; o2 &= o2 - 1u) d += T.Jp[k * T.n + __ffs(o2) - 1];
        }
        Amp acc = scale_a<Amp>((R)d, c0);
        // alpha singles (this row)
        for (uint32_t o = a; o; o &= o - 1u) {
            const int p = __ffs(o) - 1;
            for (uint32_t e = ea; e; e &= e - 1u) {
                const int q = __ffs(e) - 1;
                const R *dt = T.Dt + (q * N + p) * N;
                R v = T.hm[q * N + p] + JB[q * N + p];
                for (uint32_t o2 = a; o2; o2 &= o2 - 1u) v += dt[__ffs(o2) - 1];
                if (par(x & between(2 * p, 2 * q))) v = -v;
                axpy(acc, v, row[T.ra[a ^ (1u << p) ^ (1u << q)]]);
            }
        }
        // alpha-alpha doubles (this row)
        for (uint32_t o = a; o; o &= o - 1u) {
            const int p1 = __ffs(o) - 1;
            for (uint32_t o2 = o & (o - 1u); o2; o2 &= o2 - 1u) {
                const int p2 = __ffs(o2) - 1;
                for (uint32_t e = ea; e; e &= e - 1u) {
                    const int q1 = __ffs(e) - 1;
                    for (uint32_t e2 = e & (e - 1u); e2; e2 &= e2 - 1u) {
                        const int q2 = __ffs(e2) - 1;
                        R v = eri4<R>(T, q1, p1, q2, p2) - eri4<R>(T, q1, p2, q2, p1);
                        const int i = 2 * p1, j = 2 * p2, aa = 2 * q1, bb = 2 * q2;
                        const uint32_t x1 = x ^ (1u << i) ^ (1u << bb);
                        if (1 ^ par(x & between(i, bb)) ^ par(x1 & between(j, aa))) v = -v;
                        axpy(acc, v, row[T.ra[a ^ (1u << p1) ^ (1u << p2) ^ (1u << q1) ^ (1u << q2)]]);
                    }
                }
            }
        }
        // beta singles (partner rows, same column)
        for (int k = 0; k < nbs; ++k) {
            const BetaSingle<R> e = bs[k];
            const R *jt = T.Jt + e.t * N;
            R v = e.vb;
            for (uint32_t o = a; o; o &= o - 1u) v += jt[__ffs(o) - 1];
            if (e.cb ^ par(xa & e.M)) v = -v;
            axpy(acc, v, A.C[(size_t)e.Jb * Da + Ia]);
        }
        // beta-beta doubles (partner rows, same column)
        for (int k = 0; k < nbd; ++k) {
            const BetaDouble<R> e = bd[k];
            axpy(acc, (e.c ^ par(xa & e.M)) ? -e.v : e.v, A.C[(size_t)e.Jb * Da + Ia]);
        }
        // alpha-beta doubles: alpha p -> q outside, beta r -> s (block list) inside; value (qp|sr)
        for (uint32_t o = a; o; o &= o - 1u) {
            const int p = __ffs(o) - 1;
            for (uint32_t e = ea; e; e &= e - 1u) {
                const int q = __ffs(e) - 1;
                const int Ja = T.ra[a ^ (1u << p) ^ (1u << q)];
                const uint32_t B = between(2 * p, 2 * q);
                const int sa0 = par(xa & B);
                const R *erib = T.eri + (size_t)(q * N + p) * N * N;
                for (int k = 0; k < nbs; ++k) {
                    const BetaSingle<R> bk = bs[k];
                    const R v = erib[bk.t];
                    const int sg = bk.cb ^ par(xa & bk.M) ^ sa0 ^ par(bk.xbf & B);
                    axpy(acc, sg ? -v : v, A.C[(size_t)bk.Jb * Da + Ja]);
                }
            }
        }
        if (A.lam) A.lam[A.sa_s[Ia] | A.sb_s[Ib]] = acc;
        if (A.lamc) A.lamc[(size_t)Ib * Da + Ia] = acc;
        e_acc += dre_dot(c0, acc);
        n_acc += dre_dot(c0, c0);
    }
    block_sum2(e_acc, n_acc, red);
    if (threadIdx.x == 0) {
        A.partial[Ib] = e_acc;
        A.partial[A.Db + Ib] = n_acc;
    }
}

// ---------------------------------------------------------------- split form

template <typename R>
__device__ __forceinline__ R flip_sign(R v, uint32_t bit);
template <>
__device__ __forceinline__ float flip_sign<float>(float v, uint32_t bit) {
    return __int_as_float(__float_as_int(v) ^ (int)(bit << 31));
}
template <>
__device__ __forceinline__ double flip_sign<double>(double v, uint32_t bit) {
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)((unsigned long long)bit << 63));
}
template <>
__device__ __forceinline__ ff flip_sign<ff>(ff v, uint32_t bit) {
    return ff_flip(v, bit);
}

__device__ __forceinline__ int pair_index(int p, int q, int N) { return p * N - p * (p + 1) / 2 + (q - p - 1); }

// Split form, first kernel: the diagonal, alpha singles, alpha-alpha doubles and
// beta-beta doubles of the row, with the row, the pair-indexed same-spin integrals
// W2 and Dt in shared memory.  Adds the part k_sigma_ab wrote to the output (which
// runs first) and completes the row's energy with its share partial[2 Db + Ib].
// Jordan-Wigner signs from the prefix-parity words (bit u = parity of the bits
// below u) of a and b, PP = pp(a) ^ pp(b): the bits of x strictly between 2p and
// 2q are the alpha orbitals strictly between p and q and the beta orbitals in
// [min, max), so an alpha single p -> q has sign (-1)^(popc(PP & {p,q}) + [p<q]),
// and an alpha double p1<p2 -> q1<q2 (taken as -(a+_q1 a_p2)(a+_q2 a_p1)) has
// (-1)^popc(PP & {p1,p2,q1,q2}) times an orbital-order sign that W2 carries.
constexpr int kSameThreads = 512;

template <typename Amp, bool RA_SMEM>
__global__ void __launch_bounds__(kSameThreads, 1) k_sigma_same(RowArgs<Amp> A) {
    using R = real_of<Amp>;
    extern __shared__ __align__(16) unsigned char same_dyn[];
    __shared__ BetaDouble<R> bd[kMaxBD];
    __shared__ R JB[kMaxOrb * kMaxOrb];
    __shared__ uint8_t opair[kMaxPairs][2], epair[kMaxPairs][2];
    __shared__ int n_op, n_ep;
    __shared__ double red[2 * kSameThreads / 32];
    const SigmaTables<R> &T = A.T;
    const int Ib = blockIdx.x, N = T.N, Da = T.Da, NP = N * (N - 1) / 2;
    Amp *row = reinterpret_cast<Amp *>(same_dyn);           // [Da]
    R *W2S = reinterpret_cast<R *>(row + Da);               // [NP][NP]
    R *DtS = W2S + NP * NP;                                 // [N^3]
    uint16_t *raS = reinterpret_cast<uint16_t *>(DtS + N * N * N);  // [2^N] alpha ranks
    const uint32_t b = T.strb[Ib], xb = T.sb[Ib], eb = ~b & T.maskN;
    if (threadIdx.x == 0) {
        int no = 0, ne = 0;
        for (uint32_t o = b; o; o &= o - 1u)
            for (uint32_t o2 = o & (o - 1u); o2; o2 &= o2 - 1u) {
                opair[no][0] = (uint8_t)(__ffs(o) - 1);
                opair[no][1] = (uint8_t)(__ffs(o2) - 1);
                ++no;
            }
        for (uint32_t e = eb; e; e &= e - 1u)
            for (uint32_t e2 = e & (e - 1u); e2; e2 &= e2 - 1u) {
                epair[ne][0] = (uint8_t)(__ffs(e) - 1);
                epair[ne][1] = (uint8_t)(__ffs(e2) - 1);
                ++ne;
            }
        n_op = no;
        n_ep = ne;
    }
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
        const R *jt = T.Jt + i * N;  // i = q * N + p
        R v = 0;
        for (uint32_t o = b; o; o &= o - 1u) v += jt[__ffs(o) - 1];
        JB[i] = v;
    }
    const Amp *grow = A.C + (size_t)Ib * Da;
    for (int i = threadIdx.x; i < Da; i += blockDim.x) row[i] = grow[i];
    for (int i = threadIdx.x; i < NP * NP; i += blockDim.x) W2S[i] = A.W2[i];
    for (int i = threadIdx.x; i < N * N * N; i += blockDim.x) DtS[i] = T.Dt[i];
    if (RA_SMEM)
        for (int i = threadIdx.x; i < (1 << N); i += blockDim.x) raS[i] = T.ra[i];
    const uint16_t *rk = RA_SMEM ? raS : T.ra;
    __syncthreads();
    const int nbd = n_op * n_ep;
    for (int d = threadIdx.x; d < nbd; d += blockDim.x) {
        const int oi = d / n_ep, ei = d - oi * n_ep;
        const int r1 = opair[oi][0], r2 = opair[oi][1], s1 = epair[ei][0], s2 = epair[ei][1];
        const int i = 2 * r1 + 1, j = 2 * r2 + 1, aa = 2 * s1 + 1, bb = 2 * s2 + 1;
        const uint32_t M1 = between(i, bb), M2 = between(j, aa);
        const uint32_t xb1 = xb ^ (1u << i) ^ (1u << bb);
        BetaDouble<R> x;
        x.Jb = T.rb[b ^ (1u << r1) ^ (1u << r2) ^ (1u << s1) ^ (1u << s2)];
        x.M = M1 ^ M2;
        x.c = 1 ^ par(xb & M1) ^ par(xb1 & M2);  // T = -(a+_a a_j)(a+_b a_i)
        x.v = eri4<R>(T, s1, r1, s2, r2) - eri4<R>(T, s1, r2, s2, r1);
        bd[d] = x;
    }
    __syncthreads();
    const uint32_t ppb = prefix_parity(b);
    double e_acc = 0.0, n_acc = 0.0;
    for (int Ia = threadIdx.x; Ia < Da; Ia += blockDim.x) {
        const uint32_t a = T.stra[Ia], xa = T.sa[Ia], x = xa | xb;
        const uint32_t ea = ~a & T.maskN, PP = prefix_parity(a) ^ ppb;
        const Amp c0 = row[Ia];
        double d = T.e_shift;
        for (uint32_t o = x; o; o &= o - 1u) {
            const int k = __ffs(o) - 1;
            d += T.hdiag[k];
            for (uint32_t o2 = o & (o - 1u); o2; o2 &= o2 - 1u) d += T.Jp[k * T.n + __ffs(o2) - 1];
        }
        Amp acc = scale_a<Amp>((R)d, c0);
        // alpha singles
        for (uint32_t o = a; o; o &= o - 1u) {
            const int p = __ffs(o) - 1;
            for (uint32_t e = ea; e; e &= e - 1u) {
                const int q = __ffs(e) - 1;
                const R *dt = DtS + (q * N + p) * N;
                R v = T.hm[q * N + p] + JB[q * N + p];
                for (uint32_t o2 = a; o2; o2 &= o2 - 1u) v += dt[__ffs(o2) - 1];
                const uint32_t m = (1u << p) | (1u << q);
                if ((uint32_t)par(PP & m) ^ (uint32_t)(p < q)) v = -v;
                axpy(acc, v, row[rk[a ^ m]]);
            }
        }
        // alpha-alpha doubles: W2[(p1,p2)][(q1,q2)] holds the value and the orbital-order sign
        for (uint32_t o = a; o; o &= o - 1u) {
            const int p1 = __ffs(o) - 1;
            for (uint32_t o2 = o & (o - 1u); o2; o2 &= o2 - 1u) {
                const int p2 = __ffs(o2) - 1;
                const uint32_t m12 = (1u << p1) | (1u << p2);
                const R *w = W2S + pair_index(p1, p2, N) * NP;
                for (uint32_t e = ea; e; e &= e - 1u) {
                    const int q1 = __ffs(e) - 1;
                    const uint32_t m1 = m12 | (1u << q1);
                    const R *wq = w + pair_index(q1, 0, N);  // + q2 gives pair (q1, q2)
                    for (uint32_t e2 = e & (e - 1u); e2;) {  // two partners per iteration
                        const int qa = __ffs(e2) - 1;
                        e2 &= e2 - 1u;
                        const bool two = e2 != 0u;
                        const int qb = two ? __ffs(e2) - 1 : qa;
                        if (two) e2 &= e2 - 1u;
                        const uint32_t ma = m1 | (1u << qa), mb = m1 | (1u << qb);
                        const Amp ca = row[rk[a ^ ma]], cb = row[rk[a ^ mb]];
                        const R va = flip_sign<R>(wq[qa], (uint32_t)par(PP & ma));
                        const R vb = two ? flip_sign<R>(wq[qb], (uint32_t)par(PP & mb)) : (R)0;
                        acc2(acc, va, ca, vb, cb);
                    }
                }
            }
        }
        // beta-beta doubles (partner rows, same column), four loads in flight
        int k = 0;
        for (; k + 4 <= nbd; k += 4) {
            Amp cc[4];
            #pragma unroll
            for (int j = 0; j < 4; ++j) cc[j] = A.C[(size_t)bd[k + j].Jb * Da + Ia];
            #pragma unroll
            for (int j = 0; j < 4; ++j) {
                const BetaDouble<R> e = bd[k + j];
                axpy(acc, (e.c ^ par(xa & e.M)) ? -e.v : e.v, cc[j]);
            }
        }
        for (; k < nbd; ++k) {
            const BetaDouble<R> e = bd[k];
            axpy(acc, (e.c ^ par(xa & e.M)) ? -e.v : e.v, A.C[(size_t)e.Jb * Da + Ia]);
        }
        e_acc += dre_dot(c0, acc);
        n_acc += dre_dot(c0, c0);
        if (A.lam) {
            const Amp u = A.lam[A.sa_s[Ia] | A.sb_s[Ib]];
            A.lam[A.sa_s[Ia] | A.sb_s[Ib]] = add_a<Amp>(acc, u);
        } else if (A.lamc) {
            const Amp u = A.lamc[(size_t)Ib * Da + Ia];
            A.lamc[(size_t)Ib * Da + Ia] = add_a<Amp>(acc, u);
        }
    }
    // fixed-order block sums over kSameThreads threads
    e_acc = warp_sum(e_acc);
    n_acc = warp_sum(n_acc);
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = e_acc;
        red[kSameThreads / 32 + (threadIdx.x >> 5)] = n_acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double se = 0.0, sn = 0.0;
        for (int w = 0; w < kSameThreads / 32; ++w) {
            se += red[w];
            sn += red[kSameThreads / 32 + w];
        }
        A.partial[Ib] = se + A.partial[2 * A.Db + Ib];
        A.partial[A.Db + Ib] = sn;
    }
}

constexpr int kAbThreads = 512;
constexpr int kAbIpt = 8;  // alpha strings per thread: Da <= 4096

// Row stride (in amplitudes) of the staged partner rows part[a][k]: K amplitudes rounded
// up so that a row is an odd number of 16-byte words.  The inner loop reads whole rows of
// random partner strings; with an even number of words every row would start in the same
// half of the eight 16-byte bank groups (a 64-byte row: two of them), an odd stride spreads
// the starts over all eight.
__host__ __device__ constexpr int ab_row_stride(int K, int amp_bytes) {
    const int per = 16 / amp_bytes;  // amplitudes per 16-byte word (1, 2 or 4)
    const int words = (K + per - 1) / per;
    return ((words & 1) ? words : words + 1) * per;
}

// Integral slots per (q, p) in the staged table: K rounded up to a 16-byte multiple.
template <typename R, int K>
struct AbLayout {
    static constexpr int KP = sizeof(R) == 4 ? (K + 3) & ~3 : (K + 1) & ~1;
    // row stride of the staged integral table: an odd number of 16-byte words, so rows
    // start in every group of four banks (an even stride starts them in half the groups)
    static constexpr int W16 = KP * (int)sizeof(R) / 16;
    static constexpr int KPS = (W16 & 1) ? KP : KP + 16 / (int)sizeof(R);
};

// K consecutive real amplitudes from 16-byte-aligned shared memory (K a multiple of
// 4 floats / 2 doubles).
template <int K>
__device__ __forceinline__ void lds_c(const float *p, float (&c)[K]) {
    static_assert(K % 4 == 0, "real float chunks hold a multiple of 4 rows");
    const float4 *q = reinterpret_cast<const float4 *>(p);
    #pragma unroll
    for (int j = 0; j < K / 4; ++j) {
        const float4 v = q[j];
        c[4 * j] = v.x; c[4 * j + 1] = v.y; c[4 * j + 2] = v.z; c[4 * j + 3] = v.w;
    }
}
template <int K>
__device__ __forceinline__ void lds_c(const double *p, double (&c)[K]) {
    static_assert(K % 2 == 0, "real double chunks hold an even number of rows");
    const double2 *q = reinterpret_cast<const double2 *>(p);
    #pragma unroll
    for (int j = 0; j < K / 2; ++j) {
        const double2 v = q[j];
        c[2 * j] = v.x; c[2 * j + 1] = v.y;
    }
}

// K consecutive complex amplitudes / KP reals from 16-byte-aligned shared memory.
template <int K>
__device__ __forceinline__ void lds_c(const float2 *p, float2 (&c)[K]) {
    static_assert(K % 2 == 0, "complex64 chunks hold an even number of rows");
    const float4 *q = reinterpret_cast<const float4 *>(p);
    #pragma unroll
    for (int j = 0; j < K / 2; ++j) {
        const float4 v = q[j];
        c[2 * j] = make_float2(v.x, v.y);
        c[2 * j + 1] = make_float2(v.z, v.w);
    }
}
template <int K>
__device__ __forceinline__ void lds_c(const double2 *p, double2 (&c)[K]) {
    #pragma unroll
    for (int j = 0; j < K; ++j) c[j] = p[j];
}
// float-float amplitudes (16 bytes complex, 8 bytes real) and integrals (8 bytes)
template <int K>
__device__ __forceinline__ void lds_c(const ffc *p, ffc (&c)[K]) {
    #pragma unroll
    for (int j = 0; j < K; ++j) c[j] = p[j];
}
template <int K>
__device__ __forceinline__ void lds_c(const ff *p, ff (&c)[K]) {
    static_assert(K % 2 == 0, "real float-float chunks hold an even number of rows");
    const float4 *q = reinterpret_cast<const float4 *>(p);
    #pragma unroll
    for (int j = 0; j < K / 2; ++j) {
        const float4 v = q[j];
        c[2 * j] = ff(v.x, v.y);
        c[2 * j + 1] = ff(v.z, v.w);
    }
}
template <int KP>
__device__ __forceinline__ void lds_r(const ff *p, ff (&v)[KP]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    #pragma unroll
    for (int j = 0; j < KP / 2; ++j) {
        const float4 t = q[j];
        v[2 * j] = ff(t.x, t.y);
        v[2 * j + 1] = ff(t.z, t.w);
    }
}
template <int KP>
__device__ __forceinline__ void lds_r(const float *p, float (&v)[KP]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    #pragma unroll
    for (int j = 0; j < KP / 4; ++j) {
        const float4 t = q[j];
        v[4 * j] = t.x; v[4 * j + 1] = t.y; v[4 * j + 2] = t.z; v[4 * j + 3] = t.w;
    }
}
template <int KP>
__device__ __forceinline__ void lds_r(const double *p, double (&v)[KP]) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    #pragma unroll
    for (int j = 0; j < KP / 2; ++j) {
        const double2 t = q[j];
        v[2 * j] = t.x; v[2 * j + 1] = t.y;
    }
}

// Split form, second kernel (launched first): the alpha-beta doubles and the beta
// singles of the row.
//   sigma_ab[Ib][Ia] = sum over beta r -> s of b (partner row b') of
//       sign_b [ v_rs(a) C[b'][a] + sum over alpha p -> q of a of (qp|sr) sign_a C[b'][a'] ]
// with v_rs(a) = h_sr + sum_{k in b} ((sr|kk) - (sk|kr)) + sum_{k in a} (sr|kk).
// Written to the output (lam at the storage address, else lamc) when there is one;
// the row's share of <psi|sigma> goes to partial[2 Db + Ib].
//
// Partner rows are staged K at a time in shared memory, interleaved by column
// (part[a][k], rows padded to an odd number of 16-byte words), so one vector load brings a
// column's K partner amplitudes; the
// integrals are staged as eriS[q N + p][k].  Signs (x = spread(a) | spread(b)):
//   beta single r -> s on x:  popc(x & between(2r+1, 2s+1)) -- per (a, k): applied
//                             once to row k's sum for this a;
//   alpha single p -> q on the excited x': its alpha bits between p and q -- per
//                             (a, pq): flips the integrals' sign bits; its beta bits
//                             (orbitals lo..hi-1 of b'_k) -- per (k, pq): folded into
//                             the staged integrals.
// The alpha rank table sits in shared memory.
template <typename Amp, int K>
__global__ void __launch_bounds__(kAbThreads, 1) k_sigma_ab(RowArgs<Amp> A) {
    using R = real_of<Amp>;
    constexpr int KP = AbLayout<R, K>::KP, KPS = AbLayout<R, K>::KPS;
    extern __shared__ __align__(16) unsigned char ab_dyn[];
    __shared__ int s_Jb[kMaxBS], s_t[kMaxBS], s_cb[kMaxBS];
    __shared__ uint32_t s_M[kMaxBS], s_bf[kMaxBS];
    __shared__ R s_vb[kMaxBS];
    __shared__ int n_bs;
    __shared__ double red[kAbThreads / 32];
    const SigmaTables<R> &T = A.T;
    const int Ib = blockIdx.x, N = T.N, Da = T.Da, NN = N * N;
    constexpr int PS = ab_row_stride(K, (int)sizeof(Amp));
    Amp *part = reinterpret_cast<Amp *>(ab_dyn);                  // [Da][PS]
    R *eriS = reinterpret_cast<R *>(part + (size_t)PS * Da);      // [N*N][KPS]
    R *JtS = eriS + (size_t)NN * KPS;                             // [K][N]: (s_k r_k|kk)
    uint16_t *raS = reinterpret_cast<uint16_t *>(JtS + (size_t)K * N);  // [2^N]
    const uint32_t b = T.strb[Ib], xb = T.sb[Ib], eb = ~b & T.maskN;
    if (threadIdx.x == 0) {
        int k = 0;
        for (uint32_t o = b; o; o &= o - 1u) {
            const int r = __ffs(o) - 1;
            for (uint32_t e = eb; e; e &= e - 1u) {
                const int s = __ffs(e) - 1;
                const uint32_t bf = b ^ (1u << r) ^ (1u << s);
                s_Jb[k] = T.rb[bf];
                s_t[k] = s * N + r;
                s_M[k] = between(2 * r + 1, 2 * s + 1);
                s_bf[k] = bf;
                s_cb[k] = par(xb & s_M[k]);
                R v = 0;
                if (!A.same_gemm) {  // else the beta string's own part is in the beta product
                    v = T.hm[s * N + r];
                    for (uint32_t o2 = b; o2; o2 &= o2 - 1u) v += T.Dt[(s * N + r) * N + __ffs(o2) - 1];
                }
                s_vb[k] = v;
                ++k;
            }
        }
        if (A.same_gemm) {
            // the row itself as one more staged row: the part of the alpha singles that
            // depends on b, sum_{k in b} (qp|kk), with no beta excitation (s_t = -1)
            s_Jb[k] = Ib;
            s_t[k] = -1;
            s_M[k] = 0;
            s_bf[k] = b;
            s_cb[k] = 0;
            s_vb[k] = 0;
            ++k;
        }
        n_bs = k;
    }
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(T.ra);
        uint32_t *dst = reinterpret_cast<uint32_t *>(raS);
        for (int i = threadIdx.x; i < (1 << N) / 2; i += kAbThreads) dst[i] = src[i];
    }
    __syncthreads();
    const int nbs = n_bs;
    Amp acc[kAbIpt];
    #pragma unroll
    for (int t = 0; t < kAbIpt; ++t) acc[t] = mka<Amp>(0, 0);
    for (int k0 = 0; k0 < nbs; k0 += K) {
        const int kn = min(K, nbs - k0);
        if (k0) __syncthreads();  // the previous chunk is consumed
        for (int i = threadIdx.x; i < K * Da; i += kAbThreads) {
            const int k = i / Da, c = i - k * Da;
            part[(size_t)c * PS + k] = k < kn ? A.C[(size_t)s_Jb[k0 + k] * Da + c] : mka<Amp>(0, 0);
        }
        for (int i = threadIdx.x; i < NN * KP; i += kAbThreads) {
            const int qp = i / KP, k = i - qp * KP, q = qp / N, p = qp - q * N;
            R v = 0;
            if (k < kn && p != q) {
                const int lo = min(p, q), hi = max(p, q);
                const uint32_t mB = ((1u << hi) - 1u) & ~((1u << lo) - 1u);  // beta orbitals lo..hi-1
                const int t = s_t[k0 + k];
                R w = 0;
                if (t >= 0) {
                    w = T.eri[(size_t)qp * NN + t];
                } else {  // own row: sum over the beta string's orbitals of (qp|kk)
                    for (uint32_t o = b; o; o &= o - 1u) w += T.Jt[(size_t)qp * N + __ffs(o) - 1];
                }
                v = flip_sign<R>(w, (uint32_t)par(s_bf[k0 + k] & mB));
            }
            eriS[qp * KPS + k] = v;
        }
        for (int i = threadIdx.x; i < K * N; i += kAbThreads) {
            const int k = i / N, o = i - k * N;
            JtS[i] = (k < kn && s_t[k0 + k] >= 0) ? T.Jt[(size_t)s_t[k0 + k] * N + o] : (R)0;
        }
        __syncthreads();
        uint32_t Mk[K];
        int cbk[K];
        R vbk[K];
        #pragma unroll
        for (int k = 0; k < K; ++k) {
            const int kk = k < kn ? k0 + k : k0;
            Mk[k] = s_M[kk];
            cbk[k] = s_cb[kk];
            vbk[k] = k < kn ? s_vb[kk] : (R)0;
        }
        #pragma unroll
        for (int t = 0; t < kAbIpt; ++t) {
            const int Ia = threadIdx.x + t * kAbThreads;
            if (Ia >= Da) continue;
            const uint32_t a = T.stra[Ia], xa = T.sa[Ia], ea = ~a & T.maskN, ppa = prefix_parity(a);
            Amp sk[K];
            {   // beta singles: same column of the staged rows
                Amp c[K];
                lds_c<K>(part + (size_t)Ia * PS, c);
                #pragma unroll
                for (int k = 0; k < K; ++k) {
                    R v = vbk[k];
                    for (uint32_t o = a; o; o &= o - 1u) v += JtS[k * N + __ffs(o) - 1];
                    sk[k] = scale_a<Amp>(v, c[k]);
                }
            }
            for (uint32_t o = a; o; o &= o - 1u) {
                const int p = __ffs(o) - 1;
                // two empty orbitals per iteration: both partners' loads in flight together
                for (uint32_t e = ea; e;) {
                    const int q0 = __ffs(e) - 1;
                    e &= e - 1u;
                    const bool two = e != 0u;
                    const int q1 = two ? __ffs(e) - 1 : q0;
                    if (two) e &= e - 1u;
                    const uint32_t m0 = (1u << p) | (1u << q0), m1 = (1u << p) | (1u << q1);
                    const int J0 = raS[a ^ m0], J1 = raS[a ^ m1];
                    // alpha bits strictly between p and q
                    const uint32_t s0 = (uint32_t)par(ppa & m0) ^ (uint32_t)(p < q0);
                    const uint32_t s1 = (uint32_t)par(ppa & m1) ^ (uint32_t)(p < q1);
                    Amp c0[K], c1[K];
                    R v0[KP], v1[KP];
                    lds_c<K>(part + (size_t)J0 * PS, c0);
                    lds_c<K>(part + (size_t)J1 * PS, c1);
                    lds_r<KP>(eriS + (q0 * N + p) * KPS, v0);
                    lds_r<KP>(eriS + (q1 * N + p) * KPS, v1);
                    #pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const R w0 = flip_sign<R>(v0[k], s0);
                        const R w1 = two ? flip_sign<R>(v1[k], s1) : (R)0;
                        acc2(sk[k], w0, c0[k], w1, c1[k]);
                    }
                }
            }
            Amp tot = acc[t];
            #pragma unroll
            for (int k = 0; k < K; ++k) {
                if (k < kn) {
                    const bool neg = cbk[k] ^ par(xa & Mk[k]);
                    tot = lin2<Amp>((R)1, tot, neg ? (R)-1 : (R)1, sk[k]);
                }
            }
            acc[t] = tot;
        }
    }
    double e_acc = 0.0;
    const Amp *row = A.C + (size_t)Ib * Da;
    #pragma unroll
    for (int t = 0; t < kAbIpt; ++t) {
        const int Ia = threadIdx.x + t * kAbThreads;
        if (Ia >= Da) continue;
        const Amp c0 = row[Ia];
        e_acc += dre_dot(c0, acc[t]);
        if (A.lam) A.lam[A.sa_s[Ia] | A.sb_s[Ib]] = acc[t];
        else if (A.lamc) A.lamc[(size_t)Ib * Da + Ia] = acc[t];
    }
    // fixed-order block sum over kAbThreads threads
    e_acc = warp_sum(e_acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e_acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kAbThreads / 32; ++w) s += red[w];
        A.partial[2 * A.Db + Ib] = s;
    }
}

// ---------------------------------------------------------------- same-spin products
//
// Expectation variants 4 and 5 (single-precision states).  In the string-blocked basis
// (alpha creators before beta creators) the same-spin part of H is a matrix on one
// string index times the identity on the other:
//   Ma[a][a'] = alpha singles p -> q with h_qp + sum_{k in a} ((qp|kk) - (qk|kp)),
//               and alpha-alpha doubles (q1p1|q2p2) - (q1p2|q2p1),
// with the sign of the excitation on the alpha string alone; Mb likewise for beta.
// So two dense products, G = Ma X + X Mb^T over the phased matrix X = phi C, give that
// part of sigma~ = phi sigma.  The rest is the alpha-beta part (alpha-beta doubles, the
// beta singles' dependence on a, and the alpha singles' dependence on b) -- k_sigma_ab
// (variant 4, the latter through the row's own slot) or k_ab_tc (variant 5) -- and
// k_sigma_comb (diagonal, phase back, sum, energy).  The dense products (k_same_tc on
// the tensor cores) do every multiply of a matrix with 17% nonzeros
// at 30 qubits, on a pipe whose rate repays it, instead of scattered shared-memory
// gathers.

// Block I < Da builds alpha row I of Ma, block Da + I beta row I of Mb; thread 0 also
// writes the string's one-spin diagonal energy sum_k h_kk + sum_{k<l} [kk|ll]-[kl|lk]
// (spin-orbital tables hdiag, Jp) to dA / dB.  Ma and Mb must be zeroed before.
__global__ void __launch_bounds__(128) k_same_mats(SigmaTables<float> T, float *__restrict__ Ma,
                                                    float *__restrict__ Mb, double *__restrict__ dA,
                                                    double *__restrict__ dB, int lda, int ldb) {
    __shared__ uint8_t occ[kMaxOrb], emp[kMaxOrb];
    __shared__ int s_no, s_ne;
    const bool beta = (int)blockIdx.x >= T.Da;
    const int I = beta ? (int)blockIdx.x - T.Da : (int)blockIdx.x, N = T.N, spin = beta;
    const uint16_t *rk = beta ? T.rb : T.ra;
    const uint32_t str = beta ? T.strb[I] : T.stra[I], pps = prefix_parity(str);
    float *row = (beta ? Mb : Ma) + (size_t)I * (beta ? ldb : lda);
    if (threadIdx.x == 0) {
        int no = 0, ne = 0;
        for (int o = 0; o < N; ++o) {
            if ((str >> o) & 1u) occ[no++] = (uint8_t)o;
            else emp[ne++] = (uint8_t)o;
        }
        s_no = no;
        s_ne = ne;
        double d = 0.0;
        for (int i = 0; i < no; ++i) {
            const int k = 2 * occ[i] + spin;
            d += T.hdiag[k];
            for (int j = i + 1; j < no; ++j) d += T.Jp[k * T.n + 2 * occ[j] + spin];
        }
        (beta ? dB : dA)[I] = d;
    }
    __syncthreads();
    const int no = s_no, ne = s_ne, nsg = no * ne, npo = no * (no - 1) / 2, npe = ne * (ne - 1) / 2;
    for (int t = threadIdx.x; t < nsg + npo * npe; t += blockDim.x) {
        float v;
        uint32_t m, sg;
        if (t < nsg) {
            const int p = occ[t / ne], q = emp[t % ne];
            m = (1u << p) | (1u << q);
            v = T.hm[q * N + p];
            const float *dt = T.Dt + (q * N + p) * N;
            for (uint32_t o = str; o; o &= o - 1u) v += dt[__ffs(o) - 1];
            sg = (uint32_t)par(pps & m) ^ (uint32_t)(p < q);
        } else {
            int io = (t - nsg) / npe, ie = (t - nsg) % npe, i1 = 0, e1 = 0;
            while (io >= no - 1 - i1) io -= no - 1 - i1++;  // pair index -> (i1, i1 + 1 + io)
            while (ie >= ne - 1 - e1) ie -= ne - 1 - e1++;
            const int p1 = occ[i1], p2 = occ[i1 + 1 + io], q1 = emp[e1], q2 = emp[e1 + 1 + ie];
            m = (1u << p1) | (1u << p2) | (1u << q1) | (1u << q2);
            v = eri4<float>(T, q1, p1, q2, p2) - eri4<float>(T, q1, p2, q2, p1);
            sg = (uint32_t)par(pps & m) ^ double_order_sign(p1, p2, q1, q2);
        }
        row[rk[str ^ m]] = sg ? -v : v;
    }
}

// X[plane][Ib][Ia] = phi(a, b) * component of C[Ib][Ia] (planes: re, im).
// Three bf16 pieces of a float: x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2).
__device__ __forceinline__ void bf16x3(float v, uint16_t *p, size_t piece) {
    const __nv_bfloat16 a = __float2bfloat16_rn(v);
    const float r = v - __bfloat162float(a);
    const __nv_bfloat16 b = __float2bfloat16_rn(r);
    const __nv_bfloat16 c = __float2bfloat16_rn(r - __bfloat162float(b));
    p[0] = __bfloat16_as_ushort(a);
    p[piece] = __bfloat16_as_ushort(b);
    p[2 * piece] = __bfloat16_as_ushort(c);
}

// With Xp (tensor-core form) the planes are written as three bf16 pieces at stride px
// instead of float32 X.  With Xi (variant 5) also, per amplitude, the three words
// (re_k | im_k << 16), k = 1..3, at Xi[(Ib ldi + Ia) 3 + k - 1].
__device__ __forceinline__ void bf16x3_u(float v, uint32_t &p1, uint32_t &p2, uint32_t &p3) {
    const __nv_bfloat16 a = __float2bfloat16_rn(v);
    const float r = v - __bfloat162float(a);
    const __nv_bfloat16 b = __float2bfloat16_rn(r);
    const __nv_bfloat16 c = __float2bfloat16_rn(r - __bfloat162float(b));
    p1 = __bfloat16_as_ushort(a);
    p2 = __bfloat16_as_ushort(b);
    p3 = __bfloat16_as_ushort(c);
}

template <typename Amp>
__global__ void __launch_bounds__(kThreads) k_phase_planar(const Amp *__restrict__ C, const uint16_t *__restrict__ stra,
                                                           const uint16_t *__restrict__ strb, int Da, int Db,
                                                           int ld, uint16_t *__restrict__ Xp, size_t px,
                                                           uint32_t *__restrict__ Xi, int ldi) {
    const size_t plane = (size_t)ld * Db;  // rows padded to ld (the padding stays zero)
    for (int Ib = blockIdx.x; Ib < Db; Ib += gridDim.x) {
        const uint32_t ppb = prefix_parity(strb[Ib]);
        const size_t off = (size_t)Ib * Da, xo = (size_t)Ib * ld;
        for (int Ia = threadIdx.x; Ia < Da; Ia += blockDim.x) {
            const uint32_t neg = (uint32_t)par(stra[Ia] & ppb);
            const Amp c = C[off + Ia];
            const float xr = flip_sign<float>(re(c), neg);
            bf16x3(xr, Xp + xo + Ia, px);
            float xi = 0.f;
            if constexpr (AmpT<Amp>::kCplx) {
                xi = flip_sign<float>(im(c), neg);
                bf16x3(xi, Xp + plane + xo + Ia, px);
            }
            if (Xi) {
                uint32_t r1, r2, r3, i1, i2, i3;
                bf16x3_u(xr, r1, r2, r3);
                bf16x3_u(xi, i1, i2, i3);
                uint32_t *w = Xi + ((size_t)Ib * ldi + Ia) * 3;
                w[0] = r1 | (i1 << 16);
                w[1] = r2 | (i2 << 16);
                w[2] = r3 | (i3 << 16);
            }
        }
    }
}

// One block per row b: sigma[b][a] = (sigma_ab part already in the output) + d(a, b) C
// + phi(a, b) G[b][a], with the diagonal d = E_nuc - c + dA[a] + dB[b] + sum over
// alpha orbitals p in a of sum over beta orbitals q in b of [2p | 2q+1] (float64);
// the row's energy and norm as in k_sigma_same (fixed-order float64 sums).
// GATHER (variant 5): the alpha-beta part is not in the output but in the planes H of
// the tensor-core products (k_ab_tc); it is gathered here, in the blocked basis, as
// sum over the beta excitations r -> s of b (partner b') of
// (-1)^popc(b & between(r, s)) H[b'][col(b', rs)][a], plus H[b][own][a], in a fixed
// order, and added to G before the phase; the output is written, not added to.
template <typename Amp, bool GATHER>
__global__ void __launch_bounds__(kThreads) k_sigma_comb(RowArgs<Amp> A, SameGemm g) {
    using R = real_of<Amp>;
    __shared__ double xb[kMaxOrb];
    __shared__ double red[2 * kThreads / 32];
    __shared__ size_t s_hoff[kMaxBS];
    __shared__ int s_hneg[kMaxBS];
    const SigmaTables<R> &T = A.T;
    const int Ib = blockIdx.x, Da = T.Da, N = T.N;
    const uint32_t b = T.strb[Ib], ppb = prefix_parity(b);
    int nh = 0;
    if constexpr (GATHER) {
        // H rows to gather: entry j = (r, s) in the order of b's occupied r, empty s; the
        // last one the row's own column
        const int nb = __popc(b), ne = N - nb, nbs = nb * ne;
        nh = nbs + 1;
        if ((int)threadIdx.x < nbs) {
            const int i = threadIdx.x / ne, j = threadIdx.x - i * ne;
            uint32_t o = b, z = ~b & T.maskN;
            for (int k = 0; k < i; ++k) o &= o - 1u;
            for (int k = 0; k < j; ++k) z &= z - 1u;
            const int r = __ffs(o) - 1, sx = __ffs(z) - 1;
            const uint32_t bp = b ^ (1u << r) ^ (1u << sx);
            // column of (s occupied, r empty) among b''s excitations
            const int col = __popc(bp & ((1u << sx) - 1u)) * ne + __popc(~bp & T.maskN & ((1u << r) - 1u));
            s_hoff[threadIdx.x] = ((size_t)T.rb[bp] * g.ncols + col) * g.ldh;
            s_hneg[threadIdx.x] = par(b & between(r, sx));
        } else if ((int)threadIdx.x == nbs) {
            s_hoff[nbs] = ((size_t)Ib * g.ncols + nbs) * g.ldh;
            s_hneg[nbs] = 0;
        }
    }
    if ((int)threadIdx.x < N) {
        const int k = 2 * (int)threadIdx.x;
        double sx = 0.0;
        for (uint32_t o = b; o; o &= o - 1u) {
            const int l = 2 * (__ffs(o) - 1) + 1;
            sx += T.Jp[min(k, l) * T.n + max(k, l)];
        }
        xb[threadIdx.x] = sx;
    }
    __syncthreads();
    const double db = T.e_shift + g.dB[Ib];
    const size_t plane = (size_t)Da * A.Db, off = (size_t)Ib * Da;
    double e_acc = 0.0, n_acc = 0.0;
    for (int Ia = threadIdx.x; Ia < Da; Ia += blockDim.x) {
        const uint32_t a = T.stra[Ia], neg = (uint32_t)par(a & ppb);
        double d = db + g.dA[Ia];
        for (uint32_t o = a; o; o &= o - 1u) d += xb[__ffs(o) - 1];
        const Amp c0 = A.C[off + Ia];
        float gr = g.G[off + Ia], gi = 0.f;
        if constexpr (AmpT<Amp>::kCplx) gi = g.G[plane + off + Ia];
        if constexpr (GATHER) {
            for (int j = 0; j < nh; ++j) {
                if (!SV_IN_RANGE(s_hoff[j] + Ia, g.hplane, kChkPlane)) continue;  // checked build: skip the term
                const float *hp = g.H + s_hoff[j] + Ia;
                float hr = hp[0], hi = 0.f;
                if constexpr (AmpT<Amp>::kCplx) hi = hp[g.hplane];
                if (s_hneg[j]) { hr = -hr; hi = -hi; }
                gr += hr;
                gi += hi;
            }
        }
        Amp acc;
        if constexpr (AmpT<Amp>::kCplx)
            acc = mka<Amp>(fmaf((R)d, re(c0), flip_sign<float>(gr, neg)), fmaf((R)d, im(c0), flip_sign<float>(gi, neg)));
        else
            acc = mka<Amp>(fmaf((R)d, re(c0), flip_sign<float>(gr, neg)), (R)0);
        e_acc += dre_dot(c0, acc);
        n_acc += dre_dot(c0, c0);
        if (GATHER) {
            if (A.lam) A.lam[A.sa_s[Ia] | A.sb_s[Ib]] = acc;
            else if (A.lamc) A.lamc[off + Ia] = acc;
        } else if (A.lam) {
            const Amp u = A.lam[A.sa_s[Ia] | A.sb_s[Ib]];
            A.lam[A.sa_s[Ia] | A.sb_s[Ib]] = add_a<Amp>(acc, u);
        } else if (A.lamc) {
            const Amp u = A.lamc[off + Ia];
            A.lamc[off + Ia] = add_a<Amp>(acc, u);
        }
    }
    block_sum2(e_acc, n_acc, red);
    if (threadIdx.x == 0) {
        A.partial[Ib] = GATHER ? e_acc : e_acc + A.partial[2 * A.Db + Ib];
        A.partial[A.Db + Ib] = n_acc;
    }
}

// C[Ib][Ia] = psi[sa[Ia] | sb[Ib]]
template <typename A>
__global__ void __launch_bounds__(kThreads) k_compact(const A *__restrict__ psi, A *__restrict__ C,
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
    SV_DISPATCH_AMP(dtype, k_compact<A><<<grid, kThreads, 0, st>>>((const A *)psi, (A *)C, sa, sb, Da, total));
    return cudaGetLastError();
}

// Device pointers of the string-row tables (built by the host in sv_api.cu).
struct RowTables {
    const uint32_t *sa, *sb, *sa_s, *sb_s;
    const uint16_t *stra, *strb, *ra, *rb;
    const void *eri, *hm, *Dt, *Jt;
    int N, Da, Db;
    const void *W2 = nullptr;  // pair-indexed same-spin integrals (split form)
};

template <typename Amp>
static RowArgs<Amp> row_args(const void *C, void *lam, void *lamc, int n, const RowTables &T, const double *hdiag,
                             const double *Jp, double e_shift, double *partial) {
    using R = real_of<Amp>;
    RowArgs<Amp> A;
    A.T.sa = T.sa; A.T.sb = T.sb; A.T.stra = T.stra; A.T.strb = T.strb; A.T.ra = T.ra; A.T.rb = T.rb;
    A.T.eri = (const R *)T.eri; A.T.hm = (const R *)T.hm; A.T.Dt = (const R *)T.Dt; A.T.Jt = (const R *)T.Jt;
    A.T.hdiag = hdiag; A.T.Jp = Jp; A.T.e_shift = e_shift;
    A.T.N = T.N; A.T.n = n; A.T.Da = T.Da; A.T.maskN = (1u << T.N) - 1u;
    A.C = (const Amp *)C; A.lam = (Amp *)lam; A.lamc = (Amp *)lamc; A.sa_s = T.sa_s; A.sb_s = T.sb_s;
    A.partial = partial; A.Db = T.Db; A.W2 = (const R *)T.W2;
    A.same_gemm = 0;
    return A;
}

constexpr size_t kAbSmemCap = 225 * 1024;  // dynamic shared memory a split kernel may use

// Dynamic shared memory of k_sigma_ab for K staged rows, and of k_sigma_same.
static size_t ab_smem(int dtype, int K, const RowTables &T) {
    const size_t amp = amp_size(dtype), real = single_prec(dtype) ? 4 : 8;
    const size_t KP = real == 4 ? (size_t)((K + 3) & ~3) : (size_t)((K + 1) & ~1);
    const size_t KPS = ((KP * real / 16) & 1) ? KP : KP + 16 / real;  // AbLayout<R, K>::KPS
    const size_t PS = (size_t)ab_row_stride(K, (int)amp);
    return PS * T.Da * amp + (size_t)T.N * T.N * KPS * real + (size_t)K * T.N * real + ((size_t)2 << T.N);
}

// k_sigma_same's dynamic shared memory, with or without the alpha rank table; its
// static shared memory (the beta-double list) is below 24 KB, so 203 KB of dynamic
// memory keeps the block within the 227 KB a block may use.
constexpr size_t kSameSmemCap = 203 * 1024;

static size_t same_smem(int dtype, const RowTables &T, bool ra_in) {
    const size_t amp = amp_size(dtype), real = single_prec(dtype) ? 4 : 8, NP = (size_t)T.N * (T.N - 1) / 2;
    return (size_t)T.Da * amp + NP * NP * real + (size_t)T.N * T.N * T.N * real + (ra_in ? ((size_t)2 << T.N) : 0);
}

// Compiled chunk sizes per state type: a column of K staged amplitudes is a whole
// number of 16-byte words.
static const int kChunks[4][4] = {{2, 4, 6, 8},      // complex64
                                  {1, 2, 3, 4},      // complex128
                                  {4, 8, 12, 16},    // real float
                                  {2, 4, 6, 8}};     // real double

// Rows staged per chunk by k_sigma_ab, 0 when the split form does not fit (the
// single-kernel form runs instead).  `want` > 0 asks for that chunk size (taken when
// it is one of the compiled sizes and fits, else the largest such size below it);
// otherwise the fewest estimated issue slots, chunks * (K + 3), among the sizes that fit.
int sigma_ab_chunk(int dtype, const RowTables &T, int nb, int want) {
    if (T.Da > kAbThreads * kAbIpt || T.Db < 1 || T.N < 2) return 0;
    if (same_smem(dtype, T, false) > kSameSmemCap) return 0;
    const int *sizes = kChunks[dtype & 3];
    if (want > 0) {
        for (int i = 3; i >= 0; --i)
            if (sizes[i] <= want && ab_smem(dtype, sizes[i], T) <= kAbSmemCap) return sizes[i];
    }
    const int nbs = nb * (T.N - nb) > 0 ? nb * (T.N - nb) : 1;  // beta singles of a row
    int best = 0;
    long best_cost = 0;
    for (int i = 0; i < 4; ++i) {
        const int K = sizes[i];
        if (ab_smem(dtype, K, T) > kAbSmemCap) continue;
        const long cost = (long)((nbs + K - 1) / K) * (K + 3);
        if (!best || cost < best_cost || (cost == best_cost && K > best)) {
            best = K;
            best_cost = cost;
        }
    }
    return best;
}

const int *sigma_ab_sizes(int dtype) { return kChunks[dtype & 3]; }

template <typename Amp, int K>
static cudaError_t launch_ab(const RowArgs<Amp> &A, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_sigma_ab<Amp, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sigma_ab<Amp, K><<<A.Db, kAbThreads, smem, st>>>(A);
    return cudaGetLastError();
}

template <typename Amp, int K0, int K1, int K2, int K3>
static cudaError_t launch_ab_k4(const RowArgs<Amp> &A, int K, size_t smem, cudaStream_t st) {
    if (K == K0) return launch_ab<Amp, K0>(A, smem, st);
    if (K == K1) return launch_ab<Amp, K1>(A, smem, st);
    if (K == K2) return launch_ab<Amp, K2>(A, smem, st);
    if (K == K3) return launch_ab<Amp, K3>(A, smem, st);
    return cudaErrorInvalidValue;
}

static cudaError_t launch_ab_k(const RowArgs<float2> &A, int K, size_t smem, cudaStream_t st) {
    return launch_ab_k4<float2, 2, 4, 6, 8>(A, K, smem, st);
}
static cudaError_t launch_ab_k(const RowArgs<double2> &A, int K, size_t smem, cudaStream_t st) {
    return launch_ab_k4<double2, 1, 2, 3, 4>(A, K, smem, st);
}
static cudaError_t launch_ab_k(const RowArgs<float> &A, int K, size_t smem, cudaStream_t st) {
    return launch_ab_k4<float, 4, 8, 12, 16>(A, K, smem, st);
}
static cudaError_t launch_ab_k(const RowArgs<double> &A, int K, size_t smem, cudaStream_t st) {
    return launch_ab_k4<double, 2, 4, 6, 8>(A, K, smem, st);
}
static cudaError_t launch_ab_k(const RowArgs<ffc> &A, int K, size_t smem, cudaStream_t st) {
    return launch_ab_k4<ffc, 1, 2, 3, 4>(A, K, smem, st);
}
static cudaError_t launch_ab_k(const RowArgs<ff> &A, int K, size_t smem, cudaStream_t st) {
    return launch_ab_k4<ff, 2, 4, 6, 8>(A, K, smem, st);
}

cudaError_t launch_same_tc(const uint16_t *M, size_t pm, const uint16_t *X, size_t px, uint16_t *Xt, size_t pt,
                           float *G, int planes, int Da, int Db, int lda, int ldb, int *err, uint32_t spins, int stall,
                           cudaStream_t st);
cudaError_t launch_ab_tc(const uint32_t *Xi, int planes, const uint16_t *stra, const uint16_t *strb,
                         const uint16_t *ra, const uint16_t *Bp, size_t pb, const uint16_t *rowB, float *H,
                         size_t hplane, int Da, int Db,
                         int N, int na, int nb, int *err, uint32_t spins, int stall, int sm_count, cudaStream_t st);

template <typename Amp>
static cudaError_t launch_same_t(RowArgs<Amp> A, const RowTables &T, int dtype, int K, const SameGemm &g,
                                 int sm_count, cudaStream_t st) {
    if constexpr (sizeof(real_of<Amp>) != 4) {
        return cudaErrorInvalidValue;  // single-precision states only
    } else {
        const int grid = T.Db < sm_count * 8 ? T.Db : sm_count * 8;
        k_phase_planar<Amp><<<grid, kThreads, 0, st>>>(A.C, T.stra, T.strb, T.Da, T.Db, g.lda, g.Xp, g.px,
                                                       g.abtc ? g.Xi : nullptr, g.ldi);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (g.ev && (e = cudaEventRecord(g.ev[0], st)) != cudaSuccess) return e;
        e = launch_same_tc(g.Mp, g.pm, g.Xp, g.px, g.Xtp, g.pt, g.G, g.planes, T.Da, T.Db, g.lda, g.ldb, g.err,
                           g.spins, g.stall & 1, st);
        if (e != cudaSuccess) return e;
        if (g.ev && (e = cudaEventRecord(g.ev[1], st)) != cudaSuccess) return e;
        A.same_gemm = 1;
        if (g.abtc) {
            if (g.ev && (e = cudaEventRecord(g.ev[2], st)) != cudaSuccess) return e;
            e = launch_ab_tc(g.Xi, g.planes, T.stra, T.strb, T.ra, g.Bp, g.pb, g.rowB, g.H, g.hplane, T.Da, T.Db, T.N, g.na,
                             g.nb, g.err, g.spins, (g.stall >> 1) & 1, sm_count, st);
            if (e != cudaSuccess) return e;
            if (g.ev && (e = cudaEventRecord(g.ev[3], st)) != cudaSuccess) return e;
            k_sigma_comb<Amp, true><<<T.Db, kThreads, 0, st>>>(A, g);
        } else {
            e = launch_ab_k(A, K, ab_smem(dtype, K, T), st);
            if (e != cudaSuccess) return e;
            k_sigma_comb<Amp, false><<<T.Db, kThreads, 0, st>>>(A, g);
        }
        return cudaGetLastError();
    }
}

template <typename Amp>
static cudaError_t launch_rows_t(const RowArgs<Amp> &A, const RowTables &T, int dtype, int K, const SameGemm *g,
                                 int sm_count, cudaStream_t st) {
    if (K == 0) {
        k_sigma_rows<Amp><<<T.Db, kRowThreads, 0, st>>>(A);
        return cudaGetLastError();
    }
    if (g) return launch_same_t<Amp>(A, T, dtype, K, *g, sm_count, st);
    cudaError_t e = launch_ab_k(A, K, ab_smem(dtype, K, T), st);
    if (e != cudaSuccess) return e;
    if (same_smem(dtype, T, true) <= kSameSmemCap) {
        const size_t smem = same_smem(dtype, T, true);
        e = cudaFuncSetAttribute(k_sigma_same<Amp, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_sigma_same<Amp, true><<<T.Db, kSameThreads, smem, st>>>(A);
    } else {
        const size_t smem = same_smem(dtype, T, false);
        e = cudaFuncSetAttribute(k_sigma_same<Amp, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_sigma_same<Amp, false><<<T.Db, kSameThreads, smem, st>>>(A);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- float-float form

// Expectation variant 6 (float64 states): the split form's two kernels instantiated on
// float-float amplitudes and integrals (sv_ff.cuh), so every product and sum of an
// amplitude's connections runs on the FP32 pipe at about 48-bit precision.  The compact
// amplitudes are converted once per call (k_to_ff), the kernels sum sigma into a
// float-float compact matrix, and k_from_ff writes it back as float64 (to the dense
// vector at the storage addresses, or to the compact output); the energies and norms
// are float64 sums as in the other forms.
template <typename A, typename F>
__global__ void __launch_bounds__(kThreads) k_to_ff(const A *__restrict__ in, F *__restrict__ out, size_t count) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        if constexpr (AmpT<A>::kCplx) {
            const A v = in[i];
            ffc c;
            c.x = ff_from(v.x);
            c.y = ff_from(v.y);
            out[i] = c;
        } else {
            out[i] = ff_from(in[i]);
        }
    }
}

template <typename F, typename A>
__global__ void __launch_bounds__(kThreads) k_from_ff(const F *__restrict__ in, A *__restrict__ lam,
                                                      A *__restrict__ lamc, const uint32_t *__restrict__ sa_s,
                                                      const uint32_t *__restrict__ sb_s, int Da, int Db) {
    for (int Ib = blockIdx.x; Ib < Db; Ib += gridDim.x) {
        const F *row = in + (size_t)Ib * Da;
        for (int Ia = threadIdx.x; Ia < Da; Ia += blockDim.x) {
            A v;
            if constexpr (AmpT<A>::kCplx) v = mka<A>(ff_to(row[Ia].x), ff_to(row[Ia].y));
            else v = ff_to(row[Ia]);
            if (lam) lam[sa_s[Ia] | sb_s[Ib]] = v;
            if (lamc) lamc[(size_t)Ib * Da + Ia] = v;
        }
    }
}

template <typename A, typename F>
static cudaError_t launch_ff_t(const void *C, void *lam, void *lamc, int dtype, int n, const RowTables &Tf,
                               const double *hdiag, const double *Jp, double e_shift, double *partial, int K,
                               void *Cf, void *Lf, int sm_count, cudaStream_t st) {
    const size_t count = (size_t)Tf.Da * Tf.Db;
    int grid = (int)std::min<size_t>((count + kThreads - 1) / kThreads, (size_t)sm_count * 8);
    if (grid < 1) grid = 1;
    k_to_ff<A, F><<<grid, kThreads, 0, st>>>((const A *)C, (F *)Cf, count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    RowArgs<F> RA = row_args<F>(Cf, nullptr, Lf, n, Tf, hdiag, Jp, e_shift, partial);
    e = launch_ab_k(RA, K, ab_smem(dtype, K, Tf), st);
    if (e != cudaSuccess) return e;
    if (same_smem(dtype, Tf, true) <= kSameSmemCap) {
        const size_t smem = same_smem(dtype, Tf, true);
        e = cudaFuncSetAttribute(k_sigma_same<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_sigma_same<F, true><<<Tf.Db, kSameThreads, smem, st>>>(RA);
    } else {
        const size_t smem = same_smem(dtype, Tf, false);
        e = cudaFuncSetAttribute(k_sigma_same<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_sigma_same<F, false><<<Tf.Db, kSameThreads, smem, st>>>(RA);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int g2 = Tf.Db < sm_count * 8 ? Tf.Db : sm_count * 8;
    k_from_ff<F, A><<<g2, kThreads, 0, st>>>((const F *)Lf, (A *)lam, (A *)lamc, Tf.sa_s, Tf.sb_s, Tf.Da, Tf.Db);
    return cudaGetLastError();
}

// The float-float split form for a float64 state (complex128 or real float64): Tf holds
// the float-float integral tables (eri, hm, Dt, Jt, W2); Cf and Lf are two compact
// float-float work matrices (Da Db x 16 or 8 bytes each); K as for the split form.
// Launches k_to_ff, k_sigma_ab, k_sigma_same, k_from_ff.
cudaError_t launch_sigma_rows_ff(const void *C, void *lam, void *lamc, int dtype, int n, const RowTables &Tf,
                                 const double *hdiag, const double *Jp, double e_shift, double *partial, int K,
                                 void *Cf, void *Lf, int sm_count, cudaStream_t st) {
    if (K <= 0) return cudaErrorInvalidValue;
    if (dtype == SV_C128)
        return launch_ff_t<double2, ffc>(C, lam, lamc, dtype, n, Tf, hdiag, Jp, e_shift, partial, K, Cf, Lf, sm_count,
                                         st);
    if (dtype == SV_R64)
        return launch_ff_t<double, ff>(C, lam, lamc, dtype, n, Tf, hdiag, Jp, e_shift, partial, K, Cf, Lf, sm_count,
                                       st);
    return cudaErrorInvalidValue;
}

// The float-float form (ffc for complex128, ff for float64) of `count` amplitudes of a
// float64 state, into out (count x 16 or 8 bytes).
cudaError_t launch_to_ff(const void *C, int dtype, size_t count, void *out, int sm_count, cudaStream_t st) {
    int grid = (int)std::min<size_t>((count + kThreads - 1) / kThreads, (size_t)sm_count * 8);
    if (grid < 1) grid = 1;
    if (dtype == SV_C128)
        k_to_ff<double2, ffc><<<grid, kThreads, 0, st>>>((const double2 *)C, (ffc *)out, count);
    else if (dtype == SV_R64)
        k_to_ff<double, ff><<<grid, kThreads, 0, st>>>((const double *)C, (ff *)out, count);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// K: rows per chunk of the split form (sigma_ab_chunk), 0 for the single-kernel form.
// partial must hold 3 * Db doubles (rows: energy, norm, alpha-beta energy share).
// g (may be NULL): the product forms (single-precision states, K > 0): the phase kernel,
// the same-spin products (k_transpose_pieces + k_same_tc), then k_sigma_ab (variant 4) or k_ab_tc (variant 5, g->abtc), and
// k_sigma_comb (which in variant 5 also gathers the alpha-beta planes).
cudaError_t launch_sigma_rows(const void *C, void *lam, void *lamc, int dtype, int n, const RowTables &T, const double *hdiag,
                              const double *Jp, double e_shift, double *partial, int K, cudaStream_t st,
                              const SameGemm *g, int sm_count) {
    cudaError_t e = cudaErrorInvalidValue;
    SV_DISPATCH_AMP(dtype, e = launch_rows_t<A>(row_args<A>(C, lam, lamc, n, T, hdiag, Jp, e_shift, partial), T, dtype,
                                                K, g, sm_count, st));
    return e;
}

// Ma [Da][lda], Mb [Db][ldb] (zeroed here, padding included), dA, dB of the sector for
// single-precision tables.
cudaError_t launch_same_mats(int n, const RowTables &T, const double *hdiag, const double *Jp, float *Ma, float *Mb,
                             double *dA, double *dB, int lda, int ldb, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(Ma, 0, sizeof(float) * (size_t)T.Da * lda, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(Mb, 0, sizeof(float) * (size_t)T.Db * ldb, st);
    if (e != cudaSuccess) return e;
    RowArgs<float> A = row_args<float>(nullptr, nullptr, nullptr, n, T, hdiag, Jp, 0.0, nullptr);
    k_same_mats<<<T.Da + T.Db, 128, 0, st>>>(A.T, Ma, Mb, dA, dB, lda, ldb);
    return cudaGetLastError();
}

// This unit's check word (checked build), for sv_check_status.
SV_CHECK_READER(check_word_rows)

}  // namespace svk
