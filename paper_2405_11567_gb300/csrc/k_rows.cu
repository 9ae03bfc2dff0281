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
// Split form (default where the rows fit in shared memory): the alpha-beta doubles
// -- 2,500 of the 3,500 connections of an amplitude at 30 qubits -- read their
// partners at scattered columns of 50 other rows, which from L2 costs a 32-byte
// sector per 8-byte amplitude.  k_sigma_ab stages those partner rows, K at a time,
// in shared memory with coalesced loads and sums the alpha-beta part of sigma (and
// its energy share); k_sigma_rows<SPLIT> then adds every other group, reading its
// own row from shared memory, and completes sigma and the row's energy.
#include "sv_internal.h"
#include "sv_sigma.cuh"

namespace svk {

constexpr int kRowThreads = kThreads;

template <typename R>
struct RowArgs {
    SigmaTables<R> T;
    const cplx<R> *C;       // [Db][Da] compact sector amplitudes
    cplx<R> *lam;           // dense sigma output (nullable)
    cplx<R> *lamc;          // compact sigma output [Db][Da] (nullable)
    const uint32_t *sa_s;   // [Da] alpha spread in the storage layout: addresses
    const uint32_t *sb_s;   // [Db]
    double *partial;        // [2][Db]
    int Db;
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
constexpr int kMaxBS = 64;       // nb (N - nb) <= 8 * 8
constexpr int kMaxBD = 784;      // C(8, 2)^2

template <typename R, bool SPLIT>
__global__ void __launch_bounds__(kRowThreads) k_sigma_rows(RowArgs<R> A) {
    extern __shared__ __align__(16) unsigned char row_smem[];  // SPLIT: this block's row [Da]
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
    const cplx<R> *row = A.C + (size_t)Ib * Da;
    if (SPLIT) {
        cplx<R> *srow = reinterpret_cast<cplx<R> *>(row_smem);
        for (int i = threadIdx.x; i < Da; i += blockDim.x) srow[i] = row[i];
        row = srow;
    }
    __syncthreads();
    double e_acc = 0.0, n_acc = 0.0;
    for (int Ia = threadIdx.x; Ia < Da; Ia += blockDim.x) {
        const uint32_t a = T.stra[Ia], xa = T.sa[Ia], x = xa | xb;
        const uint32_t ea = ~a & T.maskN;
        const cplx<R> c0 = row[Ia];
        double d = T.e_shift;
        for (uint32_t o = x; o; o &= o - 1u) {
            const int k = __ffs(o) - 1;
            d += T.hdiag[k];
            for (uint32_t o2 = o & (o - 1u); o2; o2 &= o2 - 1u) d += T.Jp[k * T.n + __ffs(o2) - 1];
        }
        cplx<R> acc = mk<R>((R)d * c0.x, (R)d * c0.y);
        // alpha singles (this row)
        for (uint32_t o = a; o; o &= o - 1u) {
            const int p = __ffs(o) - 1;
            for (uint32_t e = ea; e; e &= e - 1u) {
                const int q = __ffs(e) - 1;
                const R *dt = T.Dt + (q * N + p) * N;
                R v = T.hm[q * N + p] + JB[q * N + p];
                for (uint32_t o2 = a; o2; o2 &= o2 - 1u) v += dt[__ffs(o2) - 1];
                if (par(x & between(2 * p, 2 * q))) v = -v;
                fma_c<R>(acc, v, row[T.ra[a ^ (1u << p) ^ (1u << q)]]);
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
                        fma_c<R>(acc, v, row[T.ra[a ^ (1u << p1) ^ (1u << p2) ^ (1u << q1) ^ (1u << q2)]]);
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
            fma_c<R>(acc, v, A.C[(size_t)e.Jb * Da + Ia]);
        }
        // beta-beta doubles (partner rows, same column)
        for (int k = 0; k < nbd; ++k) {
            const BetaDouble<R> e = bd[k];
            fma_c<R>(acc, (e.c ^ par(xa & e.M)) ? -e.v : e.v, A.C[(size_t)e.Jb * Da + Ia]);
        }
        // alpha-beta doubles: alpha p -> q outside, beta r -> s (block list) inside; value (qp|sr)
        for (uint32_t o = SPLIT ? 0u : a; o; o &= o - 1u) {
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
                    fma_c<R>(acc, sg ? -v : v, A.C[(size_t)bk.Jb * Da + Ja]);
                }
            }
        }
        e_acc += (double)c0.x * (double)acc.x + (double)c0.y * (double)acc.y;
        n_acc += (double)c0.x * (double)c0.x + (double)c0.y * (double)c0.y;
        if (SPLIT) {  // add the alpha-beta part k_sigma_ab wrote to the output
            if (A.lam) {
                const cplx<R> u = A.lam[A.sa_s[Ia] | A.sb_s[Ib]];
                acc.x += u.x; acc.y += u.y;
            } else if (A.lamc) {
                const cplx<R> u = A.lamc[(size_t)Ib * Da + Ia];
                acc.x += u.x; acc.y += u.y;
            }
        }
        if (A.lam) A.lam[A.sa_s[Ia] | A.sb_s[Ib]] = acc;
        if (A.lamc) A.lamc[(size_t)Ib * Da + Ia] = acc;
    }
    block_sum2(e_acc, n_acc, red);
    if (threadIdx.x == 0) {
        A.partial[Ib] = SPLIT ? e_acc + A.partial[2 * A.Db + Ib] : e_acc;
        A.partial[A.Db + Ib] = n_acc;
    }
}

// ---------------------------------------------------------------- alpha-beta part

constexpr int kAbThreads = 512;
constexpr int kAbIpt = 8;  // alpha strings per thread: Da <= 4096

// sigma_ab[Ib][Ia] = sum over alpha p->q of a and beta r->s of b of
// (qp|sr) sign C[rank(b')][rank(a')], written to the output (lam at the storage
// address, else lamc) when there is one; the row's share of <psi|sigma> goes to
// partial[2 Db + Ib].
//
// Partner rows b' are staged K at a time in shared memory (coalesced loads).  The
// sign of a term is the product of three parities (x = spread(a) | spread(b)):
//   beta single r -> s on x:           popc(x & between(2r+1, 2s+1)) -- depends on
//                                      (a, k): one bit per chunk row, applied to
//                                      that row's sum once per alpha string;
//   alpha single p -> q, alpha bits:   popc(a & between(p, q)) -- per (a, pq),
//                                      flips the integral's sign bit;
//   alpha single p -> q, beta bits of the excited string b'_k between 2p and 2q --
//                                      per (k, pq): folded into the staged
//                                      integrals eriS[k][q N + p] = +-(qp|s_k r_k).
// The rank table of alpha strings is copied to shared memory when it fits.
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

template <typename R, int K>
__global__ void __launch_bounds__(kAbThreads) k_sigma_ab(RowArgs<R> A, int ra_smem) {
    extern __shared__ __align__(16) unsigned char ab_dyn[];
    __shared__ int s_Jb[kMaxBS], s_t[kMaxBS], s_cb[kMaxBS];
    __shared__ uint32_t s_M[kMaxBS], s_bf[kMaxBS];
    __shared__ int n_bs;
    __shared__ double red[kAbThreads / 32];
    const SigmaTables<R> &T = A.T;
    const int Ib = blockIdx.x, N = T.N, Da = T.Da, NN = N * N;
    cplx<R> *part = reinterpret_cast<cplx<R> *>(ab_dyn);         // [K][Da]
    R *eriS = reinterpret_cast<R *>(part + (size_t)K * Da);      // [K][N*N]
    uint16_t *raS = reinterpret_cast<uint16_t *>(eriS + (size_t)K * NN);  // [2^N] when ra_smem
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
                ++k;
            }
        }
        n_bs = k;
    }
    const uint16_t *rk = T.ra;
    if (ra_smem) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(T.ra);
        uint32_t *dst = reinterpret_cast<uint32_t *>(raS);
        for (int i = threadIdx.x; i < (1 << N) / 2; i += kAbThreads) dst[i] = src[i];
        rk = raS;
    }
    __syncthreads();
    const int nbs = n_bs;
    cplx<R> acc[kAbIpt];
    #pragma unroll
    for (int t = 0; t < kAbIpt; ++t) acc[t] = mk<R>(0, 0);
    for (int k0 = 0; k0 < nbs; k0 += K) {
        const int kn = min(K, nbs - k0);
        if (k0) __syncthreads();  // the previous chunk is consumed
        for (int k = 0; k < K; ++k) {
            if (k < kn) {
                const cplx<R> *src = A.C + (size_t)s_Jb[k0 + k] * Da;
                for (int i = threadIdx.x; i < Da; i += kAbThreads) part[k * Da + i] = src[i];
            } else {  // rows past the end of the list contribute zero
                for (int i = threadIdx.x; i < Da; i += kAbThreads) part[k * Da + i] = mk<R>(0, 0);
            }
        }
        for (int i = threadIdx.x; i < K * NN; i += kAbThreads) {
            const int k = i / NN, qp = i - k * NN, q = qp / N, p = qp - q * N;
            R v = 0;
            if (k < kn && p != q) {
                const int lo = min(p, q), hi = max(p, q);
                const uint32_t mB = ((1u << hi) - 1u) & ~((1u << lo) - 1u);  // beta orbitals lo..hi-1
                v = flip_sign<R>(T.eri[(size_t)qp * NN + s_t[k0 + k]], (uint32_t)par(s_bf[k0 + k] & mB));
            }
            eriS[i] = v;
        }
        __syncthreads();
        uint32_t Mk[K];
        int cbk[K];
        #pragma unroll
        for (int k = 0; k < K; ++k) {
            const int kk = k < kn ? k0 + k : k0;
            Mk[k] = s_M[kk];
            cbk[k] = s_cb[kk];
        }
        #pragma unroll
        for (int t = 0; t < kAbIpt; ++t) {
            const int Ia = threadIdx.x + t * kAbThreads;
            if (Ia >= Da) continue;
            const uint32_t a = T.stra[Ia], xa = T.sa[Ia], ea = ~a & T.maskN;
            cplx<R> sk[K];
            #pragma unroll
            for (int k = 0; k < K; ++k) sk[k] = mk<R>(0, 0);
            for (uint32_t o = a; o; o &= o - 1u) {
                const int p = __ffs(o) - 1;
                for (uint32_t e = ea; e; e &= e - 1u) {
                    const int q = __ffs(e) - 1;
                    const int Ja = rk[a ^ (1u << p) ^ (1u << q)];
                    const int lo = min(p, q), hi = max(p, q);
                    const uint32_t mA = ((1u << hi) - 1u) & ~((2u << lo) - 1u);  // alpha orbitals lo+1..hi-1
                    const uint32_t sa0 = (uint32_t)par(a & mA);
                    const R *ev = eriS + q * N + p;
                    const cplx<R> *pc = part + Ja;
                    #pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const R v = flip_sign<R>(ev[k * NN], sa0);
                        const cplx<R> c = pc[k * Da];
                        sk[k].x += v * c.x;
                        sk[k].y += v * c.y;
                    }
                }
            }
            cplx<R> tot = acc[t];
            #pragma unroll
            for (int k = 0; k < K; ++k) {
                if (k < kn) {
                    const bool neg = cbk[k] ^ par(xa & Mk[k]);
                    tot.x += neg ? -sk[k].x : sk[k].x;
                    tot.y += neg ? -sk[k].y : sk[k].y;
                }
            }
            acc[t] = tot;
        }
    }
    double e_acc = 0.0;
    const cplx<R> *row = A.C + (size_t)Ib * Da;
    #pragma unroll
    for (int t = 0; t < kAbIpt; ++t) {
        const int Ia = threadIdx.x + t * kAbThreads;
        if (Ia >= Da) continue;
        const cplx<R> c0 = row[Ia];
        e_acc += (double)c0.x * (double)acc[t].x + (double)c0.y * (double)acc[t].y;
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
static RowArgs<R> row_args(const void *C, void *lam, void *lamc, int n, const RowTables &T, const double *hdiag,
                           const double *Jp, double e_shift, double *partial) {
    RowArgs<R> A;
    A.T.sa = T.sa; A.T.sb = T.sb; A.T.stra = T.stra; A.T.strb = T.strb; A.T.ra = T.ra; A.T.rb = T.rb;
    A.T.eri = (const R *)T.eri; A.T.hm = (const R *)T.hm; A.T.Dt = (const R *)T.Dt; A.T.Jt = (const R *)T.Jt;
    A.T.hdiag = hdiag; A.T.Jp = Jp; A.T.e_shift = e_shift;
    A.T.N = T.N; A.T.n = n; A.T.Da = T.Da; A.T.maskN = (1u << T.N) - 1u;
    A.C = (const cplx<R> *)C; A.lam = (cplx<R> *)lam; A.lamc = (cplx<R> *)lamc; A.sa_s = T.sa_s; A.sb_s = T.sb_s;
    A.partial = partial; A.Db = T.Db;
    return A;
}

constexpr size_t kAbSmemCap = 225 * 1024;  // dynamic shared memory the split form may use

static size_t ab_smem(int dtype, int K, const RowTables &T, bool ra_in) {
    const size_t amp = dtype == SV_C64 ? 8 : 16, real = amp / 2;
    return (size_t)K * T.Da * amp + (size_t)K * T.N * T.N * real + (ra_in ? ((size_t)2 << T.N) : 0);
}

static const int kAbChunks[] = {1, 2, 3, 4, 5, 6, 8};

// Rows staged per chunk by k_sigma_ab (0: the split form does not fit), and whether
// the alpha rank table goes to shared memory: the fewest estimated issue slots,
// chunks * (K + 3), among the sizes that fit, with the table in shared memory if
// any size allows it.
int sigma_ab_chunk(int dtype, const RowTables &T, int nb, int want, int *ra_in) {
    if (T.Da > kAbThreads * kAbIpt || T.Db < 1) return 0;
    const int nbs = nb * (T.N - nb) > 0 ? nb * (T.N - nb) : 1;  // beta singles of a row
    for (int pass = 0; pass < 2; ++pass) {
        const bool rin = pass == 0;
        int best = 0;
        long best_cost = 0;
        for (int K : kAbChunks) {
            if (want > 0 && K > want) continue;
            if (ab_smem(dtype, K, T, rin) > kAbSmemCap) continue;
            const long cost = (long)((nbs + K - 1) / K) * (K + 3);
            if (!best || cost < best_cost || (cost == best_cost && K > best)) {
                best = K;
                best_cost = cost;
            }
        }
        if (best) {
            if (ra_in) *ra_in = rin ? 1 : 0;
            return best;
        }
    }
    return 0;
}

template <typename R, int K>
static cudaError_t launch_ab(const RowArgs<R> &A, size_t smem, int ra_in, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_sigma_ab<R, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_sigma_ab<R, K><<<A.Db, kAbThreads, smem, st>>>(A, ra_in);
    return cudaGetLastError();
}

template <typename R>
static cudaError_t launch_rows_t(const RowArgs<R> &A, const RowTables &T, int dtype, int K, cudaStream_t st) {
    if (K == 0) {
        k_sigma_rows<R, false><<<T.Db, kRowThreads, 0, st>>>(A);
        return cudaGetLastError();
    }
    const bool rin = (K & 16) != 0;
    K &= 15;
    const size_t smem = ab_smem(dtype, K, T, rin);
    cudaError_t e;
    switch (K) {
        case 1: e = launch_ab<R, 1>(A, smem, rin, st); break;
        case 2: e = launch_ab<R, 2>(A, smem, rin, st); break;
        case 3: e = launch_ab<R, 3>(A, smem, rin, st); break;
        case 4: e = launch_ab<R, 4>(A, smem, rin, st); break;
        case 5: e = launch_ab<R, 5>(A, smem, rin, st); break;
        case 6: e = launch_ab<R, 6>(A, smem, rin, st); break;
        case 8: e = launch_ab<R, 8>(A, smem, rin, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const size_t row_bytes = (size_t)T.Da * sizeof(cplx<R>);
    e = cudaFuncSetAttribute(k_sigma_rows<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_bytes);
    if (e != cudaSuccess) return e;
    k_sigma_rows<R, true><<<T.Db, kRowThreads, row_bytes, st>>>(A);
    return cudaGetLastError();
}

// K: rows per chunk of the split form (sigma_ab_chunk), plus 16 when the alpha rank
// table is staged in shared memory; 0 for the single-kernel form.
// partial must hold 3 * Db doubles (rows: energy, norm, alpha-beta energy share).
cudaError_t launch_sigma_rows(const void *C, void *lam, void *lamc, int dtype, int n, const RowTables &T, const double *hdiag,
                              const double *Jp, double e_shift, double *partial, int K, cudaStream_t st) {
    if (dtype == SV_C64)
        return launch_rows_t<float>(row_args<float>(C, lam, lamc, n, T, hdiag, Jp, e_shift, partial), T, dtype, K, st);
    return launch_rows_t<double>(row_args<double>(C, lam, lamc, n, T, hdiag, Jp, e_shift, partial), T, dtype, K, st);
}

}  // namespace svk
