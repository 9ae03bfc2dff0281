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
// rotation kernels spread an operator's pairs (its alpha list x beta list) over the
// whole grid, so a launch touches only the pairs it rotates:
//   k_rotate_l   psi'[x] = c psi[x] - s sn psi[x'],  psi'[x'] = c psi[x'] + s sn psi[x]
//                over the op's pairs (alpha list x beta list, built by k_build_lists)
//   k_adjoint_l  g += s (Re conj(lam[x']) psi[x] - Re conj(lam[x]) psi[x']), then U^dagger
//                on psi and lambda (float64 per block, fixed-order sums)
//   k_rdm_rows   one block per beta string: every density-matrix element's share
// with s = (-1)^popc(x & sm), the Jordan-Wigner sign (sm = 0 for qubit
// excitations).
#include <cstring>
#include <vector>

#include "sv_internal.h"
#include "sv_check.cuh"
#include "sv_ff.cuh"
#include "sv_sigma.cuh"

namespace svk {

// An op's sign mask and its alpha / beta string flip masks and "from" patterns.
struct SectOp {
    uint32_t sm;
    uint32_t ma, fa, mb, fb;
};

struct SectTabs {
    const uint32_t *sa, *sb;       // qubit-space spreads
    const uint16_t *stra, *strb;   // strings
    const uint16_t *ra, *rb;       // ranks
    int Da, Db;
};

// Per-operator lists.  An operator acts on the determinants whose alpha string
// matches its alpha pattern and whose beta string matches its beta pattern, so its
// pairs are the product of an alpha list and a beta list.  Both are built once per
// operator list (k_build_lists) and kept on the device: one uint32 per string,
//   rank | sign << 15 | partner rank << 16,
// with sign = parity of the string's spread under the operator's sign mask (the
// Jordan-Wigner sign of the pair is the XOR of the alpha and beta entries).
// Ranks fit in 15 bits: at most C(16, 8) = 12,870 strings.
struct ListOp {
    uint32_t sm, ma, fa, mb, fb;
    uint32_t a_off, b_off;  // entry offsets of the op's alpha and beta lists
    uint32_t a_n, b_n;      // their lengths (C(N - |m|, n - |f|) per spin)
};

// Block 2k builds op k's alpha list, block 2k+1 its beta list, in rank order
// (ordered compaction with warp ballots).
__global__ void __launch_bounds__(kThreads) k_build_lists(const ListOp *__restrict__ ops, SectTabs T,
                                                          uint32_t *__restrict__ out) {
    __shared__ int wcount[kThreads / 32];
    const ListOp op = ops[blockIdx.x >> 1];
    const bool beta = blockIdx.x & 1;
    const int D = beta ? T.Db : T.Da;
    const uint16_t *str = beta ? T.strb : T.stra, *rk = beta ? T.rb : T.ra;
    const uint32_t *spr = beta ? T.sb : T.sa;
    const uint32_t m = beta ? op.mb : op.ma, f = beta ? op.fb : op.fa;
    uint32_t *dst = out + (beta ? op.b_off : op.a_off);
    const int cap = (int)(beta ? op.b_n : op.a_n);  // the host's count: writes never pass it
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    int total = 0;
    for (int base = 0; base < D; base += blockDim.x) {
        const int I = base + threadIdx.x;
        uint32_t s = 0;
        bool hit = false;
        if (I < D) {
            s = str[I];
            hit = (s & m) == f;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, hit);
        if (lane == 0) wcount[warp] = __popc(bal);
        __syncthreads();
        int off = total, sum = 0;
        for (int w = 0; w < nw; ++w) {
            const int c = wcount[w];
            if (w < warp) off += c;
            sum += c;
        }
        if (hit && off + __popc(bal & lt) < cap)
            dst[off + __popc(bal & lt)] = (uint32_t)I | ((uint32_t)par(spr[I] & op.sm) << 15) |
                                          ((uint32_t)rk[s ^ m] << 16);
        total += sum;
        __syncthreads();
    }
}

// The op's pairs (beta entry r, alpha entry i) in flattened order r na + i, spread
// over the whole grid: thread t takes pairs t, t + T, ... (T = threads in the grid),
// four at a time so their loads are in flight together.  Pair (r, i) is (I, J) with
//   I = rank_b(r) Da + rank_a(i),  J = partner_b(r) Da + partner_a(i),
// and the Jordan-Wigner sign the XOR of the two entries' sign bits.
struct PairWalk {
    int r, i, dr, di, na;
    __device__ __forceinline__ PairWalk(int na_l) : na(na_l) {
        const int T = (int)(gridDim.x * blockDim.x), g = (int)(blockIdx.x * blockDim.x + threadIdx.x);
        r = g / na_l;
        i = g - r * na_l;
        dr = T / na_l;
        di = T - dr * na_l;
    }
    __device__ __forceinline__ void next() {
        r += dr;
        i += di;
        if (i >= na) {
            i -= na;
            ++r;
        }
    }
};

constexpr int kPairBatch = 4;

// The list entries of a thread's next kPairBatch pairs (ok[v]: pair v exists).  The lists
// are read-only during a sweep, so the whole-sweep kernels load a batch's entries ahead:
// the first batch of an operator before its grid barrier, each next batch while the
// current batch's amplitudes are in flight.
struct PairBatch {
    uint32_t ea[kPairBatch], eb[kPairBatch];
    bool ok[kPairBatch];
    __device__ __forceinline__ void load(PairWalk &w, const uint32_t *al, const uint32_t *bl, int nb_l) {
        #pragma unroll
        for (int v = 0; v < kPairBatch; ++v) {
            ok[v] = w.r < nb_l;
            eb[v] = ok[v] ? bl[w.r] : 0u;  // 0: rank 0, in bounds
            ea[v] = ok[v] ? al[w.i] : 0u;
            w.next();
        }
    }
};

// psi <- exp(theta G) psi over the op's pairs.
template <typename A>
__global__ void __launch_bounds__(kThreads) k_rotate_l(A *__restrict__ psi, const uint32_t *__restrict__ al,
                                                       int na_l, const uint32_t *__restrict__ bl, int nb_l, int Da,
                                                       real_of<A> c, real_of<A> sn) {
    using R = real_of<A>;
    if (na_l <= 0) return;
    PairWalk w(na_l);
    while (w.r < nb_l) {
        size_t I[kPairBatch], J[kPairBatch];
        bool ok[kPairBatch];
        R ss[kPairBatch];
        #pragma unroll
        for (int v = 0; v < kPairBatch; ++v) {
            ok[v] = w.r < nb_l;
            const uint32_t eb = ok[v] ? bl[w.r] : 0u, ea = ok[v] ? al[w.i] : 0u;  // 0: rank 0, in bounds
            I[v] = (size_t)(eb & 0x7FFFu) * Da + (ea & 0x7FFFu);
            J[v] = (size_t)(eb >> 16) * Da + (ea >> 16);
            ss[v] = ((ea ^ eb) & 0x8000u) ? -sn : sn;
            w.next();
        }
        A u[kPairBatch], x[kPairBatch];
        #pragma unroll
        for (int v = 0; v < kPairBatch; ++v) {
            u[v] = psi[I[v]];
            x[v] = psi[J[v]];
        }
        #pragma unroll
        for (int v = 0; v < kPairBatch; ++v) {
            if (!ok[v]) continue;
            psi[I[v]] = lin2<A>(c, u[v], -ss[v], x[v]);
            psi[J[v]] = lin2<A>(c, x[v], ss[v], u[v]);
        }
    }
}

// Adjoint step over the op's pairs: the gradient term, then U^dagger on psi and
// lambda; one float64 partial per block (fixed order: every block writes its entry).
template <typename A>
__global__ void __launch_bounds__(kThreads) k_adjoint_l(A *__restrict__ psi, A *__restrict__ lam,
                                                        const uint32_t *__restrict__ al, int na_l,
                                                        const uint32_t *__restrict__ bl, int nb_l, int Da,
                                                        real_of<A> c, real_of<A> sn, double *__restrict__ partial) {
    using R = real_of<A>;
    __shared__ double red[kThreads / 32];
    double acc = 0.0;
    if (na_l > 0) {
        PairWalk w(na_l);
        while (w.r < nb_l) {
            size_t I[kPairBatch], J[kPairBatch];
            bool ok[kPairBatch], neg[kPairBatch];
            #pragma unroll
            for (int v = 0; v < kPairBatch; ++v) {
                ok[v] = w.r < nb_l;
                const uint32_t eb = ok[v] ? bl[w.r] : 0u, ea = ok[v] ? al[w.i] : 0u;
                I[v] = (size_t)(eb & 0x7FFFu) * Da + (ea & 0x7FFFu);
                J[v] = (size_t)(eb >> 16) * Da + (ea >> 16);
                neg[v] = ((ea ^ eb) & 0x8000u) != 0u;
                w.next();
            }
            A u[kPairBatch], x[kPairBatch], lu[kPairBatch], lx[kPairBatch];
            #pragma unroll
            for (int v = 0; v < kPairBatch; ++v) {
                u[v] = psi[I[v]];
                x[v] = psi[J[v]];
                lu[v] = lam[I[v]];
                lx[v] = lam[J[v]];
            }
            R t = 0;
            #pragma unroll
            for (int v = 0; v < kPairBatch; ++v) {
                if (!ok[v]) continue;
                const R ti = re_dot(lx[v], u[v]) - re_dot(lu[v], x[v]);
                t += neg[v] ? -ti : ti;
                const R ss = neg[v] ? -sn : sn;
                psi[I[v]] = lin2<A>(c, u[v], ss, x[v]);
                psi[J[v]] = lin2<A>(c, x[v], -ss, u[v]);
                lam[I[v]] = lin2<A>(c, lu[v], ss, lx[v]);
                lam[J[v]] = lin2<A>(c, lx[v], -ss, lu[v]);
            }
            acc += (double)t;
        }
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// The same adjoint step on the interleaved matrix CL[2 e] = psi[e], CL[2 e + 1] = lam[e]:
// one vector load / store per amplitude moves both, so each pair costs two scattered
// accesses instead of four and every 32-byte L2 sector it touches carries twice the
// useful bytes.  Same arithmetic in the same order as k_adjoint_l.
template <typename A>
struct alignas(2 * sizeof(A)) AmpPair {
    A c, l;
};

template <typename A>
__global__ void __launch_bounds__(kThreads) k_adjoint_li(A *__restrict__ CL, const uint32_t *__restrict__ al, int na_l,
                                                         const uint32_t *__restrict__ bl, int nb_l, int Da,
                                                         real_of<A> c, real_of<A> sn, double *__restrict__ partial) {
    using R = real_of<A>;
    __shared__ double red[kThreads / 32];
    AmpPair<A> *P = reinterpret_cast<AmpPair<A> *>(CL);
    double acc = 0.0;
    if (na_l > 0) {
        PairWalk w(na_l);
        while (w.r < nb_l) {
            size_t I[kPairBatch], J[kPairBatch];
            bool ok[kPairBatch], neg[kPairBatch];
            #pragma unroll
            for (int v = 0; v < kPairBatch; ++v) {
                ok[v] = w.r < nb_l;
                const uint32_t eb = ok[v] ? bl[w.r] : 0u, ea = ok[v] ? al[w.i] : 0u;
                I[v] = (size_t)(eb & 0x7FFFu) * Da + (ea & 0x7FFFu);
                J[v] = (size_t)(eb >> 16) * Da + (ea >> 16);
                neg[v] = ((ea ^ eb) & 0x8000u) != 0u;
                w.next();
            }
            AmpPair<A> pu[kPairBatch], px[kPairBatch];
            #pragma unroll
            for (int v = 0; v < kPairBatch; ++v) {
                pu[v] = P[I[v]];
                px[v] = P[J[v]];
            }
            R t = 0;
            #pragma unroll
            for (int v = 0; v < kPairBatch; ++v) {
                if (!ok[v]) continue;
                const A u = pu[v].c, x = px[v].c, lu = pu[v].l, lx = px[v].l;
                const R ti = re_dot(lx, u) - re_dot(lu, x);
                t += neg[v] ? -ti : ti;
                const R ss = neg[v] ? -sn : sn;
                AmpPair<A> ou, ox;
                ou.c = lin2<A>(c, u, ss, x);
                ox.c = lin2<A>(c, x, -ss, u);
                ou.l = lin2<A>(c, lu, ss, lx);
                ox.l = lin2<A>(c, lx, -ss, lu);
                P[I[v]] = ou;
                P[J[v]] = ox;
            }
            acc += (double)t;
        }
    }
    const double s = block_sum(acc, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// ---------------------------------------------------------------- whole sweeps in one launch

// The forward and reverse sweeps as one persistent launch each: the grid walks the
// operators in order, every block taking its share of an operator's pairs exactly as
// k_rotate_l / k_adjoint_li do, with a grid-wide barrier between operators (an
// operator reads amplitudes the previous one wrote in other blocks).  The per-operator
// launches of sector storage are latency bound (a few microseconds of work each on
// L2-resident data): one launch replaces their launch gaps and ramp-ups with barriers.
// Launched cooperatively, so every block is resident and every barrier can complete;
// each wait is still bounded -- past the limit the block sets *err and stops, and the
// call reports the failure.
struct SweepArgs {
    const uint32_t *lists;   // the ops' pair lists (k_build_lists)
    const int4 *info;        // per op: alpha offset, alpha length, beta offset, beta length
    const double2 *cs;       // per op: (cos theta, sin theta)
    int n_ops, Da, Db;
    unsigned int *bar;       // barrier arrivals, zero at launch
    int *err;                // set to 1 when a barrier wait runs out
    uint32_t spins;          // polls of a barrier wait
    double *partial;         // reverse sweep: [n_ops][gridDim.x] gradient partials
};

// Grid-wide barrier number `gen` (0, 1, ...): every block arrives once per barrier.
__device__ __forceinline__ bool sweep_barrier(const SweepArgs &g, unsigned int gen, volatile int *s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(g.bar, 1u);
        const unsigned int target = (gen + 1u) * gridDim.x;
        bool ok = true;
        for (uint32_t it = 0; *(volatile unsigned int *)g.bar < target; ++it) {
            if (it >= g.spins) {
                ok = false;
                atomicExch(g.err, 1);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok;
}

template <typename A>
__global__ void __launch_bounds__(kThreads) k_sweep_rotate_l(A *__restrict__ psi, SweepArgs g) {
    using R = real_of<A>;
    __shared__ volatile int s_ok;
    unsigned int gen = 0;
    for (int k = 0; k < g.n_ops; ++k) {
        const int4 li = g.info[k];
        const int na_l = li.y, nb_l = li.w;
        if (na_l <= 0 || nb_l <= 0) continue;  // no pair in the sector: nothing written, no barrier
        const uint32_t *al = g.lists + li.x, *bl = g.lists + li.z;
        PairWalk w(na_l);
        bool more = w.r < nb_l;
        PairBatch cur;
        cur.load(w, al, bl, nb_l);
        if (gen > 0 && !sweep_barrier(g, gen - 1, &s_ok)) return;
        ++gen;
        const R c = (R)g.cs[k].x, sn = (R)g.cs[k].y;
        while (more) {
            size_t I[kPairBatch], J[kPairBatch];
            R ss[kPairBatch];
            #pragma unroll
            for (int v = 0; v < kPairBatch; ++v) {
                I[v] = (size_t)(cur.eb[v] & 0x7FFFu) * g.Da + (cur.ea[v] & 0x7FFFu);
                J[v] = (size_t)(cur.eb[v] >> 16) * g.Da + (cur.ea[v] >> 16);
                ss[v] = ((cur.ea[v] ^ cur.eb[v]) & 0x8000u) ? -sn : sn;
                if (!(SV_IN_RANGE(I[v], (size_t)g.Da * g.Db, kChkPair) && SV_IN_RANGE(J[v], (size_t)g.Da * g.Db, kChkPair))) {
                    cur.ok[v] = false;  // checked build: skip the pair
                    I[v] = J[v] = 0;
                }
            }
            A u[kPairBatch], x[kPairBatch];
            #pragma unroll
            for (int v = 0; v < kPairBatch; ++v) {
                u[v] = psi[I[v]];
                x[v] = psi[J[v]];
            }
            more = w.r < nb_l;
            PairBatch nxt;
            if (more) nxt.load(w, al, bl, nb_l);
            #pragma unroll
            for (int v = 0; v < kPairBatch; ++v) {
                if (!cur.ok[v]) continue;
                psi[I[v]] = lin2<A>(c, u[v], -ss[v], x[v]);
                psi[J[v]] = lin2<A>(c, x[v], ss[v], u[v]);
            }
            if (more) cur = nxt;
        }
    }
}

// Reverse sweep on the interleaved (psi, lambda) matrix, ops n_ops - 1 down to 0; the
// arithmetic of k_adjoint_li, one float64 partial per block and op (fixed order).
template <typename A>
__global__ void __launch_bounds__(kThreads) k_sweep_adjoint_li(A *__restrict__ CL, SweepArgs g) {
    using R = real_of<A>;
    __shared__ double red[kThreads / 32];
    __shared__ volatile int s_ok;
    AmpPair<A> *P = reinterpret_cast<AmpPair<A> *>(CL);
    unsigned int gen = 0;
    for (int k = g.n_ops - 1; k >= 0; --k) {
        const int4 li = g.info[k];
        const int na_l = li.y, nb_l = li.w;
        double acc = 0.0;
        if (na_l > 0 && nb_l > 0) {
            const uint32_t *al = g.lists + li.x, *bl = g.lists + li.z;
            PairWalk w(na_l);
            bool more = w.r < nb_l;
            PairBatch cur;
            cur.load(w, al, bl, nb_l);
            if (gen > 0 && !sweep_barrier(g, gen - 1, &s_ok)) return;
            ++gen;
            const R c = (R)g.cs[k].x, sn = (R)g.cs[k].y;
            while (more) {
                size_t I[kPairBatch], J[kPairBatch];
                bool neg[kPairBatch];
                #pragma unroll
                for (int v = 0; v < kPairBatch; ++v) {
                    I[v] = (size_t)(cur.eb[v] & 0x7FFFu) * g.Da + (cur.ea[v] & 0x7FFFu);
                    J[v] = (size_t)(cur.eb[v] >> 16) * g.Da + (cur.ea[v] >> 16);
                    neg[v] = ((cur.ea[v] ^ cur.eb[v]) & 0x8000u) != 0u;
                    if (!(SV_IN_RANGE(I[v], (size_t)g.Da * g.Db, kChkPair) &&
                          SV_IN_RANGE(J[v], (size_t)g.Da * g.Db, kChkPair))) {
                        cur.ok[v] = false;  // checked build: skip the pair
                        I[v] = J[v] = 0;
                    }
                }
                AmpPair<A> pu[kPairBatch], px[kPairBatch];
                #pragma unroll
                for (int v = 0; v < kPairBatch; ++v) {
                    pu[v] = P[I[v]];
                    px[v] = P[J[v]];
                }
                more = w.r < nb_l;
                PairBatch nxt;
                if (more) nxt.load(w, al, bl, nb_l);
                R t = 0;
                #pragma unroll
                for (int v = 0; v < kPairBatch; ++v) {
                    if (!cur.ok[v]) continue;
                    const A u = pu[v].c, x = px[v].c, lu = pu[v].l, lx = px[v].l;
                    const R ti = re_dot(lx, u) - re_dot(lu, x);
                    t += neg[v] ? -ti : ti;
                    const R ss = neg[v] ? -sn : sn;
                    AmpPair<A> ou, ox;
                    ou.c = lin2<A>(c, u, ss, x);
                    ox.c = lin2<A>(c, x, -ss, u);
                    ou.l = lin2<A>(c, lu, ss, lx);
                    ox.l = lin2<A>(c, lx, -ss, lu);
                    P[I[v]] = ou;
                    P[J[v]] = ox;
                }
                acc += (double)t;
                if (more) cur = nxt;
            }
        }
        const double s = block_sum(acc, red);
        if (threadIdx.x == 0) g.partial[(size_t)k * gridDim.x + blockIdx.x] = s;
    }
}

// The row sums' arithmetic: float32 or float64 for those states, float-float (hi + lo
// float32 words, error-free transformations) for float64 states converted to it.
__device__ __forceinline__ double to_double(float x) { return (double)x; }
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(ff x) { return ff_to(x); }
__device__ __forceinline__ ff re_dot(ffc u, ffc v) { return ff_fma(u.y, v.y, u.x * v.x); }
__device__ __forceinline__ ff im_dot(ffc u, ffc v) { return ff_fma(u.x, v.y, -(u.y * v.x)); }
__device__ __forceinline__ ff re_dot(ff u, ff v) { return u * v; }
__device__ __forceinline__ ff im_dot(ff, ff) { return ff(0, 0); }
// fixed shuffle tree as warp_sum, each step a float-float addition
__device__ __forceinline__ ff warp_sum(ff v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ff w;
        w.hi = __shfl_down_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_down_sync(0xffffffffu, v.lo, o);
        v = v + w;
    }
    return v;
}

// Density matrix by rows: a block takes beta strings (rows) Ib = blockIdx.x,
// blockIdx.x + gridDim.x, ...; for each row
//   norm and alpha occupations   sum_a |C[b][a]|^2 (a_p)                (all warps)
//   beta occupations             the row norm when b holds p
//   alpha pairs p < q            sum over a with q in a, p not in a of
//                                conj(C[b][a']) C[b][a] (-1)^popc(x & between(2p, 2q)), a' = a - q + p
//                                (those a from the pair's list, built once per sector)
//   beta pairs p < q (b holds q, not p)
//                                sum_a conj(C[b'][a]) C[b][a] (-1)^popc(x & between(2p+1, 2q+1))
// (x = spread(a) | spread(b)), in the element order norm, n occupations
// (j = 2p + sigma), alpha pairs, beta pairs.  Each pair element belongs to one warp
// (pairs dealt round-robin to the warps), which sums it over the row with its lanes
// and one warp reduction; the norm and occupations are summed by every warp over a
// share of the row.  Each warp writes its sums to its own shared slots; after each row
// the block adds them (the owner's slot for a pair element, the warps in order for the
// others) into float64 running sums, written to partial[e][blockIdx.x] at the end:
// fixed-order sums.
template <typename A>
__global__ void __launch_bounds__(kThreads) k_rdm_rows(const A *__restrict__ C, SectTabs T, int N,
                                                       const uint32_t *__restrict__ alist,
                                                       const int4 *__restrict__ ainfo,
                                                       double *__restrict__ partial) {
    using R = real_of<A>;
    extern __shared__ double rdm_s[];  // [2 n_el] running sums, then [kThreads/32][2 n_el] warp slots
    const int n = 2 * N, npair = N * (N - 1) / 2, n_el = 1 + n + 2 * npair, W = 2 * n_el;
    constexpr int NW = kThreads / 32;
    double *acc = rdm_s, *slot = rdm_s + W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *my = slot + warp * W;
    for (int i = threadIdx.x; i < W; i += blockDim.x) acc[i] = 0.0;
    for (int Ib = blockIdx.x; Ib < T.Db; Ib += gridDim.x) {
        const uint32_t b = T.strb[Ib], xb = T.sb[Ib];
        const A *row = C + (size_t)Ib * T.Da;
        // norm and alpha occupations (every warp, a share of the row)
        R nrm = 0, occ[16];
        #pragma unroll
        for (int p = 0; p < 16; ++p) occ[p] = 0;
        for (int Ia = threadIdx.x; Ia < T.Da; Ia += blockDim.x) {
            const A c = row[Ia];
            const R w = re_dot(c, c);
            const uint32_t a = T.stra[Ia];
            nrm += w;
            #pragma unroll
            for (int p = 0; p < 16; ++p)
                if ((a >> p) & 1u) occ[p] += w;
        }
        nrm = warp_sum(nrm);
        if (lane == 0) {
            my[0] = to_double(nrm);
            my[1] = 0.0;
        }
        #pragma unroll
        for (int p = 0; p < 16; ++p) {
            if (p >= N) break;
            const R s = warp_sum(occ[p]);
            if (lane == 0) {
                my[2 * (1 + 2 * p)] = to_double(s);
                my[2 * (1 + 2 * p) + 1] = 0.0;
                my[2 * (2 + 2 * p)] = ((b >> p) & 1u) ? to_double(nrm) : 0.0;
                my[2 * (2 + 2 * p) + 1] = 0.0;
            }
        }
        // pair elements: element e = 1 + n + k (k = 0 .. 2 npair - 1; alpha pairs first) to warp k % NW
        for (int k = warp; k < 2 * npair; k += NW) {
            const int s = k >= npair, kk = s ? k - npair : k;
            int p = 0, rem = kk;
            while (rem >= N - 1 - p) {
                rem -= N - 1 - p;
                ++p;
            }
            const int q = p + 1 + rem, e = 1 + n + k;
            const uint32_t m = (1u << p) | (1u << q), f = 1u << q;
            const uint32_t bm = between(2 * p + s, 2 * q + s);
            R re = 0, im = 0;
            if (s == 0) {
                // the alpha strings holding q but not p, from the pair's list: entry =
                // rank | parity of its alpha bits under bm << 15 | partner rank << 16
                const int4 li = ainfo[kk];
                const uint32_t *L = alist + li.x, rsg = (uint32_t)par(xb & bm);
                for (int i = lane; i < li.y; i += 32) {
                    const uint32_t ea = L[i];
                    if (!(SV_IN_RANGE(ea & 0x7FFFu, T.Da, kChkRank) && SV_IN_RANGE(ea >> 16, T.Da, kChkRank)))
                        continue;  // checked build: skip the entry
                    const A u = row[ea & 0x7FFFu], v = row[ea >> 16];
                    R ar = re_dot(v, u), ai = im_dot(v, u);  // conj(v) u
                    if (((ea >> 15) & 1u) ^ rsg) { ar = -ar; ai = -ai; }
                    re += ar;
                    im += ai;
                }
            } else if ((b & m) == f) {
                const uint32_t r2 = T.rb[b ^ m];
                if (SV_IN_RANGE(r2, T.Db, kChkRank)) {  // checked build: a bad rank skips the partner row
                    const A *row2 = C + (size_t)r2 * T.Da;
                    for (int Ia = lane; Ia < T.Da; Ia += 32) {
                        const A u = row[Ia], v = row2[Ia];
                        R ar = re_dot(v, u), ai = im_dot(v, u);
                        if (par((T.sa[Ia] | xb) & bm)) { ar = -ar; ai = -ai; }
                        re += ar;
                        im += ai;
                    }
                }
            }
            re = warp_sum(re);
            im = warp_sum(im);
            if (lane == 0) {
                my[2 * e] = to_double(re);
                my[2 * e + 1] = to_double(im);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < W; i += blockDim.x) {
            const int e = i >> 1;
            double t = 0.0;
            if (e < 1 + n) {
                for (int w = 0; w < NW; ++w) t += slot[w * W + i];
            } else {
                t = slot[((e - 1 - n) % NW) * W + i];
            }
            acc[i] += t;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < W; i += blockDim.x) partial[(size_t)i * gridDim.x + blockIdx.x] = acc[i];
}

// out[i] = C[idx[i]] or 0 when idx[i] is 0xFFFFFFFF (a basis state outside the sector)
template <typename A>
__global__ void k_gather_c(const A *__restrict__ psi, const uint32_t *__restrict__ idx, int count,
                           A *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        out[i] = idx[i] == 0xFFFFFFFFu ? mka<A>(0, 0) : psi[idx[i]];
}

// ---------------------------------------------------------------- launchers

static SectTabs tabs(const uint32_t *sa, const uint32_t *sb, const uint16_t *stra, const uint16_t *strb,
                     const uint16_t *ra, const uint16_t *rb, int Da, int Db) {
    SectTabs t;
    t.sa = sa; t.sb = sb; t.stra = stra; t.strb = strb; t.ra = ra; t.rb = rb; t.Da = Da; t.Db = Db;
    return t;
}

// Alpha / beta string parts of a qubit-space op.
static void sect_op_from(const OpDesc &d, int N, SectOp *dst) {
    SectOp o;
    o.sm = d.sm;
    o.ma = o.fa = o.mb = o.fb = 0;
    for (int q = 0; q < N; ++q) {
        if ((d.m >> (2 * q)) & 1u) o.ma |= 1u << q;
        if ((d.from >> (2 * q)) & 1u) o.fa |= 1u << q;
        if ((d.m >> (2 * q + 1)) & 1u) o.mb |= 1u << q;
        if ((d.from >> (2 * q + 1)) & 1u) o.fb |= 1u << q;
    }
    *dst = o;
}

// Blocks of the list kernels: one per beta-list entry, at most bps per SM (8 by default).
int sector_grid(int Db, int sm_count, int bps) {
    const int cap = sm_count * (bps > 0 ? bps : 8);
    return Db < cap ? Db : cap;
}

// Host side of the lists: counts from the patterns, offsets, and the build launch.
static uint64_t choose(int n, int k) {
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

size_t list_op_bytes() { return sizeof(ListOp); }

// Fill the ListOp of op d (qubit-space masks) for a sector with na / nb electrons
// among N orbitals: its alpha list at entry a_off, its beta list right after it.
// Returns the alpha and beta list lengths through na_l, nb_l.
void list_op_from(const OpDesc &d, int N, int na, int nb, uint32_t a_off, void *dst, int *na_l, int *nb_l) {
    SectOp s;
    sect_op_from(d, N, &s);
    *na_l = (int)choose(N - __builtin_popcount(s.ma), na - __builtin_popcount(s.fa));
    *nb_l = (int)choose(N - __builtin_popcount(s.mb), nb - __builtin_popcount(s.fb));
    ListOp o;
    o.sm = s.sm; o.ma = s.ma; o.fa = s.fa; o.mb = s.mb; o.fb = s.fb;
    o.a_off = a_off;
    o.b_off = a_off + (uint32_t)*na_l;
    o.a_n = (uint32_t)*na_l;
    o.b_n = (uint32_t)*nb_l;
    *(ListOp *)dst = o;
}

cudaError_t launch_build_lists(const void *ops, int n_ops, const uint32_t *sa, const uint32_t *sb,
                               const uint16_t *stra, const uint16_t *strb, const uint16_t *ra, const uint16_t *rb,
                               int Da, int Db, uint32_t *out, cudaStream_t st) {
    if (n_ops <= 0) return cudaSuccess;
    SectTabs T = tabs(sa, sb, stra, strb, ra, rb, Da, Db);
    k_build_lists<<<2 * n_ops, kThreads, 0, st>>>((const ListOp *)ops, T, out);
    return cudaGetLastError();
}

cudaError_t launch_rotate_l(void *psi, int dtype, const uint32_t *al, int na_l, const uint32_t *bl, int nb_l, int Da,
                            double c, double s, int grid, cudaStream_t st) {
    if (na_l <= 0 || nb_l <= 0) return cudaSuccess;
    SV_DISPATCH_AMP(dtype, k_rotate_l<A><<<grid, kThreads, 0, st>>>((A *)psi, al, na_l, bl, nb_l, Da,
                                                                     (real_of<A>)c, (real_of<A>)s));
    return cudaGetLastError();
}

// partial: grid doubles (every block writes its entry, zero when it has no rows).
cudaError_t launch_adjoint_l(void *psi, void *lam, int dtype, const uint32_t *al, int na_l, const uint32_t *bl,
                             int nb_l, int Da, double c, double s, int grid, double *partial, cudaStream_t st) {
    SV_DISPATCH_AMP(dtype, k_adjoint_l<A><<<grid, kThreads, 0, st>>>((A *)psi, (A *)lam, al, na_l, bl, nb_l, Da,
                                                                      (real_of<A>)c, (real_of<A>)s, partial));
    return cudaGetLastError();
}

// CL: the interleaved (psi, lam) matrix (launch_interleave), 16-byte aligned.
cudaError_t launch_adjoint_li(void *CL, int dtype, const uint32_t *al, int na_l, const uint32_t *bl, int nb_l, int Da,
                              double c, double s, int grid, double *partial, cudaStream_t st) {
    SV_DISPATCH_AMP(dtype, k_adjoint_li<A><<<grid, kThreads, 0, st>>>((A *)CL, al, na_l, bl, nb_l, Da,
                                                                       (real_of<A>)c, (real_of<A>)s, partial));
    return cudaGetLastError();
}

// Blocks of a whole-sweep launch: at most bps per SM (8 by default) and no more than
// can be resident at once (a cooperative launch needs every block resident).
template <typename K>
static int sweep_grid_for(K kernel, int Db, int sm_count, int bps) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int want = bps > 0 ? bps : 8;
    if (per_sm > want) per_sm = want;
    const int cap = per_sm * sm_count;
    return Db < cap ? Db : cap;
}

int sweep_grid(int dtype, bool adjoint, int Db, int sm_count, int bps) {
    int grid = 0;
    SV_DISPATCH_AMP(dtype, grid = adjoint ? sweep_grid_for(k_sweep_adjoint_li<A>, Db, sm_count, bps)
                                          : sweep_grid_for(k_sweep_rotate_l<A>, Db, sm_count, bps));
    return grid;
}

// One cooperative launch of the forward (adjoint = false: ops 0 .. n_ops-1 on psi) or the
// reverse sweep (adjoint = true: ops n_ops-1 .. 0 on the interleaved matrix, gradient
// partials [n_ops][grid] into partial).  info: the ops' int4 list records (device), cs
// their (cos, sin) (device), bar a zeroed device counter, err the device error flag.
// A refused cooperative launch returns its error (the caller falls back to one launch
// per op).
cudaError_t launch_sweep_l(void *buf, int dtype, bool adjoint, const uint32_t *lists, const int *info,
                           const double *cs, int n_ops, int Da, int Db, int grid, unsigned int *bar, int *err,
                           uint32_t spins, double *partial, cudaStream_t st) {
    if (n_ops <= 0) return cudaSuccess;
    if (grid <= 0) return cudaErrorInvalidValue;
    SweepArgs g;
    g.lists = lists; g.info = (const int4 *)info; g.cs = (const double2 *)cs; g.n_ops = n_ops; g.Da = Da; g.Db = Db;
    g.bar = bar; g.err = err; g.spins = spins; g.partial = partial;
    void *args[] = {&buf, &g};
    cudaError_t e = cudaErrorInvalidValue;
    SV_DISPATCH_AMP(dtype, e = cudaLaunchCooperativeKernel(
                               adjoint ? (const void *)k_sweep_adjoint_li<A> : (const void *)k_sweep_rotate_l<A>,
                               dim3(grid), dim3(kThreads), args, 0, st));
    return e;
}

int rdm_rows_elements(int n) { return 1 + n + (n / 2) * (n / 2 - 1); }

int rdm_rows_grid(int Db, int sm_count, int bps) {
    const int cap = sm_count * (bps > 0 ? bps : 4);
    return Db < cap ? Db : cap;
}

// partial: [2 n_el][grid] doubles (n_el = rdm_rows_elements(n)), reduced by launch_reduce_rows.
// alist / ainfo: the alpha-pair lists (one list op per pair p < q in (p, q) order with flip
// mask {p, q}, "from" pattern {q} and sign mask between(2p, 2q)) and their int4 records.
// ff_form: C holds the float-float form of a float64 state (ffc for complex128, ff for
// float64), as launch_to_ff writes it.
cudaError_t launch_rdm_rows(const void *C, int dtype, int ff_form, int n, const uint32_t *sa, const uint32_t *sb,
                            const uint16_t *stra, const uint16_t *strb, const uint16_t *ra, const uint16_t *rb, int Da,
                            int Db, int grid, const uint32_t *alist, const int *ainfo, double *partial,
                            cudaStream_t st) {
    SectTabs T = tabs(sa, sb, stra, strb, ra, rb, Da, Db);
    const size_t smem = sizeof(double) * 2 * rdm_rows_elements(n) * (1 + kThreads / 32);  // <= 40 KB (n <= 32)
    if (ff_form) {
        if (dtype == SV_C128)
            k_rdm_rows<ffc><<<grid, kThreads, smem, st>>>((const ffc *)C, T, n / 2, alist, (const int4 *)ainfo, partial);
        else if (dtype == SV_R64)
            k_rdm_rows<ff><<<grid, kThreads, smem, st>>>((const ff *)C, T, n / 2, alist, (const int4 *)ainfo, partial);
        else
            return cudaErrorInvalidValue;  // single-precision states have no float-float form
        return cudaGetLastError();
    }
    SV_DISPATCH_AMP(dtype, k_rdm_rows<A><<<grid, kThreads, smem, st>>>((const A *)C, T, n / 2, alist,
                                                                       (const int4 *)ainfo, partial));
    return cudaGetLastError();
}

cudaError_t launch_gather_c(const void *psi, int dtype, const uint32_t *idx, int count, void *out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    int grid = (count + kThreads - 1) / kThreads;
    if (grid > 1024) grid = 1024;
    SV_DISPATCH_AMP(dtype, k_gather_c<A><<<grid, kThreads, 0, st>>>((const A *)psi, idx, count, (A *)out));
    return cudaGetLastError();
}

// This unit's check word (checked build), for sv_check_status.
SV_CHECK_READER(check_word_sector)

}  // namespace svk
