// k_abtc.cu -- the alpha-beta part of sigma~ = phi sigma (expectation variant 5) as
// products on the tensor cores.
//
// In the string-blocked basis (all alpha creators before all beta creators) the
// alpha-beta part of H is sum_{pq,rs} (pq|rs) E^a_pq E^b_rs with the sign of E^a_pq
// taken on the alpha string alone and that of E^b_rs on the beta string alone (a pair
// of fermion operators passes the other spin's creators without a sign).  For an
// output string pair (a, b):
//   sigma~_ab(a, b) = sum over beta excitations r -> s of b (partner b' = b - r + s) of
//                       s_b(b, rs) H[b'][col(b', rs)][a]  +  H[b][own][a]
//   H[b'][j][a] = sum_kappa A_b'[a][kappa] B[j(b')][kappa]
// over kappa = the N orbitals p (diagonal, kappa = p) and the N (N - 1) / 2 unordered
// pairs p < q (kappa = N + pair index): (pq|rs) = (qp|rs) for real orbitals, so one K
// entry serves both directions, and for a given a at most one direction applies:
//   A_b'[a][p]      = X(a, b') if p in a, else 0,
//   A_b'[a][{p,q}]  = s_a(a, pq) X(a ^ {p, q}, b') if exactly one of p, q is in a, else 0,
//   B[j][p]         = (pp|sr),  B[j][{p,q}] = (qp|sr) for the j-th excitation (s in b',
//                     r not in b') of b',
//   B[own][p] = 0,  B[own][{p,q}] = sum_{l in b'} (qp|ll),
// with X = phi C (phi(a, b) = (-1)^popc(a & pp(b))) and s_a the parity of a's bits
// strictly between p and q.  The p = q, own-column term (the alpha-beta Coulomb
// diagonal) is left to the diagonal.  Per b' the columns are its nb (N - nb)
// excitations plus the own column (at most 51 where N <= 16 and each spin has at most 4096
// strings), padded to 64; K = N (N + 1) / 2 <= 136, padded to a multiple of 16.
//
// k_ab_tc: a persistent kernel over units (128-string alpha tile, partner row b').
// Sixteen builder warps (four per tile row, four K each) stage the b' row of X as bf16
// pieces (written once per sigma by the phase kernel: per amplitude three words
// (re_k | im_k << 16), k = 1, 2, 3; asynchronous copies, one unit ahead), gather A for
// the tile's rows K = 16 at a time through a per-tile table (partner offset | sign per
// row and kappa, rebuilt when the tile changes), flipping sign bits and pairing halves
// only, and write it to tensor memory (tcgen05.st: each builder warp its lane quarter,
// row = lane, two K per column), where the MMAs read A; they copy the unit's B rows
// (pieces of a precomputed table, the rows named by a per-partner-row column table read
// one unit ahead) into shared memory in the canonical no-swizzle
// K-major layout (core matrices of 8 rows x 16 bytes);
// lane 0 of warp 16 issues tcgen05.mma kind::f16 (six piece products per plane:
// float32-level accuracy) into one of two tensor-memory accumulators; eight epilogue
// warps (two per tensor-memory lane quarter) drain each finished accumulator into H
// while the next unit is built.  Stage ring with full / empty mbarriers, accumulator
// full / empty mbarriers; all waits bounded (past the limit: *err set, copies and MMAs
// waited for, tensor memory freed, return).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sv_check.cuh"
#include "sv_internal.h"

namespace svk {

namespace {

constexpr int kAbBuild = 512;                  // builder threads (16 warps): 4 per tile row
constexpr int kAbKpt = 4;                      // K entries of a stage per builder thread (16 / 4)
constexpr int kAbEpi = 256;                    // epilogue threads (8 warps: two per tensor-memory lane quarter)
constexpr int kAbThreadsTc = kAbBuild + 32 + kAbEpi;  // builders, the MMA warp, the epilogue warps
constexpr int kAbM = 128;                      // alpha strings per tile
constexpr int kAbKc = 16;                      // K (orbitals and orbital pairs) per stage
constexpr int kAbS = 4;                        // stages
constexpr int kAbMaxK = 144;                   // N (N + 1) / 2 <= 136 for N <= 16, padded to 16
constexpr int kAbMaxN = 64;                    // columns per accumulator: nb (N - nb) + 1 <= 51 within the limits
constexpr int kAbACols = kAbKc / 2;            // tensor-memory columns of one bf16 piece of A (two K per column)
constexpr int kAbAccCols = 2 * kAbMaxN;        // one accumulator: both planes
constexpr int kAbAStage = 6 * kAbACols;        // A columns per stage: 2 planes x 3 pieces
constexpr int kAbABase = 2 * kAbAccCols;       // first A column (after the two accumulators)
static_assert(kAbABase + kAbS * kAbAStage <= 512, "tensor memory: accumulators and A stages in 512 columns");

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// One poll: a try-wait that suspends the thread until the phase completes or at most
// kAbPollNs nanoseconds have passed (a thread waiting here wakes as soon as the phase
// completes, and takes no issue slots meanwhile).
constexpr uint32_t kAbPollNs = 64;
__device__ __forceinline__ bool ab_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity), "n"(kAbPollNs)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool ab_wait(uint32_t mbar, uint32_t parity, uint32_t spins) {
    for (uint32_t it = 0; it < spins; ++it)
        if (ab_try(mbar, parity)) return true;
    return false;
}

__device__ __forceinline__ void ab_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void ab_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void builders_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kAbBuild) : "memory"); }

// Barrier over the builder warps (named barrier 1) or the epilogue warps (2) that also
// returns, to every thread of the group, whether any of them passed `v` true: a
// decision the whole group takes the same way.
__device__ __forceinline__ bool builders_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kAbBuild)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ bool epi_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 2, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(kAbEpi)
        : "memory");
    return r != 0;
}

// Canonical no-swizzle K-major descriptor: K-adjacent core matrices 128 bytes apart,
// adjacent 8-row groups 256 bytes apart (16 K elements = two 16-byte cores per row).
__device__ __forceinline__ uint64_t ab_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(256u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// The twelve (P = 2) or six MMAs of one K block in stage S: per plane the six piece products
// (A piece, B piece) = (0,0) (0,1) (1,0) (0,2) (1,1) (2,0) into the plane's accumulator
// (columns dacc + plane kAbMaxN).  Every operand is a compile-time offset from the
// loop-invariant tensor-memory base and B descriptor, so the issuing thread spends a
// few instructions per MMA; `first` starts the accumulation (the unit's first K block).
constexpr int kAbStageBytes = 3 * kAbMaxN * kAbKc * 2;  // B ring stage: three pieces of 64 rows x 16 K
template <int P, int S>
__device__ __forceinline__ void ab_mma_stage(uint32_t tmem, uint64_t d0, uint32_t dacc, uint32_t idesc, uint32_t first) {
    constexpr int pa[6] = {0, 0, 1, 0, 1, 2}, pbk[6] = {0, 1, 0, 2, 1, 0};
    constexpr uint32_t kPieceD = (kAbMaxN * kAbKc * 2) >> 4, kStageD = kAbStageBytes >> 4;
    #pragma unroll
    for (int pl = 0; pl < P; ++pl) {
        #pragma unroll
        for (int x = 0; x < 6; ++x) {
            // A from tensor memory (lanes = tile rows, two K per column), B from shared memory;
            // B descriptor: that of the ring's start plus the byte offset in 16-byte units (the
            // start-address field does not carry: shared addresses < 256 KB)
            const uint32_t ta = tmem + (uint32_t)(kAbABase + S * kAbAStage + (pl * 3 + pa[x]) * kAbACols);
            const uint64_t db = d0 + (uint64_t)(S * kStageD + pbk[x] * kPieceD);
            const uint32_t acc = x > 0 ? 1u : first ^ 1u;
            asm volatile(
                "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, q;\n\t}\n" ::"r"(dacc + (uint32_t)(pl * kAbMaxN)),
                "r"(ta), "l"(db), "r"(idesc), "r"(acc)
                : "memory");
        }
    }
}

// byte offset of (row r, 16-byte column kc) in a tile of 16 K
__device__ __forceinline__ uint32_t ab_off(int r, int kc) { return (uint32_t)(((r >> 3) * 2 + kc) * 128 + (r & 7) * 16); }

__device__ __forceinline__ void split3(float v, uint32_t &p1, uint32_t &p2, uint32_t &p3) {
    const __nv_bfloat16 a = __float2bfloat16_rn(v);
    const float r = v - __bfloat162float(a);
    const __nv_bfloat16 b = __float2bfloat16_rn(r);
    const __nv_bfloat16 c = __float2bfloat16_rn(r - __bfloat162float(b));
    p1 = __bfloat16_as_ushort(a);
    p2 = __bfloat16_as_ushort(b);
    p3 = __bfloat16_as_ushort(c);
}

__device__ __forceinline__ int ab_par(uint32_t x) { return __popc(x) & 1; }

// bits strictly between i and j
__device__ __forceinline__ uint32_t ab_between(int i, int j) {
    const int lo = min(i, j), hi = max(i, j);
    return ((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u);
}


}  // namespace

struct AbTcArgs {
    const uint32_t *Xi;       // [Db][ldi][3]: per amplitude of X = phi C, words (re_k | im_k << 16), k = 1, 2, 3
    int ldi;                  // row stride of Xi in amplitudes (a multiple of 4: 16-byte rows)
    const uint16_t *stra, *strb, *ra;
    const uint16_t *Bp;       // pieces [3][rowsB][256] of the B table (rows: N^2 integral rows, Db own rows, a zero row)
    const uint16_t *rowB;     // [Db][64]: the B-table row of each column of partner row b' (k_ab_rows)
    size_t pb;                // piece stride of Bp (elements)
    float *H;                 // planes [P][Db][ncols][ldh]
    int ldh;                  // row stride of H (floats, a multiple of 32: 128-byte rows)
    size_t hplane;
    int Da, Db, N, na, nb, ncols, nK, units;
    uint32_t maskN;
    int *err;
    uint32_t spins;           // mbarrier polls (each with a short sleep) before a wait gives up
    int stall;                // test hook: the builders stage and write nothing, so the MMA issuer's
                              // and the epilogue's first waits run out with nothing in flight
};

// K entries per tile row in the table (nK * 16) plus 4: an odd number of 8-byte words
// per row, so the builders' 8-byte reads of 16 consecutive rows hit distinct bank pairs.
__host__ __device__ __forceinline__ int ab_tstride(int nK) { return nK * kAbKc + 4; }

template <int P>
__global__ void __launch_bounds__(kAbThreadsTc, 1) k_ab_tc(AbTcArgs g) {
    extern __shared__ uint8_t ab_smem[];
    __shared__ __align__(8) uint64_t full[kAbS], empty[kAbS], accf[2], acce[2], done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;
    __shared__ uint8_t s_kp[kAbMaxK], s_kq[kAbMaxK];
    // dynamic: stage ring of B (1024-aligned), the two staged X rows, the tile's table; the A
    // stages live in tensor memory (columns kAbABase + s kAbAStage + (plane 3 + piece) kAbACols)
    constexpr int kStageBytes = kAbStageBytes;
    const uint32_t raw = su32(ab_smem), sbase = (raw + 1023u) & ~1023u;
    uint8_t *ring = ab_smem + (sbase - raw);
    // staged X rows: ldi amplitudes copied, then 4 zero amplitudes (what zero table entries read)
    const int xstride = (g.ldi + 4) * 3;                                        // words per row buffer
    uint32_t *xrow = reinterpret_cast<uint32_t *>(ring + kAbS * kStageBytes);  // [2][ldi + 4][3]
    uint16_t *tbl = reinterpret_cast<uint16_t *>(xrow + 2 * (size_t)xstride);  // [128][tstride]
    const int tid = threadIdx.x, warp = tid >> 5;
    const int N = g.N, ncolsP = kAbMaxN, tstride = ab_tstride(g.nK);
    const int Ktot = N * (N + 1) / 2;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(&tmem_base))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == kAbBuild) {
        s_fail = 0;
        for (int s = 0; s < kAbS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&full[s])), "n"(kAbBuild) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty[s])) : "memory");
        }
        for (int t = 0; t < 2; ++t) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&accf[t])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&acce[t])), "n"(kAbEpi) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < 12; i += kAbThreadsTc) {  // the zero amplitudes after each row buffer
        xrow[g.ldi * 3 + i] = 0u;
        xrow[xstride + g.ldi * 3 + i] = 0u;
    }
    // kappa -> (p, q): p = q = kappa below N, then the pairs p < q in order
    for (int k = tid; k < kAbMaxK; k += kAbThreadsTc) {
        int p = 0, q = 0;
        if (k < N) {
            p = q = k;
        } else if (k < Ktot) {
            int pi = k - N;
            while (pi >= N - 1 - p) { pi -= N - 1 - p; ++p; }
            q = p + 1 + pi;
        }
        s_kp[k] = (uint8_t)p;
        s_kq[k] = (uint8_t)q;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp < kAbBuild / 32 && g.stall) {
        // test hook: no copy, no tensor-memory store, no arrival
    } else if (warp < kAbBuild / 32) {
        // ------------------------------------------------------------ builders
        const int r = tid & (kAbM - 1), hf = tid >> 7;  // tile row; which 4 of a stage's 16 K
        const int rowbytes = g.ldi * 12;                // a multiple of 16
        const uint32_t zoff = (uint32_t)g.ldi * 3;      // table entry of a zero (the zero amplitude)
        auto stage_row = [&](int row, int buf) {        // asynchronous copy of X row `row`
            const uint8_t *src = reinterpret_cast<const uint8_t *>(g.Xi) + (size_t)row * rowbytes;
            uint8_t *dst = reinterpret_cast<uint8_t *>(xrow + (size_t)buf * xstride);
            for (int i = tid * 16; i < rowbytes; i += kAbBuild * 16)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst + i)), "l"(src + i) : "memory");
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        int cur_tile = -1, it = 0, gch = 0;
        // this thread's share of the B copies: entries i = tid + 256 k of (piece, row, core
        // column); shared-memory offsets fixed, global rows set per unit
        int bdst[1], bsel[1];
        #pragma unroll
        for (int k = 0; k < 1; ++k) {
            const int i = tid + k * kAbBuild;
            bsel[k] = i < ncolsP * 6 ? i : -1;
            const int ii = bsel[k] < 0 ? 0 : i, piece = ii / (ncolsP * 2), rem = ii - piece * ncolsP * 2;
            bdst[k] = piece * (ncolsP * kAbKc * 2) + (int)ab_off(rem >> 1, rem & 1);
        }
        const uint16_t *bsrc[1] = {g.Bp};
        int brow[1];
        #pragma unroll
        for (int k = 0; k < 1; ++k) {
            const int ii = bsel[k] < 0 ? 0 : bsel[k], rem = ii - (ii / (ncolsP * 2)) * ncolsP * 2;
            brow[k] = g.rowB[(size_t)((int)blockIdx.x % g.Db) * kAbMaxN + (rem >> 1)];
        }
        stage_row((int)blockIdx.x % g.Db, 0);
        for (int u = blockIdx.x; u < g.units; u += gridDim.x, ++it) {
            const int atile = u / g.Db, buf = it & 1;
            asm volatile("cp.async.wait_all;" ::: "memory");
            // this unit's row has landed; every builder is done with the previous unit
            if (builders_any(tid == 0 && s_fail)) break;
            const int un = u + (int)gridDim.x;  // the next unit
            if (un < g.units) stage_row(un % g.Db, buf ^ 1);
            if (atile != cur_tile) {
                // the tile's table: per row and kappa, the word offset in a row buffer of the
                // partner amplitude (3 J; 3 ldi, a zero amplitude, where the entry is zero)
                // | sign << 14 (this thread: quarter hf of the row's entries)
                cur_tile = atile;
                const int Ia = atile * kAbM + r;
                const bool valid = Ia < g.Da;
                const uint32_t a = valid ? g.stra[Ia] : 0u;
                const int part = tstride / (kAbBuild / kAbM);
                for (int k = hf * part; k < (hf + 1) * part; ++k) {
                    uint32_t e = zoff;
                    if (valid && k < Ktot) {
                        const int p = s_kp[k], q = s_kq[k];
                        if (p == q) {
                            if ((a >> p) & 1u) e = 3u * (uint32_t)Ia;
                        } else if (((a >> p) ^ (a >> q)) & 1u) {
                            const uint32_t ap = a ^ (1u << p) ^ (1u << q);
                            e = 3u * (uint32_t)g.ra[ap] | ((uint32_t)ab_par(a & ab_between(p, q)) << 14);
                        }
                    }
                    tbl[r * tstride + k] = (uint16_t)e;
                }
                builders_sync();  // the rows' entries are read by the other quarters' threads
            }
            // this unit's B rows (read one unit ahead from the per-partner-row table)
            #pragma unroll
            for (int k = 0; k < 1; ++k) {
                const int ii = bsel[k] < 0 ? 0 : bsel[k], piece = ii / (ncolsP * 2), rem = ii - piece * ncolsP * 2;
                bsrc[k] = g.Bp + (size_t)piece * g.pb + (size_t)brow[k] * 256 + (rem & 1) * 8;
                if (un < g.units) brow[k] = g.rowB[(size_t)(un % g.Db) * kAbMaxN + (rem >> 1)];
            }
            const uint32_t *xr = xrow + (size_t)buf * xstride;
            const uint16_t *trow = tbl + r * tstride + hf * kAbKpt;
            for (int c = 0; c < g.nK; ++c, ++gch) {
                const int s = gch % kAbS;
                // B rows of this K block into registers (ncolsP rows x 2 core columns x 3 pieces)
                uint4 bv[1];
                #pragma unroll
                for (int k = 0; k < 1; ++k)
                    if (bsel[k] >= 0) bv[k] = *reinterpret_cast<const uint4 *>(bsrc[k] + c * kAbKc);
                // this thread's 8 K entries of row r: three words each (pieces 1..3, re | im << 16),
                // sign bits flipped by the entry's sign
                uint32_t w[kAbKpt][3];
                {
                    const uint2 tv = *reinterpret_cast<const uint2 *>(trow + c * kAbKc);
                    const uint32_t te[2] = {tv.x, tv.y};
                    #pragma unroll
                    for (int k = 0; k < kAbKpt; ++k) {
                        const uint32_t e = (k & 1) ? te[k >> 1] >> 16 : te[k >> 1] & 0xFFFFu;
                        // checked build: an offset past the row buffer reads the zero amplitude
                        const uint32_t *x =
                            xr + (SV_IN_RANGE((e & 0x3FFFu) + 2u, (uint32_t)xstride, kChkGather) ? (e & 0x3FFFu) : zoff);
                        w[k][0] = x[0];
                        w[k][1] = x[1];
                        w[k][2] = x[2];
                    }
                    #pragma unroll
                    for (int k = 0; k < kAbKpt; ++k) {
                        const uint32_t e = (k & 1) ? te[k >> 1] >> 16 : te[k >> 1] & 0xFFFFu;
                        const uint32_t flip = (e >> 14) * 0x80008000u;
                        w[k][0] ^= flip;
                        w[k][1] ^= flip;
                        w[k][2] ^= flip;
                    }
                }
                // the stage is free once the MMAs of K block gch - kAbS are done; every builder
                // waits itself (a timeout sets s_fail, which ends the other waits at once; the
                // builders then stop together at the next unit)
                if (gch >= kAbS && !s_fail && !ab_wait(su32(&empty[s]), (uint32_t)(((gch / kAbS) - 1) & 1), g.spins))
                    s_fail = 1;
                uint8_t *st = ring + s * kStageBytes;
                // A: this thread's row (its tensor-memory lane) and 4 K = 2 columns of each piece
                __syncwarp();
                #pragma unroll
                for (int pl = 0; pl < P; ++pl) {
                    const uint32_t sel = pl ? 0x7632u : 0x5410u;  // the im or the re halves of two words
                    #pragma unroll
                    for (int pc = 0; pc < 3; ++pc) {
                        const uint32_t ta = tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                                            (uint32_t)(kAbABase + s * kAbAStage + (pl * 3 + pc) * kAbACols + hf * 2);
                        asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(ta),
                                     "r"(__byte_perm(w[0][pc], w[1][pc], sel)), "r"(__byte_perm(w[2][pc], w[3][pc], sel))
                                     : "memory");
                    }
                }
                #pragma unroll
                for (int k = 0; k < 1; ++k)
                    if (bsel[k] >= 0) *reinterpret_cast<uint4 *>(st + bdst[k]) = bv[k];
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B, for the MMAs' reads
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");   // A written
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                ab_arrive(su32(&full[s]));
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (tid >= kAbBuild + 32) {
        // ------------------------------------------------------------ epilogue warps
        // drain each unit's accumulator (row bp, tile row r = this thread's lane) into H
        // (two warps per lane quarter, taking alternate 16-column chunks)
        const int quarter = warp & 3, r = quarter * 32 + (tid & 31), eh = (warp - kAbBuild / 32 - 1) >> 2;
        int it = 0;
        for (int u = blockIdx.x; u < g.units; u += gridDim.x, ++it) {
            const int atile = u / g.Db, bp = u - atile * g.Db, t = it & 1, ia = atile * kAbM + r;
            bool bad = false;
            if (tid == kAbBuild + 32) {
                if (!ab_wait(su32(&accf[t]), (uint32_t)((it >> 1) & 1), g.spins)) s_fail = 1;
                bad = s_fail != 0;
            }
            if (epi_any(bad)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const bool ok_row = ia < g.Da;
            #pragma unroll
            for (int pl = 0; pl < P; ++pl) {
                const uint32_t tbase =
                    tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(t * kAbAccCols + pl * kAbMaxN);
                float *Hp = g.H + (size_t)pl * g.hplane + (size_t)bp * g.ncols * g.ldh + ia;
                for (int c = 16 * eh; c < g.ncols; c += 32) {
                    uint32_t v[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                          "=r"(v[15])
                        : "r"(tbase + (uint32_t)c)
                        : "memory");
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (ok_row) {
                        #pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c + j < g.ncols) Hp[(size_t)(c + j) * g.ldh] = __uint_as_float(v[j]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            ab_arrive(su32(&acce[t]));
        }
    } else if (tid == kAbBuild) {
        // ------------------------------------------------------------ MMA issuer
        // kind::f16, D float32, A and B bf16, both K-major, N = ncolsP, M = 128
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ncolsP >> 3) << 17) |
                               ((uint32_t)(kAbM >> 4) << 24);
        const uint64_t d0 = ab_desc(sbase);
        int gch = 0, it = 0;
        bool stop = false;
        for (int u = blockIdx.x; u < g.units && !stop; u += gridDim.x, ++it) {
            const int t = it & 1;
            if (it >= 2 && !ab_wait(su32(&acce[t]), (uint32_t)(((it >> 1) - 1) & 1), g.spins)) { s_fail = 1; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int c = 0; c < g.nK; ++c, ++gch) {
                const int s = gch % kAbS;
                if (!ab_wait(su32(&full[s]), (uint32_t)((gch / kAbS) & 1), g.spins) || s_fail) {
                    s_fail = 1;
                    stop = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dacc = tmem + (uint32_t)(t * kAbAccCols), first = c == 0 ? 1u : 0u;
                static_assert(kAbS == 4, "one case per stage");
                switch (s) {
                    case 0: ab_mma_stage<P, 0>(tmem, d0, dacc, idesc, first); break;
                    case 1: ab_mma_stage<P, 1>(tmem, d0, dacc, idesc, first); break;
                    case 2: ab_mma_stage<P, 2>(tmem, d0, dacc, idesc, first); break;
                    default: ab_mma_stage<P, 3>(tmem, d0, dacc, idesc, first); break;
                }
                ab_commit(su32(&empty[s]));
            }
            if (!stop) ab_commit(su32(&accf[t]));
        }
        ab_commit(su32(&done));  // every MMA issued above has completed when `done` does
    }
    __syncwarp();
    const bool ok = ab_wait(su32(&done), 0u, g.spins);
    if (!ok) s_fail = 1;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && s_fail) atomicExch(g.err, 1);
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

namespace {

// B table rows (K index kappa as in k_ab_tc: p = q = kappa below N, then the pairs
// p < q): t = s N + r (t < N^2): B[t][kappa] = (qp|sr) = eri[(q N + p) N^2 + t];
// N^2 + b': sum_{l in b'} (qp|ll) for p != q (Jt[(q N + p) N + l]), 0 for p = q;
// N^2 + Db: zeros.  Written as three bf16 pieces; rows of 256.
__global__ void __launch_bounds__(256) k_ab_table(const float *__restrict__ eri, const float *__restrict__ Jt,
                                                  const uint16_t *__restrict__ strb, int N, int Db,
                                                  uint16_t *__restrict__ Bp, size_t pb) {
    const int row = blockIdx.x, kap = threadIdx.x, NN = N * N, Ktot = N * (N + 1) / 2;
    float v = 0.f;
    if (kap < Ktot) {
        int p = 0, q = 0;
        if (kap < N) {
            p = q = kap;
        } else {
            int pi = kap - N;
            while (pi >= N - 1 - p) { pi -= N - 1 - p; ++p; }
            q = p + 1 + pi;
        }
        if (row < NN) {
            v = eri[(size_t)(q * N + p) * NN + row];
        } else if (row < NN + Db && p != q) {
            for (uint32_t o = strb[row - NN]; o; o &= o - 1u) v += Jt[(size_t)(q * N + p) * N + __ffs(o) - 1];
        }
    }
    uint32_t a1, a2, a3;
    split3(v, a1, a2, a3);
    const size_t at = (size_t)row * 256 + kap;
    Bp[at] = (uint16_t)a1;
    Bp[pb + at] = (uint16_t)a2;
    Bp[2 * pb + at] = (uint16_t)a3;
}

// The B-table row of each column of partner row b' (one block of kAbMaxN threads per
// b'): column j < nb (N - nb) is the j-th excitation s (occupied) -> r (empty) of b', s
// the (j / (N - nb))-th occupied and r the (j % (N - nb))-th empty orbital in increasing
// order, row s N + r; column nb (N - nb) is b''s own row N^2 + b'; the rest the zero row.
__global__ void __launch_bounds__(kAbMaxN) k_ab_rows(const uint16_t *__restrict__ strb, int N, int nb, int Db,
                                                     uint16_t *__restrict__ rowB) {
    const int bp = blockIdx.x, t = threadIdx.x, ne = N - nb, nbs = nb * ne;
    int row = N * N + Db;
    if (t < nbs) {
        uint32_t o = strb[bp], z = ~o & ((1u << N) - 1u);
        for (int k = 0; k < t / ne; ++k) o &= o - 1u;
        for (int k = 0; k < t % ne; ++k) z &= z - 1u;
        row = (__ffs(o) - 1) * N + (__ffs(z) - 1);
    } else if (t == nbs) {
        row = N * N + bp;
    }
    rowB[(size_t)bp * kAbMaxN + t] = (uint16_t)row;
}

size_t ab_tc_smem(int Da, int N) {
    const size_t stage = 3 * kAbMaxN * kAbKc * 2;
    const int nK = (N * (N + 1) / 2 + kAbKc - 1) / kAbKc;
    const size_t ldi = ((size_t)Da + 3) / 4 * 4;
    return 1024 + kAbS * stage + 2 * (ldi + 4) * 12 + (size_t)kAbM * ab_tstride(nK) * 2;
}

}  // namespace

// Rows of the B table (and its piece stride): N^2 + Db + 1 rows of 256.
size_t ab_table_rows(int N, int Db) { return (size_t)N * N + Db + 1; }

// Elements of the per-partner-row column table (uint16) that launch_ab_table writes.
size_t ab_rowb_elems(int Db) { return (size_t)Db * kAbMaxN; }

// The B table pieces and, where rowB is given, the column table [Db][64] of the sector
// with nb beta electrons (two launches).
cudaError_t launch_ab_table(const float *eri, const float *Jt, const uint16_t *strb, int N, int nb, int Db,
                            uint16_t *Bp, size_t pb, uint16_t *rowB, cudaStream_t st) {
    if (N * N > 256 || nb < 0 || nb > N) return cudaErrorInvalidValue;
    k_ab_table<<<(unsigned)ab_table_rows(N, Db), 256, 0, st>>>(eri, Jt, strb, N, Db, Bp, pb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !rowB) return e;
    if (nb * (N - nb) + 1 > kAbMaxN) return cudaSuccess;  // more columns than k_ab_tc takes: no column table
    k_ab_rows<<<Db, kAbMaxN, 0, st>>>(strb, N, nb, Db, rowB);
    return cudaGetLastError();
}

// Whether the tensor-core alpha-beta form applies: N <= 16, D <= 4096 per spin, at most
// 64 columns, and its shared memory fits.
bool ab_tc_fits(int planes, int Da, int Db, int na, int nb, int N) {
    (void)planes;
    (void)na;
    if (N > 16 || N < 1 || Da > 4096 || Db > 4096 || Da < 1 || Db < 1) return false;
    if (nb * (N - nb) + 1 > kAbMaxN) return false;
    return ab_tc_smem(Da, N) <= 227 * 1024 - 1024;
}

// Row stride (amplitudes) of the interleaved X pieces the kernel reads.
int ab_xi_ld(int Da) { return (Da + 3) / 4 * 4; }

// Row stride (floats) of the product planes H: whole 128-byte lines, so that each epilogue
// warp's store of 32 consecutive alpha strings fills one line (tile starts are multiples
// of 128 strings).
int ab_h_ld(int Da) { return (Da + 31) / 32 * 32; }

// H = the per-partner-row products (see above); Xi [Db][ab_xi_ld(Da)][3] the phased
// amplitudes as bf16 pieces (phase kernel); Bp the B table pieces; H planes
// [planes][Db][ncols][ab_h_ld(Da)] (hplane elements apart); rowB the column table of
// launch_ab_table.
// spins: polls of each bounded wait; stall: the test hook of AbTcArgs.
cudaError_t launch_ab_tc(const uint32_t *Xi, int planes, const uint16_t *stra, const uint16_t *strb,
                         const uint16_t *ra, const uint16_t *Bp, size_t pb, const uint16_t *rowB, float *H, size_t hplane, int Da, int Db,
                         int N, int na, int nb, int *err, uint32_t spins, int stall, int sm_count, cudaStream_t st) {
    if (!ab_tc_fits(planes, Da, Db, na, nb, N) || ((uintptr_t)Xi & 15) || ((uintptr_t)Bp & 15) || (pb & 7) ||
        !rowB || spins < 1)
        return cudaErrorInvalidValue;
    AbTcArgs g;
    g.Xi = Xi; g.ldi = ab_xi_ld(Da); g.stra = stra; g.strb = strb; g.ra = ra; g.Bp = Bp; g.pb = pb; g.rowB = rowB; g.H = H;
    g.hplane = hplane; g.ldh = ab_h_ld(Da); g.Da = Da; g.Db = Db; g.N = N; g.na = na; g.nb = nb;
    g.ncols = nb * (N - nb) + 1;
    g.nK = (N * (N + 1) / 2 + kAbKc - 1) / kAbKc;
    g.units = ((Da + kAbM - 1) / kAbM) * Db;
    g.maskN = (1u << N) - 1u;
    g.err = err;
    g.spins = spins;
    g.stall = stall;
    const int grid = g.units < sm_count ? g.units : sm_count;
    const size_t sm = ab_tc_smem(Da, N);
    cudaError_t e;
    if (planes == 2) {
        e = cudaFuncSetAttribute(k_ab_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_ab_tc<2><<<grid, kAbThreadsTc, sm, st>>>(g);
    } else {
        e = cudaFuncSetAttribute(k_ab_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_ab_tc<1><<<grid, kAbThreadsTc, sm, st>>>(g);
    }
    return cudaGetLastError();
}

// This unit's check word (checked build), for sv_check_status.
SV_CHECK_READER(check_word_abtc)

}  // namespace svk
