// k_tcgemm.cu -- the same-spin products of the string-blocked expectation (variant 4)
// on the tensor cores: tcgen05.mma kind::f16 on bf16 operands with every float32 value
// split into three bf16 pieces (x = x1 + x2 + x3, each the rest of the previous
// rounded to bf16), six products x1 y1 + x1 y2 + x2 y1 + x1 y3 + x2 y2 + x3 y1 (the
// dropped terms are below 2^-24 of a product) accumulated in float32 in tensor memory:
// float32-level accuracy at the bf16 tensor rate.
//
// For plane p (re / im) one output tile, 128 alpha strings a (M) x kTcN beta strings b
// (N), accumulates both products in the same tensor-memory tile:
//   G[p][b][a] = sum_a' Ma[a][a'] X[p][b][a']          (K = D_alpha)
//              + sum_b' Xt[p][a][b'] Mb[b][b']          (K = D_beta)
// (Ma, Mb symmetric; Xt the transposed planes, so both operands of both products are
// K-contiguous).  Operand tiles (rows x 32 bf16 of K, 64-byte rows) are moved by TMA
// (cp.async.bulk.tensor, 64-byte swizzle; rows and K beyond the matrix read as zero)
// into a ring of kTcStages stages.  Warp roles: lane 0 of warp 0 issues the copies,
// lane 0 of warp 1 the MMAs; a full barrier per stage counts the copied bytes, an
// empty barrier per stage is signalled by tcgen05.commit once the MMAs that read it
// are done, and a last commit releases the four warps to the epilogue (tensor memory
// -> registers -> G).  Every wait is bounded: past the limit the kernel sets *err,
// waits (bounded) for its copies and MMAs in flight, frees its tensor memory and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include "sv_internal.h"

namespace svk {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;                              // alpha strings per tile (tensor-memory lanes)
constexpr int kTcN = 256;                              // beta strings per tile (tensor-memory columns)
constexpr int kTcKb = 32;                              // K (bf16 elements, 64 bytes) per stage
constexpr int kTcABytes = kTcM * kTcKb * 2;            // one piece of A in one stage
constexpr int kTcBBytes = kTcN * kTcKb * 2;            // one piece of B in one stage
constexpr int kTcStageBytes = 3 * kTcABytes + 3 * kTcBBytes;
constexpr int kTcStages = 3;                           // 3 x 72 KB
constexpr int kTcSmem = kTcStages * kTcStageBytes + 1024;  // + alignment of the ring to 1024 bytes

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand tile with 64-byte swizzle: start
// address, stride byte offset 512 (8 rows of 64 bytes), descriptor version 1, swizzle
// mode 4 (64-byte).  The leading byte offset is unused for swizzled K-major tiles.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t spins) {
    for (uint32_t it = 0; it < spins; ++it) {
        if (mbar_try(mbar, parity)) return true;
        __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap *map, int k, int row, int c3, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(k), "r"(row), "r"(c3), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tma_4d(uint32_t dst, const CUtensorMap *map, int k, int row, int p, int c,
                                       uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"((uint64_t)map), "r"(k), "r"(row), "r"(p), "r"(c), "r"(mbar)
        : "memory");
}

struct TcOut {
    float *G;  // [P][Db][Da]
    int Da, Db;
    int *err;
    uint32_t spins;  // mbarrier polls (each with a short sleep) before a wait gives up
    int stall;       // test hook: the producer issues no copy, so the MMA issuer's first wait runs out
};

// Tensor maps (innermost first): ma {K = Da, rows Da, piece}, mb {K = Db, rows Db, piece},
// x {K = Da, rows Db, plane, piece}, xt {K = Db, rows Da, plane, piece}; box {32, rows of a
// tile, 1, 1}.
__global__ void __launch_bounds__(kTcThreads, 1)
    k_same_tc(const __grid_constant__ CUtensorMap ma, const __grid_constant__ CUtensorMap mb,
              const __grid_constant__ CUtensorMap x, const __grid_constant__ CUtensorMap xt, TcOut g) {
    extern __shared__ uint8_t tc_smem[];
    __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages], done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int s_fail;
    __shared__ int s_issued, s_consumed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.x * kTcN, m0 = blockIdx.y * kTcM, p = blockIdx.z;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "n"(kTcN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
        for (int s = 0; s < kTcStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base, sbase = (smem_u32(tc_smem) + 1023u) & ~1023u;
    const int nA = (g.Da + kTcKb - 1) / kTcKb, nB = (g.Db + kTcKb - 1) / kTcKb, nIt = nA + nB;
    if (tid == 0) {
        // producer: K block it into stage it % kTcStages once the MMAs of block it - kTcStages are done
        int it = 0;
        for (; it < (g.stall ? 0 : nIt); ++it) {
            const int s = it % kTcStages;
            if (it >= kTcStages && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((it / kTcStages - 1) & 1), g.spins)) {
                s_fail = 1;
                break;
            }
            if (s_fail) break;
            const uint32_t st = sbase + (uint32_t)(s * kTcStageBytes), fb = smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "n"(kTcStageBytes)
                         : "memory");
            #pragma unroll
            for (int c = 0; c < 3; ++c) {
                if (it < nA) {  // alpha side: A = Ma rows a, B = X[p] rows b, K = a'
                    tma_3d(st + c * kTcABytes, &ma, it * kTcKb, m0, c, fb);
                    tma_4d(st + 3 * kTcABytes + c * kTcBBytes, &x, it * kTcKb, n0, p, c, fb);
                } else {        // beta side: A = Xt[p] rows a, B = Mb rows b, K = b'
                    tma_4d(st + c * kTcABytes, &xt, (it - nA) * kTcKb, m0, p, c, fb);
                    tma_3d(st + 3 * kTcABytes + c * kTcBBytes, &mb, (it - nA) * kTcKb, n0, c, fb);
                }
            }
        }
        s_issued = it;
    } else if (tid == 32) {
        // MMA issuer: kind::f16, D float32, A and B bf16, both K-major, N = kTcN, M = kTcM
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                               ((uint32_t)(kTcM >> 4) << 24);
        int it = 0;
        for (; it < nIt; ++it) {
            const int s = it % kTcStages;
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((it / kTcStages) & 1), g.spins)) {
                s_fail = 1;
                break;
            }
            if (s_fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = sbase + (uint32_t)(s * kTcStageBytes);
            // (A piece, B piece) of the six products: x1 y1, x1 y2, x2 y1, x1 y3, x2 y2, x3 y1
            const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
            #pragma unroll
            for (int t = 0; t < 6; ++t) {
                const uint32_t a = base + pa[t] * kTcABytes, b = base + 3 * kTcABytes + pb[t] * kTcBBytes;
                #pragma unroll
                for (int ks = 0; ks < kTcKb / 16; ++ks) {  // K = 16 per instruction: 32 bytes into the 64-byte rows
                    const uint32_t acc = (it > 0 || t > 0 || ks > 0) ? 1u : 0u;
                    const uint64_t da = tc_desc(a + ks * 32), db = tc_desc(b + ks * 32);
                    asm volatile(
                        "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}\n" ::"r"(tmem),
                        "l"(da), "l"(db), "r"(idesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        s_consumed = it;
        // the last commit: every MMA issued above is done when `done` completes
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(&done))
                     : "memory");
    }
    __syncwarp();
    bool ok = mbar_wait(smem_u32(&done), 0u, g.spins);
    if (!ok) s_fail = 1;
    __syncthreads();
    if (s_fail && tid == 0) {
        // copies issued but not consumed by the MMAs: let them land before the CTA exits
        for (int it = s_consumed; it < s_issued; ++it)
            mbar_wait(smem_u32(&full[it % kTcStages]), (uint32_t)((it / kTcStages) & 1), g.spins);
    }
    __syncthreads();
    ok = !s_fail;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int m = m0 + warp * 32 + lane;  // this thread's tensor-memory lane: alpha string a
        #pragma unroll 1
        for (int c = 0; c < kTcN; c += 8) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "r"(taddr)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < g.Da) {
                #pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int n = n0 + c + j;
                    if (n < g.Db) g.G[((size_t)p * g.Db + n) * g.Da + m] = __uint_as_float(v[j]);
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(g.err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTcN) : "memory");
}

// Three bf16 pieces of n floats (x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2)),
// at piece stride `piece`.
__device__ __forceinline__ void split3(float v, uint16_t &p1, uint16_t &p2, uint16_t &p3) {
    const __nv_bfloat16 a = __float2bfloat16_rn(v);
    const float r = v - __bfloat162float(a);
    const __nv_bfloat16 b = __float2bfloat16_rn(r);
    const __nv_bfloat16 c = __float2bfloat16_rn(r - __bfloat162float(b));
    p1 = __bfloat16_as_ushort(a);
    p2 = __bfloat16_as_ushort(b);
    p3 = __bfloat16_as_ushort(c);
}

__global__ void __launch_bounds__(256) k_split_bf16x3(const float *__restrict__ x, uint16_t *__restrict__ out,
                                                      size_t n, size_t piece) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        split3(x[i], out[i], out[piece + i], out[2 * piece + i]);
}

// Xt[c][p][a][b] = X[c][p][b][a] over 32 x 32 tiles for the three pieces c (z = 3 p + c;
// the padding columns of Xt stay zero: the buffer is zeroed when allocated).
__global__ void __launch_bounds__(256) k_transpose_pieces(const uint16_t *__restrict__ X, uint16_t *__restrict__ Xt,
                                                          int Da, int Db, int lda, int ldb, size_t px, size_t pt) {
    __shared__ uint16_t t[32][34];
    const int p = blockIdx.z / 3, c = blockIdx.z - 3 * p, a0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    const uint16_t *Xp = X + c * px + (size_t)p * Db * lda;
    uint16_t *Xtp = Xt + c * pt + (size_t)p * Da * ldb;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int b = b0 + i, a = a0 + threadIdx.x;
        t[i][threadIdx.x] = (b < Db && a < Da) ? Xp[(size_t)b * lda + a] : (uint16_t)0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int a = a0 + i, b = b0 + threadIdx.x;
        if (a < Da && b < Db) Xtp[(size_t)a * ldb + b] = t[threadIdx.x][i];
    }
}

// cuTensorMapEncodeTiled from the driver (through the runtime's entry-point query, so
// the library links no driver library).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    return fn;
}

// A bf16 tensor map of `rank` dims (innermost first) with byte strides of dims 1.., box
// {kTcKb, rows, 1, 1}, 64-byte swizzle, zero fill.
bool encode_map(CUtensorMap *m, const void *base, int rank, const uint64_t *dims, const uint64_t *strides,
                uint32_t rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t box[4] = {(cuuint32_t)kTcKb, rows, 1, 1}, es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void *>(base),
              (const cuuint64_t *)dims, (const cuuint64_t *)strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// G = the two same-spin products of the planes (see above); err: a device int, set
// to 1 when a wait ran out.  M: the bf16 pieces of [Ma | Mb] (piece stride pm; Mb at
// Da lda), X: the pieces of the phased planes (stride px), Xt: room for the transposed
// pieces (stride pt), written here.  Rows padded to lda / ldb (multiples of 8); the
// pointers 16-byte aligned and the piece strides multiples of 8 elements (TMA's rules).
// spins: polls of each bounded wait; stall: the test hook of TcOut.
cudaError_t launch_same_tc(const uint16_t *M, size_t pm, const uint16_t *X, size_t px, uint16_t *Xt, size_t pt,
                           float *G, int planes, int Da, int Db, int lda, int ldb, int *err, uint32_t spins, int stall,
                           cudaStream_t st) {
    if (Da < 1 || Db < 1 || lda % 8 || ldb % 8 || pm % 8 || px % 8 || pt % 8 || spins < 1 || ((uintptr_t)M & 15) ||
        ((uintptr_t)X & 15) || ((uintptr_t)Xt & 15))
        return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_same_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_transpose_pieces<<<dim3((Da + 31) / 32, (Db + 31) / 32, 3 * planes), dim3(32, 8), 0, st>>>(X, Xt, Da, Db, lda,
                                                                                                 ldb, px, pt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    CUtensorMap ma, mb, mx, mt;
    const uint64_t P = (uint64_t)planes;
    const uint64_t dma[3] = {(uint64_t)Da, (uint64_t)Da, 3}, sma[2] = {(uint64_t)lda * 2, (uint64_t)pm * 2};
    const uint64_t dmb[3] = {(uint64_t)Db, (uint64_t)Db, 3}, smb[2] = {(uint64_t)ldb * 2, (uint64_t)pm * 2};
    const uint64_t dx[4] = {(uint64_t)Da, (uint64_t)Db, P, 3},
                   sx[3] = {(uint64_t)lda * 2, (uint64_t)Db * lda * 2, (uint64_t)px * 2};
    const uint64_t dt[4] = {(uint64_t)Db, (uint64_t)Da, P, 3},
                   stt[3] = {(uint64_t)ldb * 2, (uint64_t)Da * ldb * 2, (uint64_t)pt * 2};
    if (!encode_map(&ma, M, 3, dma, sma, kTcM) || !encode_map(&mb, M + (size_t)Da * lda, 3, dmb, smb, kTcN) ||
        !encode_map(&mx, X, 4, dx, sx, kTcN) || !encode_map(&mt, Xt, 4, dt, stt, kTcM))
        return cudaErrorInvalidValue;
    const TcOut g{G, Da, Db, err, spins, stall};
    k_same_tc<<<dim3((Db + kTcN - 1) / kTcN, (Da + kTcM - 1) / kTcM, planes), kTcThreads, kTcSmem, st>>>(ma, mb, mx,
                                                                                                       mt, g);
    return cudaGetLastError();
}

// The three bf16 pieces of n floats (piece stride `piece` elements).
cudaError_t launch_split_bf16x3(const float *x, uint16_t *out, size_t n, size_t piece, int sm_count, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    size_t grid = (n + 255) / 256;
    if (grid > (size_t)sm_count * 8) grid = (size_t)sm_count * 8;
    k_split_bf16x3<<<(unsigned)grid, 256, 0, st>>>(x, out, n, piece);
    return cudaGetLastError();
}

}  // namespace svk
