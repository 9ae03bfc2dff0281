// sv_internal.h -- host-side structures shared by the library's translation units.
// Not part of the public C-ABI (include/sv.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "sv.h"

struct sv_ham;

// Runs the statement(s) with `A` bound to the amplitude type of a state dtype.
#define SV_DISPATCH_AMP(dtype, ...)                      \
    switch (dtype) {                                     \
        case SV_C64: { using A = float2; __VA_ARGS__; } break;  \
        case SV_C128: { using A = double2; __VA_ARGS__; } break; \
        case SV_R32: { using A = float; __VA_ARGS__; } break;    \
        default: { using A = double; __VA_ARGS__; } break;       \
    }

namespace svk {

// Bytes of one amplitude, and whether the state's arithmetic is single precision.
inline size_t amp_size(int dtype) { return dtype == SV_C64 ? 8 : dtype == SV_C128 ? 16 : dtype == SV_R32 ? 4 : 8; }
inline bool single_prec(int dtype) { return dtype == SV_C64 || dtype == SV_R32; }
inline bool is_complex(int dtype) { return dtype == SV_C64 || dtype == SV_C128; }

// ---------------------------------------------------------------- excitation ops

// One excitation prepared for the rotation kernels.  The pair (x, x ^ m) is
// rotated for every basis index x whose bits on the mask equal `from` (the
// determinant that T maps to x ^ m).  The Jordan-Wigner sign of T on x is
// (-1)^popc(x & sm): for a single i->a, sm = bits strictly between i and a; for a
// double with sorted mask positions q0<q1<q2<q3, sm = bits strictly between q0 and
// q1 plus bits strictly between q2 and q3, whichever two of the four are occupied.
struct OpDesc {
    uint32_t m = 0;     // flip mask
    uint32_t from = 0;  // bits of the "from" determinant on the mask
    uint32_t sm = 0;    // sign mask
    int nbits = 0;      // 2 (single) or 4 (double)
    int pos[4] = {0, 0, 0, 0};  // mask positions, ascending
    double c = 1.0, s = 0.0;    // cos(theta), sin(theta), taken on the host in float64
};

// Storage layout: bit perm[q] of an amplitude's address holds qubit q.
// map_bits applies it to a qubit-space bit mask.
inline uint32_t map_bits(uint32_t m, const int *perm) {
    uint32_t r = 0;
    while (m) {
        int q = __builtin_ctz(m);
        r |= 1u << perm[q];
        m &= m - 1u;
    }
    return r;
}

// Validate one excitation for an n-qubit register and fill `d` (without angles),
// with masks and positions in the storage layout `perm`.
bool make_op(const sv_excitation &e, int n, const int *perm, OpDesc &d, std::string &why);

// Bits strictly between positions a and b (order irrelevant).
inline uint32_t bits_between(int a, int b) {
    if (a > b) { int t = a; a = b; b = t; }
    if (b - a <= 1) return 0u;
    uint64_t hi = (1ull << b) - 1ull;        // bits < b
    uint64_t lo = (1ull << (a + 1)) - 1ull;  // bits <= a
    return (uint32_t)(hi & ~lo);
}

// ---------------------------------------------------------------- Hamiltonian tables

// Double-excitation group: every Pauli string whose X-part is the 4-bit mask m.
// At a basis index x with exactly two of the four mask bits set, the sum of those
// strings equals <x^m|H|x> = (-1)^popc(x & sm) * v[split], where split says which
// mask bit pairs with the lowest one among the occupied (or, equivalently, the
// empty) pair: 0 -> q1, 1 -> q2, 2 -> q3, and v = [ai|bj] - [aj|bi] for occupied
// i<j and empty a<b.  Other x are not connected by this mask.
template <typename R>
struct DoubleRec {
    uint32_t m, sm;
    uint32_t b0, b1, b2;  // bit(q0), bit(q1), bit(q2)
    uint32_t pad;
    R v[3];
};

// Single-excitation group (mask {i, a}, same spin): at x with exactly one of the
// two bits set, <x^m|H|x> = (-1)^popc(x & sm) * (h_ai + sum_k x_k W[k]),
// W[k] = [ai|kk] - [ak|ki] (zero for k in {i, a}).
template <typename R>
struct SingleRec {
    uint32_t m, sm;
    R h;
    R pad;
};

// Host copy of the tables for one (n, precision).
template <typename R>
struct HostTables {
    std::vector<DoubleRec<R>> dbl;
    std::vector<SingleRec<R>> sgl;
    std::vector<R> W;          // [n_singles][n]
    std::vector<double> hdiag; // [n] h_kk per spin-orbital (qubit order)
    std::vector<double> Jp;    // [n][n] [kk|ll] - [kl|lk] (0 on the diagonal), qubit order
    std::vector<double> hdiag_s, Jp_s;  // the same indexed by storage bit (record scan)
};

// Device copy of the tables, built lazily per (n, dtype) and cached in the Hamiltonian.
// Same-spin part of sigma as dense products in the string-blocked basis (expectation
// variant 4, single-precision states): with the determinant written as the alpha
// creators followed by the beta creators, an alpha excitation's sign depends on the
// alpha string alone and a beta excitation's on the beta string alone, so
//   sigma~_same[b][a] = sum_a' Ma[a][a'] C~[b][a'] + sum_b' Mb[b][b'] C~[b'][a]
// with C~[b][a] = phi(a, b) C[b][a], phi = (-1)^popc(a & pp(b)) the reordering sign
// between the interleaved and the blocked creator orders (pp = prefix parity).
struct SameGemm {
    const float *Ma = nullptr, *Mb = nullptr;  // [Da][Da], [Db][Db], symmetric
    const double *dA = nullptr, *dB = nullptr; // one-spin diagonal energies per string (float64)
    float *G = nullptr;                        // same-spin sigma~ [planes][Db][Da]
    // every operand as three bf16 pieces at a piece stride: [Ma | Mb] (Mp, pm), the
    // phased planes [planes][Db][lda] (Xp, px), their transposes [planes][Da][ldb] (Xtp, pt)
    const uint16_t *Mp = nullptr;
    uint16_t *Xp = nullptr, *Xtp = nullptr;
    size_t pm = 0, px = 0, pt = 0;
    int planes = 2;                            // 2 complex (re, im), 1 real
    int lda = 0, ldb = 0;                      // row strides of Ma / X and Mb / Xt: D rounded up to 4, zero padded
    int *err = nullptr;                        // device flag set by k_same_tc / k_ab_tc when a wait runs out
    uint32_t spins = 1u << 22;                 // polls of each of their bounded waits
    cudaEvent_t *ev = nullptr;                 // profiling (may be NULL): events around the same-spin
                                               // products [0], [1] and the alpha-beta products [2], [3]
    int stall = 0;                             // test hook: bit 0 k_same_tc, bit 1 k_ab_tc issue nothing
    // variant 5: the alpha-beta part on the tensor cores (k_ab_tc) into planes H
    // [planes][Db][ncols][ldh] (hplane floats apart), gathered by k_sigma_comb; Bp: the
    // bf16 pieces [3][N^2 + Db + 1][256] of its integral table (piece stride pb)
    int abtc = 0;
    uint32_t *Xi = nullptr;                    // phased amplitudes as interleaved bf16 pieces [Db][ldi][3]
    int ldi = 0;
    const uint16_t *Bp = nullptr;
    size_t pb = 0;
    const uint16_t *rowB = nullptr;            // [Db][64] B-table row of each column of a partner row
    float *H = nullptr;
    size_t hplane = 0;
    int ldh = 0;                               // row stride of H (floats, a multiple of 32)
    int ncols = 0, na = 0, nb = 0;
};

struct DevTables {
    uint64_t serial = 0;   // unique per table set (keys the per-handle same-spin matrices)
    int n = 0;
    int dtype = 0;
    int n_dbl = 0, n_sgl = 0;
    void *dbl = nullptr;   // DoubleRec<R>[n_dbl]
    void *sgl = nullptr;   // SingleRec<R>[n_sgl]
    void *W = nullptr;     // R[n_sgl * n]
    double *hdiag = nullptr;    // qubit order (string rows)
    double *Jp = nullptr;
    double *hdiag_s = nullptr;  // storage order (record scan)
    double *Jp_s = nullptr;
    // string-row tables (k_rows.cu), state precision
    void *eri_r = nullptr;  // [N^4] (pq|rs)
    void *hm_r = nullptr;   // [N^2] h_pq
    void *Dt = nullptr;     // [N^3] (qp|kk) - (qk|kp)
    void *Jt = nullptr;     // [N^3] (qp|kk)
    void *W2 = nullptr;     // [NP][NP] same-spin doubles by (q1<q2, p1<p2) pairs
    // the same five tables as float-float pairs (float64 tables only; expectation variant 6)
    void *eri_ff = nullptr, *hm_ff = nullptr, *Dt_ff = nullptr, *Jt_ff = nullptr, *W2_ff = nullptr;
    // tiled-pass schedule (k_expect.cu); empty until first needed
    struct Pass {
        uint32_t S;        // local qubit set (bit mask over storage positions)
        int first_dbl, n_dbl, first_sgl, n_sgl;
        int owns_diag;
    };
    std::vector<Pass> passes;
    void *pass_dbl = nullptr;  // doubles regrouped by pass, local-index form
    void *pass_sgl = nullptr;
    void *pass_W = nullptr;
    int tile_bits = 0;
    ~DevTables();
};

template <typename R>
void build_tables(const sv_ham &H, int n, HostTables<R> &out);

// Re-express the record-scan tables in the storage layout `perm` (masks mapped bit
// by bit; per-spin-orbital arrays moved to their storage positions).
template <typename R>
void permute_tables(HostTables<R> &t, const int *perm, int n);

// <x|H|x> in float64 on the host.
double diag_energy(const sv_ham &H, uint32_t x, int n);

}  // namespace svk

// ---------------------------------------------------------------- handles

struct sv_ham {
    int n_orb = 0;
    double e_nuc = 0.0;
    std::vector<double> h;    // [N][N]
    std::vector<double> eri;  // [N][N][N][N] chemist (pq|rs)
    std::map<std::string, std::unique_ptr<svk::DevTables>> dev;  // key: device, n, dtype, layout
    int device = -1;
};

// Per-operator pair lists kept on the device: the lists, then the op records, then
// per op (alpha offset, alpha length, beta offset, beta length) as int4.
struct OpLists {
    void *buf = nullptr;
    size_t bytes = 0;
    std::vector<uint32_t> key;  // sector counts and every op's masks the lists were built for
    std::vector<int> info;      // the per-op int4 records, host copy
    const int *dinfo = nullptr; // their device copy (inside buf)
};

struct sv_ctx {
    int n = 0;
    sv_dtype dtype = SV_C64;
    cudaStream_t stream = nullptr;
    int device = 0;
    uint64_t dim = 0;          // 2^n
    size_t amp_bytes = 8;      // bytes per amplitude
    int storage = 0;           // 0 dense 2^n vector, 1 sector (compact string-row matrix)
    uint64_t elems = 0;        // amplitudes stored per vector
    void *psi = nullptr;
    void *lam = nullptr;
    bool own_psi = true, own_lam = true;
    // prepared state
    bool prepared = false;
    bool at_ref = false;       // psi holds the HF reference exactly as sv_prepare_hf wrote it
    bool nvtx_open = false;    // a phase range of this handle is open (NVTX)
    bool failed = false;
    int na = -1, nb = -1;
    int ref_kind = 0;          // 0 none, 1 HF determinant, 2 stored vector
    uint32_t ref_det = 0;      // HF determinant (ref_kind 1)
    void *ref_vec = nullptr;   // device copy of the reference (ref_kind 2)
    double ref_shift = 0.0;    // c in lambda = (H - c) psi
    // sector list (basis indices of the (na, nb) sector, ascending) for gather kernels
    uint32_t *sector = nullptr;
    uint64_t sector_len = 0;
    int sector_na = -1, sector_nb = -1;
    // string-row view of the sector (k_rows.cu): alpha / beta strings, ranks, spreads
    uint32_t *str_sa = nullptr, *str_sb = nullptr;    // qubit-space spreads
    uint32_t *str_sa_s = nullptr, *str_sb_s = nullptr;  // storage-space spreads
    uint16_t *str_a = nullptr, *str_b = nullptr, *rank_a = nullptr, *rank_b = nullptr;
    int Da = 0, Db = 0, str_na = -1, str_nb = -1;
    std::vector<uint16_t> h_stra, h_strb, h_ra, h_rb;  // host copies (sector storage indexing)
    size_t str_bytes = 0;
    void *Cbuf = nullptr;      // compact amplitudes [Db][Da]
    size_t Cbuf_bytes = 0;
    void *Lbuf = nullptr;      // compact sigma [Db][Da] (operator screening)
    size_t Lbuf_bytes = 0;
    // per-op alpha / beta pair lists (k_build_lists): the ansatz's (sector storage
    // rotations and adjoint steps) and the screened pool's
    OpLists lists, pool_lists;
    OpLists rdm_lists;         // the 1-RDM's alpha-pair lists (one per orbital pair p < q)
    void *CLbuf = nullptr;     // compact amplitudes and sigma interleaved [Db][Da][2] (screening)
    size_t CLbuf_bytes = 0;
    // reduction scratch
    double *partials = nullptr;
    size_t partials_cap = 0;   // doubles
    double *dout = nullptr;    // small device output buffer
    size_t dout_cap = 0;
    double *hpinned = nullptr; // pinned host staging
    size_t hpinned_cap = 0;
    // checkpoints / saved final state
    std::vector<void *> ckpt;
    void *saved = nullptr;
    int64_t ckpt_interval = 0;
    int64_t max_bytes = 0;
    uint64_t bytes_owned = 0;
    int expect_variant = 0;
    int64_t ab_chunk = 0;      // SV_OPT_AB_CHUNK: partner rows per chunk of k_sigma_ab (0 auto)
    // launch geometry (blocks per SM), set by sv_autotune or the options
    int rot_bps = 32;          // dense k_rotate / k_adjoint / k_adjoint_i
    int sect_bps = 8;          // sector k_rotate_l / k_adjoint_l
    int rdm_bps = 4;           // k_rdm_rows
    int rdm_variant = 0;
    int pool_variant = 0;      // 0 auto (= 2); 1 string scan; 2 pair lists
    int l2_fetch = 32;         // context L2 fetch granularity during dense sweeps (0: leave it)
    int rev_inter = 1;         // dense reverse sweep on psi and lambda interleaved (k_adjoint_i) where it can
    bool lam_pair = false;     // lam's allocation holds two vectors: lam, then the working copy `saved`
    int *kerr = nullptr;       // device flag of kernels with bounded waits (k_same_tc, k_ab_tc)
    int64_t wait_polls = 1 << 22;  // polls of each of their bounded waits (SV_OPT_WAIT_POLLS)
    int test_stall = 0;        // SV_OPT_TEST_STALL: bit 0 k_same_tc, bit 1 k_ab_tc issue no copy / MMA
    // sector storage, whole-sweep launches (k_sweep_rotate_l / k_sweep_adjoint_li): a barrier
    // counter (first 256 bytes) and the ops' (cos, sin) on the device, their host staging
    void *sweep_buf = nullptr;
    size_t sweep_bytes = 0;
    std::vector<double> sweep_host;
    int sweep_mode = 1;        // SV_OPT_SECTOR_SWEEP: 1 one launch per sweep where possible, 0 one per op
    int sweep_bps = 2;         // SV_OPT_SWEEP_BLOCKS_PER_SM: blocks per SM of a whole-sweep launch
    // expectation variant 6: the compact amplitudes and sigma as float-float matrices
    void *ffbuf = nullptr;
    size_t ffbuf_bytes = 0;
    int *hkerr = nullptr;      // its pinned host copy, checked after stream synchronisations
    // same-spin products (expectation variant 4): matrices for one table set and sector,
    // and the phased-psi / product planes
    void *sg_mats = nullptr;
    size_t sg_mats_bytes = 0;
    uint64_t sg_serial = 0;
    int sg_na = -1, sg_nb = -1;
    void *sg_buf = nullptr;
    size_t sg_buf_bytes = 0;
    uint64_t sg_buf_geom = 0;  // the planes' geometry (their row padding is zeroed when it changes)
    float *ab_H = nullptr;     // variant 5: the alpha-beta product planes
    size_t ab_H_bytes = 0;
    // storage layout: address bit perm[q] holds qubit q (identity by default);
    // layout_auto: sv_energy_grad picks it from its operator list
    int perm[32];
    bool layout_auto = true;
    // phase profiling (SV_OPT_PROFILE)
    bool profile = false;
    cudaEvent_t ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double phase_ms[SV_PHASES] = {0, 0, 0, 0, 0, 0, 0, 0};
    cudaEvent_t tcev[4] = {nullptr, nullptr, nullptr, nullptr};  // around the tensor-core products
    int tc_timed = 0;          // bit 0: same-spin products timed in this call, bit 1: alpha-beta
    // bookkeeping
    uint64_t launches = 0;
    std::string err;
    int sm_count = 148;
    int l2_bytes = 0;          // the device's L2 size
};
