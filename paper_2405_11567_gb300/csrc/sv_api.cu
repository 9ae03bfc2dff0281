// sv_api.cu -- the C-ABI entry points declared in include/sv.h.
//
// Host orchestration only: argument validation (every check runs before any
// device work, so SV_ERR_ARG leaves the device untouched), buffer management,
// and the order of kernel launches on the handle's stream.  Every step of the
// path itself runs in the kernels of k_state.cu (rotations, adjoint sweep),
// k_rows.cu and k_expect.cu (expectation), k_rdm.cu, k_pool.cu and k_sector.cu
// (sector storage).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sv_internal.h"

#include <nvtx3/nvToolsExt.h>

namespace svk {
int rotate_grid(uint64_t npairs, int sm_count, int bps);
cudaError_t launch_set_basis(void *psi, int dtype, uint32_t x, cudaStream_t st);
cudaError_t launch_rotate(void *psi, int dtype, int n, const OpDesc &d, int sm_count, int bps, cudaStream_t st);
cudaError_t launch_adjoint(void *psi, void *lam, int dtype, int n, const OpDesc &d, int grid,
                           double *partial, cudaStream_t st);
cudaError_t launch_reduce_rows(const double *partials, int rows, int cols, double *out, cudaStream_t st);
cudaError_t launch_adjoint_i(void *cl, int dtype, int n, const OpDesc &d, int grid, double *partial, cudaStream_t st);
cudaError_t launch_interleave_zero(const void *psi, void *cl, int dtype, int n, int sm_count, cudaStream_t st);
cudaError_t launch_scatter_odd(const void *lamc, void *cl, int dtype, const uint32_t *sa_s, const uint32_t *sb_s,
                               int Da, int Db, int sm_count, cudaStream_t st);
int expect_gather_grid(uint64_t count, int sm_count);
cudaError_t launch_expect_gather(const void *psi, void *sigma, int dtype, int n, const uint32_t *sector,
                                 uint64_t count, const DevTables &T, double e_shift, int grid,
                                 double *partial, cudaStream_t st);
int rdm_gather_grid(uint64_t count, int sm_count);
int rdm_elements_bytes(int n, const int *perm, std::vector<uint8_t> &out);
cudaError_t launch_permute(const void *in, void *out, int dtype, int n, const int *sg, int sm_count, cudaStream_t st);
cudaError_t launch_gather(const void *psi, int dtype, const uint32_t *addr, int count, void *out, cudaStream_t st);
void pool_op_from(const OpDesc &d, int N, void *dst);
size_t pool_op_bytes();
cudaError_t launch_pool_grad(const void *C, const void *L, int dtype, const void *ops, int n_ops, const uint32_t *sa,
                             const uint32_t *sb, const uint16_t *stra, const uint16_t *strb, const uint16_t *ra,
                             const uint16_t *rb, int Da, int Db, double *out, cudaStream_t st);
cudaError_t launch_interleave(const void *C, const void *L, int dtype, void *CL, size_t count, int sm_count,
                              cudaStream_t st);
cudaError_t launch_pool_grad_l(const void *CL, int dtype, const uint32_t *lists, const int *info, int n_ops, int Da,
                               int Db, double *out, cudaStream_t st);
cudaError_t launch_rdm_gather(const void *psi, int dtype, const uint32_t *sector, uint64_t count,
                              const void *elems, int n_el, int grid, double *partial, cudaStream_t st);
// sector storage (k_sector.cu)
int sector_grid(int Db, int sm_count, int bps);
size_t list_op_bytes();
void list_op_from(const OpDesc &d, int N, int na, int nb, uint32_t a_off, void *dst, int *na_l, int *nb_l);
cudaError_t launch_build_lists(const void *ops, int n_ops, const uint32_t *sa, const uint32_t *sb,
                               const uint16_t *stra, const uint16_t *strb, const uint16_t *ra, const uint16_t *rb,
                               int Da, int Db, uint32_t *out, cudaStream_t st);
cudaError_t launch_rotate_l(void *psi, int dtype, const uint32_t *al, int na_l, const uint32_t *bl, int nb_l, int Da,
                            double c, double s, int grid, cudaStream_t st);
int sweep_grid(int dtype, bool adjoint, int Db, int sm_count, int bps);
cudaError_t launch_sweep_l(void *buf, int dtype, bool adjoint, const uint32_t *lists, const int *info,
                           const double *cs, int n_ops, int Da, int Db, int grid, unsigned int *bar, int *err,
                           uint32_t spins, double *partial, cudaStream_t st);
cudaError_t launch_adjoint_li(void *CL, int dtype, const uint32_t *al, int na_l, const uint32_t *bl, int nb_l, int Da,
                              double c, double s, int grid, double *partial, cudaStream_t st);
cudaError_t launch_adjoint_l(void *psi, void *lam, int dtype, const uint32_t *al, int na_l, const uint32_t *bl,
                             int nb_l, int Da, double c, double s, int grid, double *partial, cudaStream_t st);
int rdm_rows_elements(int n);
int rdm_rows_grid(int Db, int sm_count, int bps);
cudaError_t launch_to_ff(const void *C, int dtype, size_t count, void *out, int sm_count, cudaStream_t st);
cudaError_t launch_rdm_rows(const void *C, int dtype, int ff_form, int n, const uint32_t *sa, const uint32_t *sb,
                            const uint16_t *stra, const uint16_t *strb, const uint16_t *ra, const uint16_t *rb, int Da,
                            int Db, int grid, const uint32_t *alist, const int *ainfo, double *partial,
                            cudaStream_t st);
cudaError_t launch_gather_c(const void *psi, int dtype, const uint32_t *idx, int count, void *out, cudaStream_t st);

struct RowTables {
    const uint32_t *sa, *sb, *sa_s, *sb_s;
    const uint16_t *stra, *strb, *ra, *rb;
    const void *eri, *hm, *Dt, *Jt;
    int N, Da, Db;
    const void *W2 = nullptr;  // pair-indexed same-spin integrals (split form)
};
cudaError_t launch_sigma_rows_ff(const void *C, void *lam, void *lamc, int dtype, int n, const RowTables &Tf,
                                 const double *hdiag, const double *Jp, double e_shift, double *partial, int K,
                                 void *Cf, void *Lf, int sm_count, cudaStream_t st);
cudaError_t launch_compact(const void *psi, void *C, int dtype, const uint32_t *sa, const uint32_t *sb, int Da,
                           int Db, int sm_count, cudaStream_t st);
cudaError_t launch_sigma_rows(const void *C, void *lam, void *lamc, int dtype, int n, const RowTables &T, const double *hdiag,
                              const double *Jp, double e_shift, double *partial, int K, cudaStream_t st,
                              const SameGemm *g, int sm_count);
cudaError_t launch_same_mats(int n, const RowTables &T, const double *hdiag, const double *Jp, float *Ma, float *Mb,
                             double *dA, double *dB, int lda, int ldb, cudaStream_t st);
cudaError_t launch_split_bf16x3(const float *x, uint16_t *out, size_t n, size_t piece, int sm_count, cudaStream_t st);
size_t ab_table_rows(int N, int Db);
size_t ab_rowb_elems(int Db);
cudaError_t launch_ab_table(const float *eri, const float *Jt, const uint16_t *strb, int N, int nb, int Db, uint16_t *Bp,
                            size_t pb, uint16_t *rowB, cudaStream_t st);
bool ab_tc_fits(int planes, int Da, int Db, int na, int nb, int N);
int ab_xi_ld(int Da);
int ab_h_ld(int Da);
int sigma_ab_chunk(int dtype, const RowTables &T, int nb, int want);
const int *sigma_ab_sizes(int dtype);

DevTables::~DevTables() {
    void *ptrs[] = {dbl,    sgl,   W,     hdiag, Jp,       hdiag_s,  Jp_s,  eri_r, hm_r, Dt,
                    Jt,     W2,    eri_ff, hm_ff, Dt_ff, Jt_ff, W2_ff, pass_dbl, pass_sgl, pass_W};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}
}  // namespace svk

using namespace svk;

// ---------------------------------------------------------------- errors

static thread_local std::string g_err = "no error";

namespace svk {
void set_thread_error(const std::string &m) { g_err = m; }
// the check words of the kernel units (sv_check.cuh)
uint32_t check_word_sector();
uint32_t check_word_rows();
uint32_t check_word_abtc();
uint32_t check_word_pool();
}  // namespace svk

static sv_status fail(sv_handle h, sv_status st, const std::string &msg) {
    g_err = msg;
    if (h) {
        h->err = msg;
        if (st == SV_ERR_CUDA) h->failed = true;
    }
    return st;
}

#define SV_CUDA(h, call)                                                                          \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            cudaGetLastError();                                                                   \
            return fail((h), SV_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
        }                                                                                         \
    } while (0)

#define SV_TRY(expr)                       \
    do {                                   \
        sv_status s_ = (expr);             \
        if (s_ != SV_OK) return s_;        \
    } while (0)

// Makes the handle's device current for the duration of a call and restores the
// caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------- buffers

static sv_status dev_alloc(sv_handle h, void **p, size_t bytes, const char *what) {
    *p = nullptr;
    if (h->max_bytes > 0 && h->bytes_owned + bytes > (uint64_t)h->max_bytes)
        return fail(h, SV_ERR_OOM, std::string("device byte cap reached allocating ") + what);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(h, SV_ERR_OOM, std::string("cudaMalloc failed for ") + what + ": " + cudaGetErrorString(e));
    }
    h->bytes_owned += bytes;
    return SV_OK;
}

static void dev_free(sv_handle h, void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    h->bytes_owned -= std::min<uint64_t>(h->bytes_owned, bytes);
}

// Bytes of one state-sized vector: 2^n amplitudes (dense storage) or the
// C(N, na) C(N, nb) amplitudes of the sector (sector storage).
static size_t vec_bytes(sv_handle h) { return (size_t)h->elems * h->amp_bytes; }

// The interleaved (amplitude, sigma) matrix of sector-sized vectors: 2 Da Db amplitudes
// (pool screening over pair lists, the sector adjoint sweep).
static sv_status ensure_clbuf(sv_handle h) {
    const size_t need = std::max<size_t>(2 * (size_t)h->Da * h->Db * h->amp_bytes, 16);
    if (h->CLbuf_bytes >= need) return SV_OK;
    dev_free(h, h->CLbuf, h->CLbuf_bytes);
    h->CLbuf = nullptr;
    h->CLbuf_bytes = 0;
    SV_TRY(dev_alloc(h, &h->CLbuf, need, "interleaved amplitudes and sigma"));
    h->CLbuf_bytes = need;
    return SV_OK;
}

// The adjoint vector.  Dense storage: lam and the reverse sweep's working copy of
// psi(theta) (`saved`) in one allocation, lam first, so that the sweep can also run on
// the two interleaved by amplitude in the same bytes (k_adjoint_i); where two vectors
// do not fit, lam alone (and `saved` separately, if at all).
static sv_status ensure_lam(sv_handle h) {
    if (h->lam) return SV_OK;
    if (h->storage == 0 && !h->saved) {
        void *p = nullptr;
        if (dev_alloc(h, &p, 2 * vec_bytes(h), "adjoint vector and working copy") == SV_OK) {
            h->lam = p;
            h->own_lam = true;
            h->lam_pair = true;
            h->saved = (uint8_t *)p + vec_bytes(h);
            return SV_OK;
        }
        cudaGetLastError();
    }
    SV_TRY(dev_alloc(h, &h->lam, vec_bytes(h), "adjoint vector"));
    h->own_lam = true;
    return SV_OK;
}

// The device flag of kernels with bounded waits and its pinned host copy.
static sv_status ensure_kerr(sv_handle h) {
    if (!h->kerr) {
        SV_TRY(dev_alloc(h, (void **)&h->kerr, 16, "kernel error flag"));
        SV_CUDA(h, cudaMemsetAsync(h->kerr, 0, sizeof(int), h->stream));
    }
    if (!h->hkerr) {
        if (cudaMallocHost((void **)&h->hkerr, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            h->hkerr = nullptr;
            return fail(h, SV_ERR_OOM, "pinned host allocation failed");
        }
        *h->hkerr = 0;
    }
    return SV_OK;
}

// Compact sigma [Db][Da] (sector-sized).
static sv_status ensure_lbuf(sv_handle h) {
    const size_t cb = std::max<size_t>((size_t)h->Da * h->Db * h->amp_bytes, 16);
    if (h->Lbuf_bytes >= cb) return SV_OK;
    dev_free(h, h->Lbuf, h->Lbuf_bytes);
    h->Lbuf = nullptr;
    h->Lbuf_bytes = 0;
    SV_TRY(dev_alloc(h, &h->Lbuf, cb, "compact sigma"));
    h->Lbuf_bytes = cb;
    return SV_OK;
}

static sv_status ensure_partials(sv_handle h, size_t doubles) {
    if (h->partials_cap >= doubles) return SV_OK;
    if (h->partials) dev_free(h, h->partials, h->partials_cap * sizeof(double));
    h->partials = nullptr;
    h->partials_cap = 0;
    void *p;
    SV_TRY(dev_alloc(h, &p, doubles * sizeof(double), "reduction scratch"));
    h->partials = (double *)p;
    h->partials_cap = doubles;
    return SV_OK;
}

static sv_status ensure_out(sv_handle h, size_t doubles) {
    if (h->dout_cap < doubles) {
        if (h->dout) dev_free(h, h->dout, h->dout_cap * sizeof(double));
        h->dout = nullptr;
        h->dout_cap = 0;
        void *p;
        SV_TRY(dev_alloc(h, &p, doubles * sizeof(double), "device outputs"));
        h->dout = (double *)p;
        h->dout_cap = doubles;
    }
    if (h->hpinned_cap < doubles) {
        if (h->hpinned) cudaFreeHost(h->hpinned);
        h->hpinned = nullptr;
        h->hpinned_cap = 0;
        void *p = nullptr;
        cudaError_t e = cudaMallocHost(&p, doubles * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, SV_ERR_OOM, "pinned host staging allocation failed");
        }
        h->hpinned = (double *)p;
        h->hpinned_cap = doubles;
    }
    return SV_OK;
}

// Phase boundary i: closes the handle's open NVTX range and opens one named `range`
// (none when NULL; the ranges mark the host-side span of each phase's launches for a
// timeline profiler, and cost nothing without one), and records CUDA event i on the
// handle's stream when profiling (sv_phase_times).
static sv_status mark(sv_handle h, int i, const char *range) {
    if (h->nvtx_open) nvtxRangePop();
    h->nvtx_open = range != nullptr;
    if (range) nvtxRangePushA(range);
    if (!h->profile) return SV_OK;
    if (!h->ev[i]) SV_CUDA(h, cudaEventCreate(&h->ev[i]));
    SV_CUDA(h, cudaEventRecord(h->ev[i], h->stream));
    return SV_OK;
}

// Closes a phase range an early return left open.
struct NvtxClose {
    sv_handle h;
    ~NvtxClose() {
        if (h && h->nvtx_open) {
            nvtxRangePop();
            h->nvtx_open = false;
        }
    }
};

// ms between two recorded events (0 when either is missing or unreadable).
static double elapsed_ev(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (!a || !b || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.0;
    }
    return ms;
}

static float elapsed(sv_handle h, int a, int b) {
    float ms = 0.f;
    if (h->ev[a] && h->ev[b] && cudaEventElapsedTime(&ms, h->ev[a], h->ev[b]) != cudaSuccess) {
        cudaGetLastError();
        ms = 0.f;
    }
    return ms;
}

// Basis indices of the (na, nb) sector in ascending order, on the device.
static sv_status ensure_sector(sv_handle h) {
    if (h->sector && h->sector_na == h->na && h->sector_nb == h->nb) return SV_OK;
    if (h->sector) dev_free(h, h->sector, h->sector_len * sizeof(uint32_t));
    h->sector = nullptr;
    const int N = h->n / 2;
    std::vector<uint32_t> sa, sb;
    for (uint32_t s = 0; s < (1u << N); ++s) {
        int c = __builtin_popcount(s);
        if (c == h->na) sa.push_back(s);
        if (c == h->nb) sb.push_back(s);
    }
    auto spread = [&](uint32_t s, int off) {
        uint32_t x = 0;
        for (int p = 0; p < N; ++p)
            if ((s >> p) & 1u) x |= 1u << (2 * p + off);
        return x;
    };
    std::vector<uint32_t> ea(sa.size()), eb(sb.size());
    for (size_t i = 0; i < sa.size(); ++i) ea[i] = spread(sa[i], 0);
    for (size_t i = 0; i < sb.size(); ++i) eb[i] = spread(sb[i], 1);
    std::vector<uint32_t> list;
    list.reserve(ea.size() * eb.size());
    for (uint32_t a : ea)
        for (uint32_t b : eb) list.push_back(map_bits(a | b, h->perm));
    std::sort(list.begin(), list.end());
    void *p;
    SV_TRY(dev_alloc(h, &p, std::max<size_t>(1, list.size()) * sizeof(uint32_t), "sector list"));
    h->sector = (uint32_t *)p;
    h->sector_len = list.size();
    h->sector_na = h->na;
    h->sector_nb = h->nb;
    if (!list.empty())
        SV_CUDA(h, cudaMemcpyAsync(h->sector, list.data(), list.size() * sizeof(uint32_t),
                                   cudaMemcpyHostToDevice, h->stream));
    SV_CUDA(h, cudaStreamSynchronize(h->stream));
    return SV_OK;
}

// String-row view of the (na, nb) sector: strings with na (nb) set bits among N,
// ascending; their ranks; their spread over the even (odd) bit positions.
static sv_status ensure_strings(sv_handle h) {
    if (h->str_sa && h->str_na == h->na && h->str_nb == h->nb) return SV_OK;
    if (h->str_sa) {
        for (void *p : {(void *)h->str_sa, (void *)h->str_sb, (void *)h->str_sa_s, (void *)h->str_sb_s,
                        (void *)h->str_a, (void *)h->str_b, (void *)h->rank_a, (void *)h->rank_b})
            cudaFree(p);
        h->bytes_owned -= std::min<uint64_t>(h->bytes_owned, h->str_bytes);
        h->str_sa = h->str_sb = h->str_sa_s = h->str_sb_s = nullptr;
    }
    const int N = h->n / 2;
    auto strings = [&](int k, std::vector<uint16_t> &str, std::vector<uint16_t> &rank) {
        rank.assign((size_t)1 << N, 0xFFFFu);
        str.clear();
        for (uint32_t s = 0; s < (1u << N); ++s)
            if (__builtin_popcount(s) == k) {
                rank[s] = (uint16_t)str.size();
                str.push_back((uint16_t)s);
            }
    };
    std::vector<uint16_t> sa16, sb16, ra, rb;
    strings(h->na, sa16, ra);
    strings(h->nb, sb16, rb);
    std::vector<uint32_t> spa(sa16.size()), spb(sb16.size()), spa_s(sa16.size()), spb_s(sb16.size());
    for (size_t i = 0; i < sa16.size(); ++i) {
        uint32_t x = 0;
        for (int p = 0; p < N; ++p) if ((sa16[i] >> p) & 1u) x |= 1u << (2 * p);
        spa[i] = x;
        spa_s[i] = map_bits(x, h->perm);
    }
    for (size_t i = 0; i < sb16.size(); ++i) {
        uint32_t x = 0;
        for (int p = 0; p < N; ++p) if ((sb16[i] >> p) & 1u) x |= 1u << (2 * p + 1);
        spb[i] = x;
        spb_s[i] = map_bits(x, h->perm);
    }
    size_t bytes = 0;
    auto up = [&](void **dst, const void *src, size_t nb) -> sv_status {
        SV_TRY(dev_alloc(h, dst, std::max<size_t>(nb, 16), "string tables"));
        bytes += std::max<size_t>(nb, 16);
        SV_CUDA(h, cudaMemcpy(*dst, src, nb, cudaMemcpyHostToDevice));
        return SV_OK;
    };
    SV_TRY(up((void **)&h->str_sa, spa.data(), spa.size() * 4));
    SV_TRY(up((void **)&h->str_sb, spb.data(), spb.size() * 4));
    SV_TRY(up((void **)&h->str_sa_s, spa_s.data(), spa_s.size() * 4));
    SV_TRY(up((void **)&h->str_sb_s, spb_s.data(), spb_s.size() * 4));
    SV_TRY(up((void **)&h->str_a, sa16.data(), sa16.size() * 2));
    SV_TRY(up((void **)&h->str_b, sb16.data(), sb16.size() * 2));
    SV_TRY(up((void **)&h->rank_a, ra.data(), ra.size() * 2));
    SV_TRY(up((void **)&h->rank_b, rb.data(), rb.size() * 2));
    h->str_bytes = bytes;
    h->Da = (int)sa16.size();
    h->Db = (int)sb16.size();
    h->str_na = h->na;
    h->str_nb = h->nb;
    h->h_stra = sa16;
    h->h_strb = sb16;
    h->h_ra = ra;
    h->h_rb = rb;
    if (h->storage == 1) return SV_OK;  // the state itself is the compact matrix
    size_t cb = (size_t)h->Da * h->Db * h->amp_bytes;
    if (h->Cbuf_bytes < cb) {
        dev_free(h, h->Cbuf, h->Cbuf_bytes);
        h->Cbuf = nullptr;
        h->Cbuf_bytes = 0;
        SV_TRY(dev_alloc(h, &h->Cbuf, std::max<size_t>(cb, 16), "compact sector amplitudes"));
        h->Cbuf_bytes = std::max<size_t>(cb, 16);
    }
    return SV_OK;
}

// ---------------------------------------------------------------- Hamiltonian tables

template <typename R>
static sv_status upload_tables(sv_handle h, sv_ham_handle ham, DevTables &T) {
    HostTables<R> ht;
    build_tables<R>(*ham, h->n, ht);
    permute_tables<R>(ht, h->perm, h->n);
    T.n_dbl = (int)ht.dbl.size();
    T.n_sgl = (int)ht.sgl.size();
    auto up = [&](void **dst, const void *src, size_t bytes) -> sv_status {
        cudaError_t e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) {
            cudaGetLastError();
            *dst = nullptr;
            return fail(h, SV_ERR_OOM, "Hamiltonian table allocation failed");
        }
        if (bytes) SV_CUDA(h, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
        return SV_OK;
    };
    SV_TRY(up(&T.dbl, ht.dbl.data(), ht.dbl.size() * sizeof(DoubleRec<R>)));
    SV_TRY(up(&T.sgl, ht.sgl.data(), ht.sgl.size() * sizeof(SingleRec<R>)));
    SV_TRY(up(&T.W, ht.W.data(), ht.W.size() * sizeof(R)));
    SV_TRY(up((void **)&T.hdiag, ht.hdiag.data(), ht.hdiag.size() * sizeof(double)));
    SV_TRY(up((void **)&T.Jp, ht.Jp.data(), ht.Jp.size() * sizeof(double)));
    SV_TRY(up((void **)&T.hdiag_s, ht.hdiag_s.data(), ht.hdiag_s.size() * sizeof(double)));
    SV_TRY(up((void **)&T.Jp_s, ht.Jp_s.data(), ht.Jp_s.size() * sizeof(double)));
    // spatial integrals in the state precision for the string-row kernel
    const int N = ham->n_orb;
    std::vector<R> eri(ham->eri.begin(), ham->eri.end()), hm(ham->h.begin(), ham->h.end());
    std::vector<R> Dt((size_t)N * N * N), Jt((size_t)N * N * N);
    auto E = [&](int p, int q, int r, int s) { return ham->eri[(((size_t)p * N + q) * N + r) * N + s]; };
    for (int q = 0; q < N; ++q)
        for (int p = 0; p < N; ++p)
            for (int k = 0; k < N; ++k) {
                Jt[((size_t)q * N + p) * N + k] = (R)E(q, p, k, k);
                Dt[((size_t)q * N + p) * N + k] = (R)(E(q, p, k, k) - E(q, k, k, p));
            }
    SV_TRY(up(&T.eri_r, eri.data(), eri.size() * sizeof(R)));
    SV_TRY(up(&T.hm_r, hm.data(), hm.size() * sizeof(R)));
    SV_TRY(up(&T.Dt, Dt.data(), Dt.size() * sizeof(R)));
    SV_TRY(up(&T.Jt, Jt.data(), Jt.size() * sizeof(R)));
    // same-spin doubles p1 < p2 -> q1 < q2 by pairs, W2[(p1,p2)][(q1,q2)] =
    // s0 ((q1p1|q2p2) - (q1p2|q2p1)), with the orbital-order part of the
    // Jordan-Wigner sign, s0 = (-1)^([p1<q2] + [q2<p2] + [p1<q1] + [p2<q1]), folded in;
    // the string-dependent part is the parity of the prefix-parity words of a and b
    // over the four orbitals (k_sigma_same).
    const int NP = N * (N - 1) / 2;
    std::vector<R> W2((size_t)std::max(NP, 1) * std::max(NP, 1));
    auto pidx = [&](int p, int q) { return p * N - p * (p + 1) / 2 + (q - p - 1); };
    for (int p1 = 0; p1 < N; ++p1)
        for (int p2 = p1 + 1; p2 < N; ++p2)
            for (int q1 = 0; q1 < N; ++q1)
                for (int q2 = q1 + 1; q2 < N; ++q2) {
                    const int s0 = (p1 < q2) ^ (q2 < p2) ^ (p1 < q1) ^ (p2 < q1);
                    const double v = E(q1, p1, q2, p2) - E(q1, p2, q2, p1);
                    W2[(size_t)pidx(p1, p2) * NP + pidx(q1, q2)] = (R)(s0 ? -v : v);
                }
    SV_TRY(up(&T.W2, W2.data(), W2.size() * sizeof(R)));
    if (sizeof(R) == 8) {
        // float-float copies (hi = nearest float, lo = nearest float of the rest) for variant 6
        auto split = [](const std::vector<R> &v) {
            std::vector<float> o(2 * v.size());
            for (size_t i = 0; i < v.size(); ++i) {
                const double x = (double)v[i];
                const float hi = (float)x;
                o[2 * i] = hi;
                o[2 * i + 1] = (float)(x - (double)hi);
            }
            return o;
        };
        const std::vector<float> e2 = split(eri), h2 = split(hm), d2 = split(Dt), j2 = split(Jt), w2 = split(W2);
        SV_TRY(up(&T.eri_ff, e2.data(), e2.size() * sizeof(float)));
        SV_TRY(up(&T.hm_ff, h2.data(), h2.size() * sizeof(float)));
        SV_TRY(up(&T.Dt_ff, d2.data(), d2.size() * sizeof(float)));
        SV_TRY(up(&T.Jt_ff, j2.data(), j2.size() * sizeof(float)));
        SV_TRY(up(&T.W2_ff, w2.data(), w2.size() * sizeof(float)));
    }
    return SV_OK;
}

static sv_status get_tables(sv_handle h, sv_ham_handle ham, DevTables **out) {
    std::string key = std::to_string(h->device) + "/" + std::to_string(h->n) + "/" + std::to_string((int)h->dtype);
    for (int q = 0; q < h->n; ++q) key += "," + std::to_string(h->perm[q]);
    auto it = ham->dev.find(key);
    if (it != ham->dev.end()) {
        *out = it->second.get();
        return SV_OK;
    }
    static uint64_t serial_counter = 0;  // guarded like the rest of a handle's calls: one caller at a time
    std::unique_ptr<DevTables> T(new DevTables());
    T->serial = ++serial_counter;
    T->n = h->n;
    T->dtype = h->dtype;
    if (single_prec(h->dtype)) SV_TRY(upload_tables<float>(h, ham, *T));
    else SV_TRY(upload_tables<double>(h, ham, *T));
    *out = T.get();
    ham->dev[key] = std::move(T);
    return SV_OK;
}

// ---------------------------------------------------------------- validation helpers

static sv_status check_ready(sv_handle h) {
    if (!h) return fail(nullptr, SV_ERR_ARG, "NULL handle");
    if (h->failed) return fail(h, SV_ERR_STATE, "handle failed earlier; prepare a state again");
    if (!h->prepared) return fail(h, SV_ERR_STATE, "no prepared state (call sv_prepare_hf or sv_prepare_state)");
    return SV_OK;
}

static sv_status build_ops(sv_handle h, const sv_excitation *ops, int n_ops, const double *theta,
                           std::vector<OpDesc> &out) {
    if (n_ops < 0) return fail(h, SV_ERR_ARG, "n_ops < 0");
    if (n_ops > 0 && (!ops || !theta)) return fail(h, SV_ERR_ARG, "NULL ops or theta");
    out.resize(n_ops);
    for (int k = 0; k < n_ops; ++k) {
        std::string why;
        if (!make_op(ops[k], h->n, h->perm, out[k], why)) {
            char buf[64];
            snprintf(buf, sizeof buf, "op %d: ", k);
            return fail(h, SV_ERR_ARG, buf + why);
        }
        if (!std::isfinite(theta[k])) return fail(h, SV_ERR_ARG, "non-finite theta");
        out[k].c = std::cos(theta[k]);
        out[k].s = std::sin(theta[k]);
    }
    return SV_OK;
}

static sv_status check_ham(sv_handle h, sv_ham_handle ham) {
    if (!ham) return fail(h, SV_ERR_ARG, "NULL Hamiltonian handle");
    if (ham->n_orb * 2 != h->n) return fail(h, SV_ERR_ARG, "Hamiltonian has n_orb != n_qubits / 2");
    return SV_OK;
}

// ---------------------------------------------------------------- internal steps

// Position of the qubit-space determinant x in the compact sector matrix
// C[rank(beta string)][rank(alpha string)], or 0xFFFFFFFF when x lies outside the
// (na, nb) sector.  Needs the host string tables (ensure_strings).
static uint32_t compact_index(sv_handle h, uint64_t x) {
    const int N = h->n / 2;
    uint32_t a = 0, b = 0;
    for (int p = 0; p < N; ++p) {
        a |= (uint32_t)((x >> (2 * p)) & 1u) << p;
        b |= (uint32_t)((x >> (2 * p + 1)) & 1u) << p;
    }
    if (__builtin_popcount(a) != h->na || __builtin_popcount(b) != h->nb) return 0xFFFFFFFFu;
    return (uint32_t)h->h_rb[b] * (uint32_t)h->Da + h->h_ra[a];
}

static sv_status prepare_reference(sv_handle h) {
    if (h->ref_kind == 1) {
        uint32_t addr = map_bits(h->ref_det, h->perm);
        if (h->storage == 1) {
            SV_TRY(ensure_strings(h));
            addr = compact_index(h, h->ref_det);
        }
        SV_CUDA(h, cudaMemsetAsync(h->psi, 0, vec_bytes(h), h->stream));
        SV_CUDA(h, launch_set_basis(h->psi, h->dtype, addr, h->stream));
        h->launches++;
    } else if (h->ref_kind == 2) {
        SV_CUDA(h, cudaMemcpyAsync(h->psi, h->ref_vec, vec_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
    } else {
        return fail(h, SV_ERR_STATE, "no reference state recorded");
    }
    return SV_OK;
}

// Sector storage: the alpha and beta pair lists of every op (k_build_lists), kept
// on the device and rebuilt only when the ops' masks (or the sector) change.
static sv_status ensure_op_lists(sv_handle h, const std::vector<OpDesc> &ops, OpLists &cache) {
    SV_TRY(ensure_strings(h));
    // the lists depend on the ops' masks and the sector only: reuse them when those match exactly
    std::vector<uint32_t> key;
    key.reserve(3 * ops.size() + 2);
    key.push_back((uint32_t)h->na);
    key.push_back((uint32_t)h->nb);
    for (const OpDesc &d : ops) {
        key.push_back(d.m);
        key.push_back(d.from);
        key.push_back(d.sm);
    }
    if (cache.buf && key == cache.key) return SV_OK;
    const int N = h->n / 2;
    const size_t ob = list_op_bytes();
    std::vector<uint8_t> host((ops.size() ? ops.size() : 1) * ob);
    std::vector<int> info(4 * ops.size());
    uint64_t off = 0;
    for (size_t k = 0; k < ops.size(); ++k) {
        int na_l = 0, nb_l = 0;  // the op's beta list follows its alpha list
        list_op_from(ops[k], N, h->na, h->nb, (uint32_t)off, host.data() + k * ob, &na_l, &nb_l);
        info[4 * k] = (int)off;
        info[4 * k + 1] = na_l;
        info[4 * k + 2] = (int)off + na_l;
        info[4 * k + 3] = nb_l;
        off += (uint64_t)(na_l + nb_l);
        if (off > (uint64_t)INT32_MAX) return fail(h, SV_ERR_ARG, "operator pair lists exceed 2^31 entries");
    }
    auto r16 = [](size_t x) { return (x + 15) / 16 * 16; };
    const size_t lb = r16((size_t)off * 4 + 16), obb = r16(std::max<size_t>(host.size(), 16)),
                 ib = r16(std::max<size_t>(info.size() * sizeof(int), 16));
    if (cache.bytes < lb + obb + ib) {
        dev_free(h, cache.buf, cache.bytes);
        cache.buf = nullptr;
        cache.bytes = 0;
        cache.key.clear();
        SV_TRY(dev_alloc(h, &cache.buf, lb + obb + ib, "operator pair lists"));
        cache.bytes = lb + obb + ib;
    }
    uint8_t *dops = (uint8_t *)cache.buf + lb;  // op records after the lists, then the int4 records
    int *dinfo = (int *)(dops + obb);
    SV_CUDA(h, cudaMemcpyAsync(dops, host.data(), ops.size() * ob, cudaMemcpyHostToDevice, h->stream));
    SV_CUDA(h, cudaMemcpyAsync(dinfo, info.data(), info.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    SV_CUDA(h, launch_build_lists(dops, (int)ops.size(), h->str_sa, h->str_sb, h->str_a, h->str_b, h->rank_a,
                                  h->rank_b, h->Da, h->Db, (uint32_t *)cache.buf, h->stream));
    h->launches++;
    SV_CUDA(h, cudaStreamSynchronize(h->stream));  // the host staging vectors go out of scope
    cache.key = key;
    cache.info = info;
    cache.dinfo = dinfo;
    return SV_OK;
}

// Dense sweeps touch runs as short as one amplitude: a 32-byte maximum L2 fetch
// granularity keeps the L2 from fetching larger blocks around runs of 32 or 64 bytes.
// The granularity is a limit of the whole CUDA context, so the entry points that run
// dense sweeps set the handle's value for the duration of the call and put the
// context's previous value back when they return (a hint: a refusal is ignored).  Only
// for states of at least four times the L2: smaller ones are served from L2, where the
// granularity buys nothing, and each change of the limit costs about half a millisecond
// of host time (measured on GB300), more than a small state's whole sweep.
struct L2FetchScope {
    size_t prev = 0;
    bool restore = false;
    explicit L2FetchScope(sv_handle h) {
        if (h->storage != 0 || h->l2_fetch <= 0) return;
        if (h->l2_bytes > 0 && vec_bytes(h) < 4 * (size_t)h->l2_bytes) return;
        if (cudaDeviceGetLimit(&prev, cudaLimitMaxL2FetchGranularity) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        if (prev == (size_t)h->l2_fetch) return;
        if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)h->l2_fetch) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        restore = true;
    }
    ~L2FetchScope() {
        if (restore && cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, prev) != cudaSuccess) cudaGetLastError();
    }
    L2FetchScope(const L2FetchScope &) = delete;
    L2FetchScope &operator=(const L2FetchScope &) = delete;
};

// The 1-RDM's alpha-pair lists: for each orbital pair p < q (in (p, q) order) the alpha
// strings holding q but not p with their partners (q -> p) and the parity of their alpha
// bits strictly between spin-orbitals 2p and 2q; kept while the sector is unchanged.
static sv_status ensure_rdm_lists(sv_handle h) {
    const int N = h->n / 2;
    std::vector<OpDesc> ops;
    for (int p = 0; p < N; ++p)
        for (int q = p + 1; q < N; ++q) {
            OpDesc d;
            d.m = (1u << (2 * p)) | (1u << (2 * q));
            d.from = 1u << (2 * q);
            d.sm = ((1u << (2 * q)) - 1u) & ~((2u << (2 * p)) - 1u);
            d.nbits = 2;
            d.pos[0] = 2 * p;
            d.pos[1] = 2 * q;
            ops.push_back(d);
        }
    if (ops.empty()) {
        SV_TRY(ensure_strings(h));  // one orbital: no pairs; the kernel reads no list
        return SV_OK;
    }
    return ensure_op_lists(h, ops, h->rdm_lists);
}

// Sector storage: the ops' (cos, sin) on the device for whole-sweep launches (uploaded
// once per call; the reverse sweep reuses them).
static sv_status upload_sweep_angles(sv_handle h, const std::vector<OpDesc> &ops) {
    const size_t need = 256 + 2 * std::max<size_t>(ops.size(), 1) * sizeof(double);
    if (h->sweep_bytes < need) {
        dev_free(h, h->sweep_buf, h->sweep_bytes);
        h->sweep_buf = nullptr;
        h->sweep_bytes = 0;
        SV_TRY(dev_alloc(h, &h->sweep_buf, need, "sweep angles"));
        h->sweep_bytes = need;
    }
    h->sweep_host.resize(2 * ops.size());
    for (size_t k = 0; k < ops.size(); ++k) {
        h->sweep_host[2 * k] = ops[k].c;
        h->sweep_host[2 * k + 1] = ops[k].s;
    }
    if (!ops.empty())
        SV_CUDA(h, cudaMemcpyAsync((uint8_t *)h->sweep_buf + 256, h->sweep_host.data(), 2 * ops.size() * sizeof(double),
                                   cudaMemcpyHostToDevice, h->stream));
    return SV_OK;
}

// One launch for a whole sector sweep (forward on psi, or reverse on the interleaved
// matrix with gradient partials [L][grid]); false (nothing launched) where the
// cooperative launch is refused or the option is off: the caller then launches per op.
static bool sweep_once(sv_handle h, bool adjoint, void *buf, size_t L, int grid, double *partial) {
    if (!h->sweep_mode || L == 0 || grid <= 0 || !h->sweep_buf || !h->kerr) return false;
    if (cudaMemsetAsync(h->sweep_buf, 0, sizeof(unsigned int), h->stream) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const cudaError_t e = launch_sweep_l(buf, h->dtype, adjoint, (const uint32_t *)h->lists.buf, h->lists.dinfo,
                                         (const double *)((const uint8_t *)h->sweep_buf + 256), (int)L, h->Da, h->Db,
                                         grid,
                                         (unsigned int *)h->sweep_buf, h->kerr, (uint32_t)h->wait_polls, partial,
                                         h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    h->launches++;
    cudaMemcpyAsync(h->hkerr, h->kerr, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    return true;
}

static sv_status forward(sv_handle h, const std::vector<OpDesc> &ops, bool checkpoints) {
    const int64_t C = h->ckpt_interval;
    if (h->storage == 1 && !ops.empty()) {
        SV_TRY(ensure_op_lists(h, ops, h->lists));
        SV_TRY(ensure_kerr(h));
        SV_TRY(upload_sweep_angles(h, ops));
        // one launch for the whole sweep unless checkpoint copies are due in the middle
        if (!(checkpoints && C > 0 && (size_t)C < ops.size()) &&
            sweep_once(h, false, h->psi, ops.size(), sweep_grid(h->dtype, false, h->Db, h->sm_count, h->sweep_bps),
                       nullptr))
            return SV_OK;
    }
    const uint32_t *L = (const uint32_t *)h->lists.buf;
    const int G = sector_grid(h->Db, h->sm_count, h->sect_bps);
    for (size_t k = 0; k < ops.size(); ++k) {
        if (h->storage == 1) {
            const int *li = &h->lists.info[4 * k];
            SV_CUDA(h, launch_rotate_l(h->psi, h->dtype, L + li[0], li[1], L + li[2], li[3], h->Da, ops[k].c,
                                       ops[k].s, G, h->stream));
        } else {
            SV_CUDA(h, launch_rotate(h->psi, h->dtype, h->n, ops[k], h->sm_count, h->rot_bps, h->stream));
        }
        h->launches++;
        if (checkpoints && C > 0 && (k + 1) % (size_t)C == 0 && k + 1 < ops.size()) {
            size_t j = (k + 1) / (size_t)C - 1;
            if (j < h->ckpt.size() && h->ckpt[j])
                SV_CUDA(h, cudaMemcpyAsync(h->ckpt[j], h->psi, vec_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
        }
    }
    return SV_OK;
}

// Checkpoint slots for an ansatz of L gates (as many as the byte cap allows).
static void plan_checkpoints(sv_handle h, size_t L) {
    size_t want = 0;
    if (h->ckpt_interval > 0 && L > 1) want = (L - 1) / (size_t)h->ckpt_interval;
    while (h->ckpt.size() > want) {
        dev_free(h, h->ckpt.back(), vec_bytes(h));
        h->ckpt.pop_back();
    }
    while (h->ckpt.size() < want) {
        void *p = nullptr;
        if (dev_alloc(h, &p, vec_bytes(h), "checkpoint") != SV_OK) {
            cudaGetLastError();
            break;  // fewer checkpoints: the reverse sweep uncomputes instead
        }
        h->ckpt.push_back(p);
    }
}

// Rows per chunk of the split string-row expectation (0: single kernel).
static int row_chunk(sv_handle h, const RowTables &R) {
    if (h->expect_variant == 2) return 0;
    return sigma_ab_chunk(h->dtype, R, h->nb, (int)h->ab_chunk);
}

// Whether the string-row expectation takes the same-spin products (variant 4):
// single-precision states whose split form fits and whose strings number at most
// 4096 per spin (matrices up to 64 MB).  Automatic choice (variant 0): where the
// sector has at least 2^20 determinants and every string at least 5% of the strings
// of its spin as same-spin partners (singles and doubles), so that the dense
// products do at most 20 times the multiplies of the sparse sums.
static bool use_same_gemm(sv_handle h, int K) {
    if (!single_prec(h->dtype) || K == 0 || h->Da > 4096 || h->Db > 4096) return false;
    if (h->expect_variant == 4 || h->expect_variant == 5) return true;
    if (h->expect_variant != 0) return false;
    const int N = h->n / 2;
    auto c2 = [](long x) { return x * (x - 1) / 2; };
    auto dens = [&](int ne, int D) {
        const long ns = (long)ne * (N - ne), nd = c2(ne) * c2(N - ne);
        return (double)(ns + nd) / (double)D;
    };
    return (double)h->Da * h->Db >= (double)(1 << 20) && dens(h->na, h->Da) >= 0.05 && dens(h->nb, h->Db) >= 0.05;
}

// Whether the same-spin product form also takes the alpha-beta part as tensor-core
// products (variant 5; where k_ab_tc's limits hold, else variant 4).  Automatic choice
// (variant 0, once the same-spin products are chosen): where its product planes
// (planes x Db x (nb (N - nb) + 1) x Da floats) take at most 16 GiB and fit under the
// handle's byte cap.
static bool use_ab_tc(sv_handle h) {
    if (h->expect_variant != 5 && h->expect_variant != 0) return false;
    const int planes = is_complex(h->dtype) ? 2 : 1, N = h->n / 2;
    if (!ab_tc_fits(planes, h->Da, h->Db, h->na, h->nb, N)) return false;
    if (h->expect_variant == 5) return true;
    const double hb = 4.0 * planes * (double)h->Db * (h->nb * (N - h->nb) + 1) * (double)ab_h_ld(h->Da);
    if (hb > (double)(16ull << 30)) return false;
    return h->max_bytes <= 0 || (double)h->bytes_owned + (h->ab_H_bytes >= hb ? 0.0 : hb) <= (double)h->max_bytes;
}

// The same-spin matrices of the table set and sector (built on first use, kept until
// either changes) and the work planes.  Rows of Ma, X and of Mb, Xt are padded to a
// multiple of 8 elements with zeros (16-byte row strides of the bf16 pieces, as TMA
// requires).
static sv_status ensure_same_gemm(sv_handle h, DevTables *T, const RowTables &R, SameGemm *g) {
    SV_TRY(ensure_kerr(h));
    const size_t Da = (size_t)h->Da, Db = (size_t)h->Db, lda = (Da + 7) / 8 * 8, ldb = (Db + 7) / 8 * 8;
    // [Ma | Mb] (float32), the one-spin diagonals, then the three bf16 pieces of [Ma | Mb]
    // then the three bf16 pieces of the alpha-beta integral table (k_ab_tc) when N^2 <= 256
    const int N = h->n / 2;
    const size_t rowsB = N * N <= 256 ? ab_table_rows(N, (int)Db) : 0, pbB = rowsB * 256;
    const size_t nm = Da * lda + Db * ldb, mf = nm * sizeof(float), dof = (mf + 255) / 256 * 256,
                 sof = (dof + (Da + Db) * sizeof(double) + 255) / 256 * 256,
                 bof = (sof + 3 * nm * sizeof(uint16_t) + 255) / 256 * 256,
                 rbo = (bof + 3 * pbB * sizeof(uint16_t) + 255) / 256 * 256,
                 mb = rbo + (rowsB ? ab_rowb_elems((int)Db) * sizeof(uint16_t) : 0);
    float *Ma = nullptr;
    if (!h->sg_mats || h->sg_serial != T->serial || h->sg_na != h->na || h->sg_nb != h->nb) {
        if (h->sg_mats_bytes < mb) {
            dev_free(h, h->sg_mats, h->sg_mats_bytes);
            h->sg_mats = nullptr;
            h->sg_mats_bytes = 0;
            SV_TRY(dev_alloc(h, &h->sg_mats, mb, "same-spin matrices"));
            h->sg_mats_bytes = mb;
        }
        Ma = (float *)h->sg_mats;
        double *dA = (double *)((uint8_t *)h->sg_mats + dof);
        SV_CUDA(h, launch_same_mats(h->n, R, T->hdiag, T->Jp, Ma, Ma + Da * lda, dA, dA + Da, (int)lda, (int)ldb,
                                    h->stream));
        SV_CUDA(h, launch_split_bf16x3(Ma, (uint16_t *)((uint8_t *)h->sg_mats + sof), nm, nm, h->sm_count,
                                       h->stream));
        h->launches += 2;
        if (rowsB) {
            SV_CUDA(h, launch_ab_table((const float *)R.eri, (const float *)R.Jt, h->str_b, N, h->nb, (int)Db,
                                       (uint16_t *)((uint8_t *)h->sg_mats + bof), pbB,
                                       (uint16_t *)((uint8_t *)h->sg_mats + rbo), h->stream));
            h->launches += 2;
        }
        h->sg_serial = T->serial;
        h->sg_na = h->na;
        h->sg_nb = h->nb;
    }
    Ma = (float *)h->sg_mats;
    const int planes = is_complex(h->dtype) ? 2 : 1;
    // X [planes][Db][lda], G [planes][Db][Da], Xt [planes][Da][ldb] (tensor-core form)
    // (each region rounded to 256 bytes: aligned starts for vector loads and TMA)
    // the three bf16 pieces of X and those of the transposes [planes][Da][ldb]; then G
    // float32 [planes][Db][Da]
    const size_t nx = (size_t)planes * Db * lda, nt = (size_t)planes * Da * ldb, ng = (size_t)planes * Db * Da;
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t xb = r256(3 * nx * sizeof(uint16_t)), tb = r256(3 * nt * sizeof(uint16_t));
    // variant 5: then the phased amplitudes as interleaved bf16 pieces [Db][ldi][3] words
    const bool abtc = use_ab_tc(h) && rowsB;
    const size_t ldi = ab_xi_ld((int)Da), gb = r256(ng * sizeof(float)), ib = abtc ? r256(Db * ldi * 12) : 0;
    const size_t need = xb + tb + gb + ib;
    const uint64_t geom = ((uint64_t)Da << 32) | ((uint64_t)Db << 3) | ((uint64_t)planes << 2) | (abtc ? 2u : 0u);
    if (h->sg_buf_bytes < need || h->sg_buf_geom != geom) {
        if (h->sg_buf_bytes < need) {
            dev_free(h, h->sg_buf, h->sg_buf_bytes);
            h->sg_buf = nullptr;
            h->sg_buf_bytes = 0;
            SV_TRY(dev_alloc(h, &h->sg_buf, need, "same-spin product planes"));
            h->sg_buf_bytes = need;
        }
        SV_CUDA(h, cudaMemsetAsync(h->sg_buf, 0, need, h->stream));  // the row padding stays zero
        h->sg_buf_geom = geom;
    }
    g->Ma = Ma;
    g->Mb = Ma + Da * lda;
    g->dA = (const double *)((const uint8_t *)h->sg_mats + dof);
    g->dB = g->dA + Da;
    uint8_t *B = (uint8_t *)h->sg_buf;
    g->Mp = (const uint16_t *)((const uint8_t *)h->sg_mats + sof);
    g->pm = nm;
    g->Xp = (uint16_t *)B;
    g->px = nx;
    g->Xtp = (uint16_t *)(B + xb);
    g->pt = nt;
    g->G = (float *)(B + xb + tb);
    g->planes = planes;
    g->lda = (int)lda;
    g->ldb = (int)ldb;
    g->err = h->kerr;
    g->spins = (uint32_t)h->wait_polls;
    g->ev = nullptr;
    if (h->profile) {
        for (cudaEvent_t &e : h->tcev)
            if (!e) SV_CUDA(h, cudaEventCreate(&e));
        g->ev = h->tcev;
    }
    g->stall = h->test_stall;
    g->abtc = 0;
    bool ab_ok = abtc;
    const int ncols = h->nb * (N - h->nb) + 1;
    const size_t hplane = Db * (size_t)ncols * ab_h_ld((int)Da), hb = (size_t)planes * hplane * sizeof(float);
    if (ab_ok && h->ab_H_bytes < hb) {
        // H [planes][Db][ncols][ab_h_ld(Da)]; where the automatic choice cannot have it, variant 4 runs
        dev_free(h, h->ab_H, h->ab_H_bytes);
        h->ab_H = nullptr;
        h->ab_H_bytes = 0;
        const sv_status st = dev_alloc(h, (void **)&h->ab_H, hb, "alpha-beta product planes");
        if (st != SV_OK && h->expect_variant != 0) return st;
        if (st != SV_OK) {
            cudaGetLastError();
            ab_ok = false;
        } else {
            h->ab_H_bytes = hb;
        }
    }
    if (ab_ok) {
        g->abtc = 1;
        g->Xi = (uint32_t *)(B + xb + tb + gb);
        g->ldi = (int)ldi;
        g->Bp = (const uint16_t *)((const uint8_t *)h->sg_mats + bof);
        g->rowB = (const uint16_t *)((const uint8_t *)h->sg_mats + rbo);
        g->pb = pbB;
        g->H = h->ab_H;
        g->hplane = hplane;
        g->ldh = ab_h_ld((int)Da);
        g->ncols = ncols;
        g->na = h->na;
        g->nb = h->nb;
        g->err = h->kerr;
    }
    return SV_OK;
}

// After a stream synchronisation: a kernel whose bounded wait ran out (k_same_tc, k_ab_tc).
static sv_status check_kernel_flag(sv_handle h) {
    if (h->hkerr && *h->hkerr) {
        *h->hkerr = 0;
        if (h->kerr) cudaMemsetAsync(h->kerr, 0, sizeof(int), h->stream);
        h->failed = true;
        return fail(h, SV_ERR_CUDA, "a bounded wait ran out (tensor-core products or a sweep's grid barrier)");
    }
    return SV_OK;
}

// The string-row expectation (sigma into lam at storage addresses, or into lamc in
// compact form), with or without the same-spin products; counts the launches.
// Whether the expectation takes the float-float split form (variant 6): float64 states
// whose split form fits; the automatic choice (variant 0) for them.
static bool use_ff(sv_handle h, int K) {
    if (single_prec(h->dtype) || K == 0) return false;
    return h->expect_variant == 6 || h->expect_variant == 0;
}

// Bytes of one compact float-float matrix of the state (rounded to 256).
static size_t ff_matrix_bytes(sv_handle h) {
    const size_t one = (size_t)h->Da * h->Db * (is_complex(h->dtype) ? 16 : 8);
    return (one + 255) / 256 * 256;
}

// The float-float work buffer with at least `bytes` (kept across calls; the expectation
// takes two matrices, the 1-RDM one).  SV_OK, or the allocation's status with nothing
// held where the bytes are not available.
static sv_status ensure_ffbuf(sv_handle h, size_t bytes) {
    if (h->ffbuf_bytes >= bytes) return SV_OK;
    dev_free(h, h->ffbuf, h->ffbuf_bytes);
    h->ffbuf = nullptr;
    h->ffbuf_bytes = 0;
    const sv_status st = dev_alloc(h, &h->ffbuf, bytes, "float-float work matrices");
    if (st == SV_OK) h->ffbuf_bytes = bytes;
    else cudaGetLastError();
    return st;
}

// The 1-RDM rows' input: the compact matrix Cm itself, or, for float64 states under
// SV_OPT_RDM_VARIANT 3 or the automatic choice, its float-float form in the work buffer
// (the automatic choice keeps float64 rows where that buffer cannot be had).
static sv_status rdm_input(sv_handle h, const void *Cm, const void **src, int *ff_form) {
    *src = Cm;
    *ff_form = 0;
    if (single_prec(h->dtype) || (h->rdm_variant != 0 && h->rdm_variant != 3)) return SV_OK;
    const sv_status st = ensure_ffbuf(h, ff_matrix_bytes(h));
    if (st != SV_OK) return h->rdm_variant == 3 ? st : SV_OK;
    SV_CUDA(h, launch_to_ff(Cm, h->dtype, (size_t)h->Da * h->Db, h->ffbuf, h->sm_count, h->stream));
    h->launches++;
    *src = h->ffbuf;
    *ff_form = 1;
    return SV_OK;
}

static sv_status sigma_rows(sv_handle h, DevTables *T, const RowTables &R, const void *C, void *lam, void *lamc,
                            double e_shift) {
    const int K = row_chunk(h, R);
    if (use_ff(h, K) && T->eri_ff) {
        const size_t r = ff_matrix_bytes(h);
        const sv_status st = ensure_ffbuf(h, 2 * r);
        if (st != SV_OK && h->expect_variant == 6) return st;
        const bool ok = st == SV_OK;  // the automatic choice falls back to the float64 split form
        if (ok) {
        RowTables Tf = R;
        Tf.eri = T->eri_ff;
        Tf.hm = T->hm_ff;
        Tf.Dt = T->Dt_ff;
        Tf.Jt = T->Jt_ff;
        Tf.W2 = T->W2_ff;
        SV_CUDA(h, launch_sigma_rows_ff(C, lam, lamc, h->dtype, h->n, Tf, T->hdiag, T->Jp, e_shift, h->partials, K,
                                        h->ffbuf, (uint8_t *)h->ffbuf + r, h->sm_count, h->stream));
        h->launches += 4;
        return SV_OK;
        }
    }
    SameGemm g;
    const bool sg = use_same_gemm(h, K);
    if (sg) SV_TRY(ensure_same_gemm(h, T, R, &g));
    SV_CUDA(h, launch_sigma_rows(C, lam, lamc, h->dtype, h->n, R, T->hdiag, T->Jp, e_shift, h->partials, K,
                                 h->stream, sg ? &g : nullptr, h->sm_count));
    h->launches += sg ? 5 : (K ? 2 : 1);
    if (sg && g.ev) h->tc_timed = 1 | (g.abtc ? 2 : 0);
    if (sg)
        SV_CUDA(h, cudaMemcpyAsync(h->hkerr, h->kerr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    return SV_OK;
}

// Expectation pass over the current state: writes the float64 sums of
// <psi|(H - c)|psi> and <psi|psi> into dout[out_off], dout[out_off + 1] (device),
// and sigma = (H - c) psi into `sigma` when it is not NULL (a state-sized vector), or,
// for dense storage with the string-row forms, into the compact [Db][Da] matrix
// `sigma_c` when that is not NULL.
static sv_status expectation(sv_handle h, sv_ham_handle ham, DevTables *T, void *sigma, double c, int out_off,
                             void *sigma_c = nullptr) {
    if (h->storage == 1) {
        // the state is already the compact matrix; sigma is compact too (every entry written)
        SV_TRY(ensure_strings(h));
        SV_TRY(ensure_partials(h, 3 * (size_t)h->Db));
        RowTables R{h->str_sa, h->str_sb, h->str_sa_s, h->str_sb_s, h->str_a, h->str_b, h->rank_a, h->rank_b,
                    T->eri_r, T->hm_r, T->Dt, T->Jt, h->n / 2, h->Da, h->Db, T->W2};
        SV_TRY(sigma_rows(h, T, R, h->psi, nullptr, sigma, ham->e_nuc - c));
        SV_CUDA(h, launch_reduce_rows(h->partials, 2, h->Db, h->dout + out_off, h->stream));
        h->launches++;
        return SV_OK;
    }
    if (h->expect_variant != 1 || !is_complex(h->dtype)) {  // the record scan serves complex states
        // string rows (default)
        SV_TRY(ensure_strings(h));
        SV_TRY(ensure_partials(h, 3 * (size_t)h->Db));
        if (sigma_c) sigma = nullptr;
        if (sigma) SV_CUDA(h, cudaMemsetAsync(sigma, 0, vec_bytes(h), h->stream));
        SV_CUDA(h, launch_compact(h->psi, h->Cbuf, h->dtype, h->str_sa_s, h->str_sb_s, h->Da, h->Db, h->sm_count,
                                  h->stream));
        h->launches++;
        RowTables R{h->str_sa, h->str_sb, h->str_sa_s, h->str_sb_s, h->str_a, h->str_b, h->rank_a, h->rank_b,
                    T->eri_r, T->hm_r, T->Dt, T->Jt, h->n / 2, h->Da, h->Db, T->W2};
        SV_TRY(sigma_rows(h, T, R, h->Cbuf, sigma, sigma_c, ham->e_nuc - c));
        SV_CUDA(h, launch_reduce_rows(h->partials, 2, h->Db, h->dout + out_off, h->stream));
        h->launches++;
        return SV_OK;
    }
    SV_TRY(ensure_sector(h));
    int grid = expect_gather_grid(h->sector_len, h->sm_count);
    SV_TRY(ensure_partials(h, 2 * (size_t)grid));
    if (sigma) SV_CUDA(h, cudaMemsetAsync(sigma, 0, vec_bytes(h), h->stream));
    SV_CUDA(h, launch_expect_gather(h->psi, sigma, h->dtype, h->n, h->sector, h->sector_len, *T,
                                    ham->e_nuc - c, grid, h->partials, h->stream));
    h->launches++;
    SV_CUDA(h, launch_reduce_rows(h->partials, 2, grid, h->dout + out_off, h->stream));
    h->launches++;
    return SV_OK;
}

// Shift constant c of lambda = (H - c) psi: the diagonal energy of the reference
// determinant (HF) or of the largest-weight determinant of a stored reference.
static double shift_for(sv_handle h, sv_ham_handle ham) {
    return diag_energy(*ham, h->ref_det, h->n);
}

// ---------------------------------------------------------------- storage layout

// Least-used qubits go to the lowest address bits: an excitation whose lowest
// address bit is b touches runs of 2^b consecutive amplitudes, so keeping the
// frequently excited qubits high keeps the rotation kernels' runs long.
static void layout_from_ops(int n, const sv_excitation *ops, int n_ops, int *perm) {
    std::vector<long> cnt(n, 0);
    for (int k = 0; k < n_ops; ++k) {
        const sv_excitation &e = ops[k];
        const bool dbl = e.kind == 2 || e.kind == 4;
        int qs[4] = {e.occ[0], e.vir[0], dbl ? e.occ[1] : -1, dbl ? e.vir[1] : -1};
        for (int q : qs)
            if (q >= 0 && q < n) cnt[q]++;
    }
    std::vector<int> order(n);
    for (int q = 0; q < n; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cnt[a] < cnt[b]; });
    for (int k = 0; k < n; ++k) perm[order[k]] = k;
    for (int q = n; q < 32; ++q) perm[q] = q;
}

static void drop_layout_caches(sv_handle h) {
    if (h->sector) dev_free(h, h->sector, h->sector_len * sizeof(uint32_t));
    h->sector = nullptr;
    h->sector_na = h->sector_nb = -1;
    h->str_na = h->str_nb = -1;  // string tables rebuilt on next use
}

// Move the prepared state (and a stored reference) to layout `np`.
static sv_status relayout(sv_handle h, const int *np) {
    bool same = true;
    for (int q = 0; q < h->n; ++q) same = same && (np[q] == h->perm[q]);
    if (same) return SV_OK;
    int inv_old[32], sg[32];
    for (int q = 0; q < h->n; ++q) inv_old[h->perm[q]] = q;
    for (int j = 0; j < h->n; ++j) sg[j] = np[inv_old[j]];
    if (h->prepared || h->ref_kind == 2) SV_TRY(ensure_lam(h));
    if (h->prepared) {
        SV_CUDA(h, launch_permute(h->psi, h->lam, h->dtype, h->n, sg, h->sm_count, h->stream));
        h->launches++;
        SV_CUDA(h, cudaMemcpyAsync(h->psi, h->lam, vec_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
    }
    if (h->ref_kind == 2 && h->ref_vec) {
        SV_CUDA(h, launch_permute(h->ref_vec, h->lam, h->dtype, h->n, sg, h->sm_count, h->stream));
        h->launches++;
        SV_CUDA(h, cudaMemcpyAsync(h->ref_vec, h->lam, vec_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
    }
    for (int q = 0; q < 32; ++q) h->perm[q] = q < h->n ? np[q] : q;
    drop_layout_caches(h);
    return SV_OK;
}

static bool is_identity(sv_handle h) {
    for (int q = 0; q < h->n; ++q)
        if (h->perm[q] != q) return false;
    return true;
}

// ---------------------------------------------------------------- autotuning

// Fastest of `reps` runs of fn (launches on the handle's stream), in ms, timed with
// CUDA events on that stream; negative when fn failed.
template <typename F>
static float time_best(sv_handle h, cudaEvent_t e0, cudaEvent_t e1, F fn, int reps = 3) {
    float best = -1.f;
    for (int r = 0; r < reps; ++r) {
        if (cudaEventRecord(e0, h->stream) != cudaSuccess) return -1.f;
        if (fn() != SV_OK) return -1.f;
        if (cudaEventRecord(e1, h->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.f;
        if (best < 0.f || ms < best) best = ms;
    }
    return best;
}

static sv_status autotune_impl(sv_handle h, sv_ham_handle ham, const std::vector<OpDesc> &d, cudaEvent_t e0,
                               cudaEvent_t e1) {
    DevTables *T;
    SV_TRY(get_tables(h, ham, &T));
    SV_TRY(ensure_lam(h));
    SV_TRY(ensure_out(h, 2));
    SV_TRY(ensure_strings(h));
    const double c = shift_for(h, ham);
    // 1. expectation form: the one-kernel string rows, and the split form at every chunk size
    {
        RowTables R{h->str_sa, h->str_sb, h->str_sa_s, h->str_sb_s, h->str_a, h->str_b, h->rank_a, h->rank_b,
                    T->eri_r, T->hm_r, T->Dt, T->Jt, h->n / 2, h->Da, h->Db, T->W2};
        const int *sizes = sigma_ab_sizes(h->dtype);
        int best_v = 2;
        int64_t best_k = 0;
        float best_t = -1.f;
        // split form; same-spin products and the tensor-core alpha-beta form (single
        // precision); the float-float split form (float64)
        const bool sp = single_prec(h->dtype);
        for (int i = -1; i < (sp ? 9 : 8); ++i) {
            h->expect_variant = i < 0 ? 2 : (i < 4 ? 3 : (!sp ? 6 : (i < 8 ? 4 : 5)));
            h->ab_chunk = i < 0 ? 0 : (i < 8 ? sizes[i & 3] : 0);
            if (i >= 0 && i < 8 && row_chunk(h, R) != sizes[i & 3]) continue;  // that size does not fit
            if (sp && i >= 4 && !use_same_gemm(h, row_chunk(h, R))) continue;
            if (i == 8 && !use_ab_tc(h)) continue;
            const float t = time_best(h, e0, e1, [&] { return expectation(h, ham, T, h->lam, c, 0); });
            if (t < 0.f) return fail(h, SV_ERR_CUDA, "autotune: expectation candidate failed");
            if (best_t < 0.f || t < best_t) {
                best_t = t;
                best_v = h->expect_variant;
                best_k = h->ab_chunk;
            }
        }
        h->expect_variant = best_v;
        h->ab_chunk = best_k;
    }
    // 2. rotation / adjoint launch geometry, on copies of psi in the adjoint vector and the
    //    saved-state buffer (psi is left alone): one rotation plus one adjoint step per candidate
    if (!d.empty()) {
        if (!h->saved) {  // as in sv_energy_grad: optional under the byte cap
            void *p = nullptr;
            if (dev_alloc(h, &p, vec_bytes(h), "saved final state") == SV_OK) h->saved = p;
            else cudaGetLastError();
        }
        const bool adj = h->saved != nullptr;  // without it only the rotation is timed
        SV_CUDA(h, cudaMemcpyAsync(h->lam, h->psi, vec_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
        if (adj) SV_CUDA(h, cudaMemcpyAsync(h->saved, h->psi, vec_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
        size_t k = 0;  // a representative op: the first double whose touched runs are long
        for (size_t j = 0; j < d.size(); ++j)
            if (d[j].nbits == 4 && d[j].pos[0] >= 4) { k = j; break; }
        // sector storage with whole-sweep launches: the two sweeps themselves are timed, on
        // copies (blocks per SM 1, 2, 4, 8); else one rotation and one adjoint step
        const bool sweeps = h->storage == 1 && h->sweep_mode && h->ckpt_interval <= 0 && adj;
        const int cands_op[] = {4, 8, 16, 32}, cands_sw[] = {1, 2, 4, 8};
        int best_b = 8;
        float best_t = -1.f;
        if (h->storage == 1) SV_TRY(ensure_op_lists(h, d, h->lists));
        SV_TRY(ensure_partials(h, (size_t)h->sm_count * 32 * (sweeps ? d.size() : 1)));
        if (sweeps) {
            SV_TRY(ensure_kerr(h));
            SV_TRY(upload_sweep_angles(h, d));
        }
        // sector storage: the adjoint step as sv_energy_grad runs it (interleaved unless checkpoints resync psi)
        bool inter = h->storage == 1 && adj && h->ckpt_interval <= 0;
        if (inter && ensure_clbuf(h) != SV_OK) {
            cudaGetLastError();
            inter = false;
        }
        if (inter) {
            SV_CUDA(h, launch_interleave(h->lam, h->saved, h->dtype, h->CLbuf, (size_t)h->Da * h->Db, h->sm_count,
                                         h->stream));
        }
        for (int ci = 0; ci < 4; ++ci) {
            const int b = (sweeps && inter) ? cands_sw[ci] : cands_op[ci];
            float t;
            if (sweeps && inter) {
                const int Gf = sweep_grid(h->dtype, false, h->Db, h->sm_count, b),
                          Gr = sweep_grid(h->dtype, true, h->Db, h->sm_count, b);
                t = time_best(h, e0, e1, [&]() -> sv_status {
                    if (!sweep_once(h, false, h->lam, d.size(), Gf, nullptr) ||
                        !sweep_once(h, true, h->CLbuf, d.size(), Gr, h->partials))
                        return fail(h, SV_ERR_CUDA, "autotune: whole-sweep launch refused");
                    return SV_OK;
                });
            } else if (h->storage == 1) {
                const uint32_t *L = (const uint32_t *)h->lists.buf;
                const int *li = &h->lists.info[4 * k];
                const int G = sector_grid(h->Db, h->sm_count, b);
                t = time_best(h, e0, e1, [&]() -> sv_status {
                    SV_CUDA(h, launch_rotate_l(h->lam, h->dtype, L + li[0], li[1], L + li[2], li[3], h->Da, d[k].c,
                                               d[k].s, G, h->stream));
                    if (inter)
                        SV_CUDA(h, launch_adjoint_li(h->CLbuf, h->dtype, L + li[0], li[1], L + li[2], li[3], h->Da,
                                                     d[k].c, d[k].s, G, h->partials, h->stream));
                    else if (adj)
                        SV_CUDA(h, launch_adjoint_l(h->lam, h->saved, h->dtype, L + li[0], li[1], L + li[2], li[3],
                                                    h->Da, d[k].c, d[k].s, G, h->partials, h->stream));
                    return SV_OK;
                });
            } else {
                // the adjoint step as sv_energy_grad runs it: interleaved in the pair buffer
                // (its two halves hold copies of psi, read here as interleaved pairs) or not
                const bool dint = h->lam_pair && h->rev_inter && h->ckpt_interval <= 0;
                const int G = rotate_grid(1ull << (h->n - 2), h->sm_count, b);
                t = time_best(h, e0, e1, [&]() -> sv_status {
                    SV_CUDA(h, launch_rotate(h->lam, h->dtype, h->n, d[k], h->sm_count, b, h->stream));
                    if (dint) SV_CUDA(h, launch_adjoint_i(h->lam, h->dtype, h->n, d[k], G, h->partials, h->stream));
                    else if (adj)
                        SV_CUDA(h, launch_adjoint(h->lam, h->saved, h->dtype, h->n, d[k], G, h->partials, h->stream));
                    return SV_OK;
                });
            }
            if (t < 0.f) return fail(h, SV_ERR_CUDA, "autotune: rotation candidate failed");
            if (best_t < 0.f || t < best_t) {
                best_t = t;
                best_b = b;
            }
        }
        if (sweeps && inter) h->sweep_bps = best_b;
        else if (h->storage == 1) h->sect_bps = best_b;
        else h->rot_bps = best_b;
    }
    // 3. 1-RDM launch geometry
    {
        SV_TRY(ensure_rdm_lists(h));
        const void *Cm = h->psi;
        if (h->storage == 0) {
            SV_CUDA(h, launch_compact(h->psi, h->Cbuf, h->dtype, h->str_sa_s, h->str_sb_s, h->Da, h->Db, h->sm_count,
                                      h->stream));
            Cm = h->Cbuf;
        }
        const int n_el = rdm_rows_elements(h->n);
        const int cands[] = {2, 4, 8, 16};
        SV_TRY(ensure_partials(h, (size_t)2 * n_el * rdm_rows_grid(h->Db, h->sm_count, 16)));
        const void *src = nullptr;
        int ff_form = 0;
        SV_TRY(rdm_input(h, Cm, &src, &ff_form));
        int best_b = 4;
        float best_t = -1.f;
        for (int b : cands) {
            const int grid = rdm_rows_grid(h->Db, h->sm_count, b);
            const float t = time_best(h, e0, e1, [&]() -> sv_status {
                SV_CUDA(h, launch_rdm_rows(src, h->dtype, ff_form, h->n, h->str_sa, h->str_sb, h->str_a, h->str_b,
                                           h->rank_a, h->rank_b, h->Da, h->Db, grid, (const uint32_t *)h->rdm_lists.buf,
                                           h->rdm_lists.dinfo, h->partials, h->stream));
                return SV_OK;
            });
            if (t < 0.f) return fail(h, SV_ERR_CUDA, "autotune: 1-RDM candidate failed");
            if (best_t < 0.f || t < best_t) {
                best_t = t;
                best_b = b;
            }
        }
        h->rdm_bps = best_b;
    }
    SV_CUDA(h, cudaStreamSynchronize(h->stream));
    return SV_OK;
}

// ---------------------------------------------------------------- C-ABI

extern "C" {

const char *sv_version(void) { return "sv-gb300 0.1 (sm_103a)"; }

uint32_t sv_check_status(void) {
    const uint32_t a = check_word_sector(), b = check_word_rows(), c = check_word_abtc(), d = check_word_pool();
    return (a & 0xFFu) | ((b & 0xFFu) << 8) | ((c & 0xFFu) << 16) | ((d & 0x0Fu) << 24) |
           ((a | b | c | d) & 0x80000000u);
}

const char *sv_last_error(sv_handle h) { return h ? h->err.c_str() : g_err.c_str(); }

uint64_t sv_launch_count(sv_handle h) { return h ? h->launches : 0; }

static uint64_t binom(int n, int k) {
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

// sect_na < 0: dense storage; otherwise sector storage of (sect_na, sect_nb).
static sv_status create_common(int n_qubits, sv_dtype dtype, void *cuda_stream, void *psi_dev, void *lam_dev,
                               sv_handle *out, int sect_na = -1, int sect_nb = -1) {
    if (!out) return fail(nullptr, SV_ERR_ARG, "NULL output handle pointer");
    *out = nullptr;
    if (n_qubits < 2 || n_qubits > SV_MAX_QUBITS || (n_qubits & 1))
        return fail(nullptr, SV_ERR_ARG, "n_qubits must be even and in [2, 32]");
    if (dtype != SV_C64 && dtype != SV_C128 && dtype != SV_R32 && dtype != SV_R64)
        return fail(nullptr, SV_ERR_ARG, "dtype must be SV_C64, SV_C128, SV_R32 or SV_R64");
    if ((psi_dev && ((uintptr_t)psi_dev & 255)) || (lam_dev && ((uintptr_t)lam_dev & 255)))
        return fail(nullptr, SV_ERR_ARG, "device buffers must be 256-byte aligned");
    sv_handle h = new sv_ctx();
    h->n = n_qubits;
    h->dtype = dtype;
    h->stream = (cudaStream_t)cuda_stream;
    h->dim = 1ull << n_qubits;
    h->elems = h->dim;
    if (sect_na >= 0) {
        h->storage = 1;
        h->na = sect_na;
        h->nb = sect_nb;
        h->elems = binom(n_qubits / 2, sect_na) * binom(n_qubits / 2, sect_nb);
        h->layout_auto = false;
    }
    h->amp_bytes = amp_size(dtype);
    for (int q = 0; q < 32; ++q) h->perm[q] = q;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(nullptr, SV_ERR_CUDA, "no CUDA device");
    }
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (cudaDeviceGetAttribute(&h->l2_bytes, cudaDevAttrL2CacheSize, h->device) != cudaSuccess) {
        cudaGetLastError();
        h->l2_bytes = 0;
    }
    if (psi_dev) {
        h->psi = psi_dev;
        h->own_psi = false;
    } else {
        sv_status s = dev_alloc(h, &h->psi, vec_bytes(h), "state vector");
        if (s != SV_OK) {
            delete h;
            return s;
        }
    }
    if (lam_dev) {
        h->lam = lam_dev;
        h->own_lam = false;
    }
    *out = h;
    return SV_OK;
}

sv_status sv_create(int n_qubits, sv_dtype dtype, void *cuda_stream, sv_handle *out) {
    return create_common(n_qubits, dtype, cuda_stream, nullptr, nullptr, out);
}

sv_status sv_create_sector(int n_qubits, int n_alpha, int n_beta, sv_dtype dtype, void *cuda_stream, sv_handle *out) {
    if (out) *out = nullptr;
    if (n_qubits < 2 || n_qubits > SV_MAX_QUBITS || (n_qubits & 1))
        return fail(nullptr, SV_ERR_ARG, "n_qubits must be even and in [2, 32]");
    const int N = n_qubits / 2;
    if (n_alpha < 0 || n_beta < 0 || n_alpha > N || n_beta > N)
        return fail(nullptr, SV_ERR_ARG, "electron counts must be in [0, n_qubits / 2]");
    return create_common(n_qubits, dtype, cuda_stream, nullptr, nullptr, out, n_alpha, n_beta);
}

sv_status sv_create_with_buffers(int n_qubits, sv_dtype dtype, void *cuda_stream, void *psi_dev, void *lam_dev,
                                 sv_handle *out) {
    if (!psi_dev) return fail(nullptr, SV_ERR_ARG, "psi_dev is required");
    return create_common(n_qubits, dtype, cuda_stream, psi_dev, lam_dev, out);
}

sv_status sv_destroy(sv_handle h) {
    if (!h) return SV_OK;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    cudaGetLastError();
    if (h->own_psi) dev_free(h, h->psi, vec_bytes(h));
    if (h->own_lam) dev_free(h, h->lam, h->lam_pair ? 2 * vec_bytes(h) : vec_bytes(h));
    dev_free(h, h->ref_vec, vec_bytes(h));
    if (!h->lam_pair) dev_free(h, h->saved, vec_bytes(h));
    for (void *p : h->ckpt) dev_free(h, p, vec_bytes(h));
    dev_free(h, h->sector, h->sector_len * sizeof(uint32_t));
    for (void *p : {(void *)h->str_sa, (void *)h->str_sb, (void *)h->str_sa_s, (void *)h->str_sb_s,
                    (void *)h->str_a, (void *)h->str_b, (void *)h->rank_a, (void *)h->rank_b})
        if (p) cudaFree(p);
    dev_free(h, h->Cbuf, h->Cbuf_bytes);
    dev_free(h, h->Lbuf, h->Lbuf_bytes);
    dev_free(h, h->sg_mats, h->sg_mats_bytes);
    dev_free(h, h->sg_buf, h->sg_buf_bytes);
    dev_free(h, h->ab_H, h->ab_H_bytes);
    dev_free(h, h->kerr, 16);
    if (h->hkerr) cudaFreeHost(h->hkerr);
    dev_free(h, h->lists.buf, h->lists.bytes);
    dev_free(h, h->pool_lists.buf, h->pool_lists.bytes);
    dev_free(h, h->rdm_lists.buf, h->rdm_lists.bytes);
    dev_free(h, h->CLbuf, h->CLbuf_bytes);
    dev_free(h, h->sweep_buf, h->sweep_bytes);
    dev_free(h, h->ffbuf, h->ffbuf_bytes);
    dev_free(h, h->partials, h->partials_cap * sizeof(double));
    dev_free(h, h->dout, h->dout_cap * sizeof(double));
    if (h->hpinned) cudaFreeHost(h->hpinned);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : h->tcev)
        if (e) cudaEventDestroy(e);
    delete h;
    return SV_OK;
}


sv_status sv_prepare_hf(sv_handle h, const int32_t *occ, int n_occ) {
    if (!h) return fail(nullptr, SV_ERR_ARG, "NULL handle");
    if (n_occ < 0 || n_occ > h->n || (n_occ > 0 && !occ)) return fail(h, SV_ERR_ARG, "bad occupation list");
    uint32_t x = 0;
    int na = 0, nb = 0;
    for (int k = 0; k < n_occ; ++k) {
        int j = occ[k];
        if (j < 0 || j >= h->n) return fail(h, SV_ERR_ARG, "occupied index out of range");
        if ((x >> j) & 1u) return fail(h, SV_ERR_ARG, "repeated occupied index");
        x |= 1u << j;
        if (j & 1) ++nb; else ++na;
    }
    if (h->storage == 1 && (na != h->na || nb != h->nb))
        return fail(h, SV_ERR_ARG, "determinant outside the handle's (n_alpha, n_beta) sector");
    DeviceGuard g(h->device);
    h->failed = false;
    h->prepared = false;
    h->ref_kind = 1;
    h->ref_det = x;
    h->na = na;
    h->nb = nb;
    SV_TRY(prepare_reference(h));
    h->prepared = true;
    h->at_ref = true;
    return SV_OK;
}

sv_status sv_prepare_state(sv_handle h, const void *amplitudes_host, int n_alpha, int n_beta) {
    if (!h) return fail(nullptr, SV_ERR_ARG, "NULL handle");
    if (!amplitudes_host) return fail(h, SV_ERR_ARG, "NULL amplitudes");
    const int N = h->n / 2;
    if (n_alpha < 0 || n_beta < 0 || n_alpha > N || n_beta > N) return fail(h, SV_ERR_ARG, "bad electron counts");
    if (h->storage == 1 && (n_alpha != h->na || n_beta != h->nb))
        return fail(h, SV_ERR_ARG, "electron counts differ from the handle's sector");
    const uint32_t even = 0x55555555u, odd = 0xAAAAAAAAu;
    double best = -1.0;
    uint32_t best_x = 0;
    for (uint64_t x = 0; x < h->dim; ++x) {
        double re = 0.0, im = 0.0;
        switch (h->dtype) {
            case SV_C64: re = ((const float *)amplitudes_host)[2 * x]; im = ((const float *)amplitudes_host)[2 * x + 1]; break;
            case SV_C128: re = ((const double *)amplitudes_host)[2 * x]; im = ((const double *)amplitudes_host)[2 * x + 1]; break;
            case SV_R32: re = ((const float *)amplitudes_host)[x]; break;
            default: re = ((const double *)amplitudes_host)[x]; break;
        }
        if (!std::isfinite(re) || !std::isfinite(im)) return fail(h, SV_ERR_ARG, "non-finite amplitude");
        double w = re * re + im * im;
        if (w == 0.0) continue;
        if (__builtin_popcount((uint32_t)x & even) != n_alpha || __builtin_popcount((uint32_t)x & odd) != n_beta)
            return fail(h, SV_ERR_ARG, "amplitude outside the (n_alpha, n_beta) sector");
        if (w > best) { best = w; best_x = (uint32_t)x; }
    }
    if (best <= 0.0) return fail(h, SV_ERR_ARG, "zero state");
    DeviceGuard g(h->device);
    h->failed = false;
    h->prepared = false;
    h->at_ref = false;
    if (!h->ref_vec) SV_TRY(dev_alloc(h, &h->ref_vec, vec_bytes(h), "reference copy"));
    if (h->storage == 1) {
        // host order is the dense qubit-order vector: keep its sector entries in C[rank(b)][rank(a)] order
        SV_TRY(ensure_strings(h));
        std::vector<uint8_t> comp(vec_bytes(h));
        for (int Ib = 0; Ib < h->Db; ++Ib)
            for (int Ia = 0; Ia < h->Da; ++Ia) {
                uint64_t x = 0;
                for (int p = 0; p < N; ++p) {
                    x |= (uint64_t)((h->h_stra[Ia] >> p) & 1u) << (2 * p);
                    x |= (uint64_t)((h->h_strb[Ib] >> p) & 1u) << (2 * p + 1);
                }
                memcpy(comp.data() + ((size_t)Ib * h->Da + Ia) * h->amp_bytes,
                       (const uint8_t *)amplitudes_host + x * h->amp_bytes, h->amp_bytes);
            }
        SV_CUDA(h, cudaMemcpyAsync(h->ref_vec, comp.data(), comp.size(), cudaMemcpyHostToDevice, h->stream));
    } else if (is_identity(h)) {
        SV_CUDA(h, cudaMemcpyAsync(h->ref_vec, amplitudes_host, vec_bytes(h), cudaMemcpyHostToDevice, h->stream));
    } else {
        // host order is qubit order: upload to the scratch vector, then move bit q to bit perm[q]
        SV_TRY(ensure_lam(h));
        SV_CUDA(h, cudaMemcpyAsync(h->lam, amplitudes_host, vec_bytes(h), cudaMemcpyHostToDevice, h->stream));
        SV_CUDA(h, launch_permute(h->lam, h->ref_vec, h->dtype, h->n, h->perm, h->sm_count, h->stream));
        h->launches++;
    }
    SV_CUDA(h, cudaStreamSynchronize(h->stream));
    h->ref_kind = 2;
    h->ref_det = best_x;
    h->na = n_alpha;
    h->nb = n_beta;
    SV_TRY(prepare_reference(h));
    h->prepared = true;
    return SV_OK;
}

sv_status sv_get_state(sv_handle h, void *amplitudes_host) {
    SV_TRY(check_ready(h));
    if (!amplitudes_host) return fail(h, SV_ERR_ARG, "NULL output");
    DeviceGuard g(h->device);
    if (h->storage == 1) {
        // compact matrix back to the host, scattered into the dense qubit-order vector
        SV_TRY(ensure_strings(h));
        std::vector<uint8_t> comp(vec_bytes(h));
        SV_CUDA(h, cudaMemcpyAsync(comp.data(), h->psi, comp.size(), cudaMemcpyDeviceToHost, h->stream));
        SV_CUDA(h, cudaStreamSynchronize(h->stream));
        memset(amplitudes_host, 0, (size_t)h->dim * h->amp_bytes);
        const int N = h->n / 2;
        for (int Ib = 0; Ib < h->Db; ++Ib)
            for (int Ia = 0; Ia < h->Da; ++Ia) {
                uint64_t x = 0;
                for (int p = 0; p < N; ++p) {
                    x |= (uint64_t)((h->h_stra[Ia] >> p) & 1u) << (2 * p);
                    x |= (uint64_t)((h->h_strb[Ib] >> p) & 1u) << (2 * p + 1);
                }
                memcpy((uint8_t *)amplitudes_host + x * h->amp_bytes,
                       comp.data() + ((size_t)Ib * h->Da + Ia) * h->amp_bytes, h->amp_bytes);
            }
        return SV_OK;
    }
    const void *src = h->psi;
    if (!is_identity(h)) {
        // back to qubit order through the scratch vector
        int inv[32];
        for (int q = 0; q < h->n; ++q) inv[h->perm[q]] = q;
        SV_TRY(ensure_lam(h));
        SV_CUDA(h, launch_permute(h->psi, h->lam, h->dtype, h->n, inv, h->sm_count, h->stream));
        h->launches++;
        src = h->lam;
    }
    SV_CUDA(h, cudaMemcpyAsync(amplitudes_host, src, vec_bytes(h), cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(h, cudaStreamSynchronize(h->stream));
    return SV_OK;
}

sv_status sv_get_amplitudes(sv_handle h, const uint64_t *basis, int count, void *amplitudes_host) {
    SV_TRY(check_ready(h));
    if (count < 0 || (count > 0 && (!basis || !amplitudes_host))) return fail(h, SV_ERR_ARG, "bad arguments");
    if (count == 0) return SV_OK;
    for (int i = 0; i < count; ++i)
        if (basis[i] >= h->dim) return fail(h, SV_ERR_ARG, "basis index out of range");
    DeviceGuard g(h->device);
    std::vector<uint32_t> addr(count);
    if (h->storage == 1) SV_TRY(ensure_strings(h));
    for (int i = 0; i < count; ++i)
        addr[i] = h->storage == 1 ? compact_index(h, basis[i]) : map_bits((uint32_t)basis[i], h->perm);
    // scratch: the addresses, then the gathered amplitudes, in the reduction buffer
    const size_t addr_doubles = ((size_t)count * 4 + 7) / 8;
    const size_t out_off = (addr_doubles + 1) / 2 * 2;  // 16-byte aligned for complex128
    const size_t amp_doubles = ((size_t)count * h->amp_bytes + 7) / 8;
    SV_TRY(ensure_partials(h, out_off + amp_doubles));
    uint32_t *d_addr = (uint32_t *)h->partials;
    void *d_out = h->partials + out_off;
    SV_CUDA(h, cudaMemcpyAsync(d_addr, addr.data(), (size_t)count * 4, cudaMemcpyHostToDevice, h->stream));
    if (h->storage == 1) SV_CUDA(h, launch_gather_c(h->psi, h->dtype, d_addr, count, d_out, h->stream));
    else SV_CUDA(h, launch_gather(h->psi, h->dtype, d_addr, count, d_out, h->stream));
    h->launches++;
    SV_CUDA(h, cudaMemcpyAsync(amplitudes_host, d_out, (size_t)count * h->amp_bytes, cudaMemcpyDeviceToHost,
                               h->stream));
    SV_CUDA(h, cudaStreamSynchronize(h->stream));
    return SV_OK;
}

sv_status sv_state_device_ptr(sv_handle h, void **psi_dev) {
    if (!h || !psi_dev) return fail(h, SV_ERR_ARG, "NULL argument");
    h->at_ref = false;  // the caller may write the state through the pointer
    *psi_dev = h->psi;
    return SV_OK;
}

sv_status sv_ham_create(int n_orb, const double *hmat, const double *eri, double e_nuc, sv_ham_handle *out) {
    if (!out) return fail(nullptr, SV_ERR_ARG, "NULL output handle pointer");
    *out = nullptr;
    if (n_orb < 1 || n_orb > SV_MAX_QUBITS / 2) return fail(nullptr, SV_ERR_ARG, "n_orb must be in [1, 16]");
    if (!hmat || !eri) return fail(nullptr, SV_ERR_ARG, "NULL integrals");
    if (!std::isfinite(e_nuc)) return fail(nullptr, SV_ERR_ARG, "non-finite e_nuc");
    const int N = n_orb;
    auto tol = [](double a, double b) { return std::fabs(a - b) <= 1e-12 * std::max(1.0, std::fabs(a)); };
    for (int p = 0; p < N; ++p)
        for (int q = 0; q < N; ++q) {
            double v = hmat[p * N + q];
            if (!std::isfinite(v)) return fail(nullptr, SV_ERR_ARG, "non-finite h");
            if (!tol(v, hmat[q * N + p])) return fail(nullptr, SV_ERR_ARG, "h is not symmetric");
        }
    auto E = [&](int p, int q, int r, int s) { return eri[(((size_t)p * N + q) * N + r) * N + s]; };
    for (int p = 0; p < N; ++p)
        for (int q = 0; q < N; ++q)
            for (int r = 0; r < N; ++r)
                for (int s = 0; s < N; ++s) {
                    double v = E(p, q, r, s);
                    if (!std::isfinite(v)) return fail(nullptr, SV_ERR_ARG, "non-finite eri");
                    if (!tol(v, E(q, p, r, s)) || !tol(v, E(p, q, s, r)) || !tol(v, E(r, s, p, q)))
                        return fail(nullptr, SV_ERR_ARG, "eri lacks the 8-fold symmetry of real orbitals");
                }
    sv_ham_handle H = new sv_ham();
    H->n_orb = N;
    H->e_nuc = e_nuc;
    H->h.assign(hmat, hmat + (size_t)N * N);
    H->eri.assign(eri, eri + (size_t)N * N * N * N);
    *out = H;
    return SV_OK;
}

sv_status sv_ham_destroy(sv_ham_handle ham) {
    if (!ham) return SV_OK;
    ham->dev.clear();
    delete ham;
    return SV_OK;
}

sv_status sv_apply_ansatz(sv_handle h, const sv_excitation *ops, int n_ops, const double *theta) {
    SV_TRY(check_ready(h));
    std::vector<OpDesc> d;
    SV_TRY(build_ops(h, ops, n_ops, theta, d));
    DeviceGuard g(h->device);
    L2FetchScope l2(h);
    if (h->layout_auto && n_ops > 0 && h->storage == 0 && h->at_ref && h->ref_kind == 1) {
        // the state is still the HF determinant: take the layout the operator list prefers
        // (as sv_energy_grad does) by writing the determinant anew in it, one store
        int np[32];
        layout_from_ops(h->n, ops, n_ops, np);
        bool same = true;
        for (int q = 0; q < h->n; ++q) same = same && np[q] == h->perm[q];
        if (!same) {
            for (int q = 0; q < 32; ++q) h->perm[q] = q < h->n ? np[q] : q;
            drop_layout_caches(h);
            SV_TRY(prepare_reference(h));
            SV_TRY(build_ops(h, ops, n_ops, theta, d));
        }
    }
    h->at_ref = false;
    SV_TRY(forward(h, d, false));
    return SV_OK;
}

sv_status sv_energy(sv_handle h, sv_ham_handle ham, double *e_out) {
    SV_TRY(check_ready(h));
    SV_TRY(check_ham(h, ham));
    if (!e_out) return fail(h, SV_ERR_ARG, "NULL e_out");
    DeviceGuard g(h->device);
    DevTables *T;
    SV_TRY(get_tables(h, ham, &T));
    SV_TRY(ensure_out(h, 2));
    const double c = shift_for(h, ham);
    SV_TRY(expectation(h, ham, T, nullptr, c, 0));
    SV_CUDA(h, cudaMemcpyAsync(h->hpinned, h->dout, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(h, cudaStreamSynchronize(h->stream));
    SV_TRY(check_kernel_flag(h));
    *e_out = c + h->hpinned[0] / h->hpinned[1];
    return SV_OK;
}

sv_status sv_energy_grad(sv_handle h, sv_ham_handle ham, const sv_excitation *ops, int n_ops, const double *theta,
                         double *e_out, double *grad_out) {
    if (!h) return fail(nullptr, SV_ERR_ARG, "NULL handle");
    if (h->ref_kind == 0) return fail(h, SV_ERR_STATE, "no reference state recorded");
    SV_TRY(check_ham(h, ham));
    std::vector<OpDesc> d;
    SV_TRY(build_ops(h, ops, n_ops, theta, d));  // validates in any layout
    h->at_ref = false;
    DeviceGuard g(h->device);
    L2FetchScope l2(h);
    NvtxClose nvtx_close{h};
    if (h->layout_auto && n_ops > 0 && h->storage == 0) {
        int np[32];
        layout_from_ops(h->n, ops, n_ops, np);
        SV_TRY(relayout(h, np));
        SV_TRY(build_ops(h, ops, n_ops, theta, d));
    }
    const size_t L = d.size();
    DevTables *T;
    SV_TRY(get_tables(h, ham, &T));
    SV_TRY(ensure_lam(h));
    SV_TRY(ensure_out(h, 2 + L));
    // state buffers first (so the byte cap drops checkpoints, not required scratch)
    if (!h->saved) {
        void *p = nullptr;
        if (dev_alloc(h, &p, vec_bytes(h), "saved final state") == SV_OK) h->saved = p;
        else cudaGetLastError();
    }
    const bool sect = h->storage == 1;
    if (sect) SV_TRY(ensure_strings(h));
    const int G = sect ? sector_grid(h->Db, h->sm_count, h->sect_bps)
                       : rotate_grid(1ull << (h->n - 2), h->sm_count, h->rot_bps);
    size_t need = 0;
    if (sect) {
        need = 3 * (size_t)h->Db;
    } else if (h->expect_variant == 1 && is_complex(h->dtype)) {
        SV_TRY(ensure_sector(h));
        need = 2 * (size_t)expect_gather_grid(h->sector_len, h->sm_count);
    } else {
        SV_TRY(ensure_strings(h));
        need = 3 * (size_t)h->Db;
    }
    SV_TRY(ensure_partials(h, std::max<size_t>((size_t)G * std::max<size_t>(L, 1), need)));
    plan_checkpoints(h, L);
    h->prepared = false;
    h->tc_timed = 0;
    SV_TRY(mark(h, 0, "sv_energy_grad: reference"));
    SV_TRY(prepare_reference(h));
    h->prepared = true;
    SV_TRY(mark(h, 1, "sv_energy_grad: forward sweep"));
    SV_TRY(forward(h, d, true));
    SV_TRY(mark(h, 2, "sv_energy_grad: working copy"));
    // The reverse sweep un-applies the ops to a working copy of psi(theta), so that psi
    // keeps psi(theta): in sector storage without checkpoint resynchronisation, the
    // interleaved (psi, lambda) matrix; else the saved-state buffer.  Where neither can be
    // allocated under the byte cap, the sweep runs on psi and psi(theta) is recomputed.
    const int64_t C = h->ckpt_interval;
    bool inter = sect && C <= 0 && L > 0;
    if (inter && ensure_clbuf(h) != SV_OK) {
        cudaGetLastError();
        inter = false;
    }
    // dense storage: psi(theta) and lambda interleaved by amplitude in the adjoint pair
    // buffer (k_adjoint_i), where it exists, checkpoints do not resynchronise the working
    // copy and sigma comes from the string-row forms (compact, then scattered)
    bool dint = !sect && C <= 0 && L > 0 && h->lam_pair && h->rev_inter &&
                !(h->expect_variant == 1 && is_complex(h->dtype));
    if (dint && ensure_lbuf(h) != SV_OK) {
        cudaGetLastError();
        dint = false;
    }
    void *wpsi = (!inter && !dint && h->saved) ? h->saved : h->psi;
    if (wpsi != h->psi)
        SV_CUDA(h, cudaMemcpyAsync(wpsi, h->psi, vec_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
    if (dint) {  // lam[2x] = psi[x], lam[2x + 1] = 0: the copy and the zeroing of lambda in one pass
        SV_CUDA(h, launch_interleave_zero(h->psi, h->lam, h->dtype, h->n, h->sm_count, h->stream));
        h->launches++;
    }
    const double c = shift_for(h, ham);
    SV_TRY(mark(h, 3, "sv_energy_grad: expectation"));
    if (dint) {
        SV_TRY(expectation(h, ham, T, nullptr, c, 0, h->Lbuf));
        SV_CUDA(h, launch_scatter_odd(h->Lbuf, h->lam, h->dtype, h->str_sa_s, h->str_sb_s, h->Da, h->Db, h->sm_count,
                                      h->stream));
        h->launches++;
    } else {
        SV_TRY(expectation(h, ham, T, h->lam, c, 0));
    }
    SV_TRY(mark(h, 4, "sv_energy_grad: reverse sweep"));
    // reverse sweep
    if (inter) {
        SV_CUDA(h, launch_interleave(h->psi, h->lam, h->dtype, h->CLbuf, (size_t)h->Da * h->Db, h->sm_count,
                                     h->stream));
        h->launches++;
    }
    // sector storage: the reverse sweep in one launch where it can (gradient partials
    // [L][Gs], Gs its grid), else one launch per op ([L][G])
    int Gred = G;
    bool swept = false;
    if (inter) {
        const int Gs = sweep_grid(h->dtype, true, h->Db, h->sm_count, h->sweep_bps);
        if (Gs > 0 && Gs <= G && sweep_once(h, true, h->CLbuf, L, Gs, h->partials)) {
            swept = true;
            Gred = Gs;
        }
    }
    for (size_t kk = swept ? 0 : L; kk-- > 0;) {
        if (inter) {
            const uint32_t *LB = (const uint32_t *)h->lists.buf;
            const int *li = &h->lists.info[4 * kk];
            SV_CUDA(h, launch_adjoint_li(h->CLbuf, h->dtype, LB + li[0], li[1], LB + li[2], li[3], h->Da, d[kk].c,
                                         d[kk].s, G, h->partials + kk * (size_t)G, h->stream));
        } else if (sect) {
            const uint32_t *LB = (const uint32_t *)h->lists.buf;
            const int *li = &h->lists.info[4 * kk];
            SV_CUDA(h, launch_adjoint_l(wpsi, h->lam, h->dtype, LB + li[0], li[1], LB + li[2], li[3], h->Da,
                                        d[kk].c, d[kk].s, G, h->partials + kk * (size_t)G, h->stream));
        } else if (dint) {
            SV_CUDA(h, launch_adjoint_i(h->lam, h->dtype, h->n, d[kk], G, h->partials + kk * (size_t)G, h->stream));
        } else {
            SV_CUDA(h, launch_adjoint(wpsi, h->lam, h->dtype, h->n, d[kk], G, h->partials + kk * (size_t)G,
                                      h->stream));
        }
        h->launches++;
        // the working copy now holds the state after ops[0..kk-1]; resynchronise it from a
        // checkpoint if one holds it
        if (!inter && !dint && C > 0 && kk > 0 && kk % (size_t)C == 0) {
            size_t j = kk / (size_t)C - 1;
            if (j < h->ckpt.size() && h->ckpt[j])
                SV_CUDA(h, cudaMemcpyAsync(wpsi, h->ckpt[j], vec_bytes(h), cudaMemcpyDeviceToDevice, h->stream));
        }
    }
    SV_CUDA(h, launch_reduce_rows(h->partials, (int)L, Gred, h->dout + 2, h->stream));
    h->launches++;
    SV_TRY(mark(h, 5, "sv_energy_grad: restore"));
    SV_CUDA(h, cudaMemcpyAsync(h->hpinned, h->dout, (2 + L) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    // leave psi(theta) in the handle (only a sweep on psi itself took it away)
    if (!inter && !dint && wpsi == h->psi) {
        SV_TRY(prepare_reference(h));
        SV_TRY(forward(h, d, false));
    }
    SV_TRY(mark(h, 6, nullptr));
    SV_CUDA(h, cudaStreamSynchronize(h->stream));
    SV_TRY(check_kernel_flag(h));
    if (h->profile) {
        h->phase_ms[0] = elapsed(h, 0, 1);
        h->phase_ms[1] = elapsed(h, 1, 2);
        h->phase_ms[2] = elapsed(h, 3, 4);
        h->phase_ms[3] = elapsed(h, 4, 5);
        h->phase_ms[4] = elapsed(h, 5, 6);
        h->phase_ms[6] = (h->tc_timed & 1) ? elapsed_ev(h->tcev[0], h->tcev[1]) : 0.0;
        h->phase_ms[7] = (h->tc_timed & 2) ? elapsed_ev(h->tcev[2], h->tcev[3]) : 0.0;
    }
    const double nrm = h->hpinned[1];
    if (e_out) *e_out = c + h->hpinned[0] / nrm;
    if (grad_out)
        for (size_t k = 0; k < L; ++k) grad_out[k] = 2.0 * h->hpinned[2 + k] / nrm;
    return SV_OK;
}

sv_status sv_pool_gradients(sv_handle h, sv_ham_handle ham, const sv_excitation *pool, int n_pool, double *e_out,
                            double *grad_out) {
    SV_TRY(check_ready(h));
    SV_TRY(check_ham(h, ham));
    if (n_pool < 0 || (n_pool > 0 && (!pool || !grad_out))) return fail(h, SV_ERR_ARG, "bad pool arguments");
    const int ident[32] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15,
                           16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31};
    const bool use_lists = h->pool_variant != 1;
    const size_t ob = pool_op_bytes();
    std::vector<uint8_t> host_ops(use_lists ? 0 : (size_t)n_pool * ob);
    std::vector<OpDesc> descs;
    descs.reserve(n_pool);
    for (int k = 0; k < n_pool; ++k) {
        OpDesc d;
        std::string why;
        if (!make_op(pool[k], h->n, ident, d, why)) {
            char buf[64];
            snprintf(buf, sizeof buf, "pool op %d: ", k);
            return fail(h, SV_ERR_ARG, buf + why);
        }
        if (use_lists) descs.push_back(d);
        else pool_op_from(d, h->n / 2, host_ops.data() + (size_t)k * ob);
    }
    DeviceGuard g(h->device);
    DevTables *T;
    SV_TRY(get_tables(h, ham, &T));
    SV_TRY(ensure_strings(h));
    SV_TRY(ensure_lbuf(h));
    if (use_lists && n_pool > 0) {
        SV_TRY(ensure_op_lists(h, descs, h->pool_lists));
        SV_TRY(ensure_clbuf(h));
    }
    const size_t op_doubles = ((size_t)host_ops.size() + 7) / 8;
    SV_TRY(ensure_partials(h, 3 * (size_t)h->Db + op_doubles));
    SV_TRY(ensure_out(h, 2 + (size_t)n_pool));
    const double c = shift_for(h, ham);
    const void *Cm = h->storage == 1 ? h->psi : h->Cbuf;  // compact amplitudes
    if (h->storage == 0) {
        SV_CUDA(h, launch_compact(h->psi, h->Cbuf, h->dtype, h->str_sa_s, h->str_sb_s, h->Da, h->Db, h->sm_count,
                                  h->stream));
        h->launches++;
    }
    RowTables R{h->str_sa, h->str_sb, h->str_sa_s, h->str_sb_s, h->str_a, h->str_b, h->rank_a, h->rank_b,
                T->eri_r, T->hm_r, T->Dt, T->Jt, h->n / 2, h->Da, h->Db, T->W2};
    SV_TRY(sigma_rows(h, T, R, Cm, nullptr, h->Lbuf, ham->e_nuc - c));
    SV_CUDA(h, launch_reduce_rows(h->partials, 2, h->Db, h->dout, h->stream));
    h->launches++;
    if (n_pool > 0 && use_lists) {
        SV_CUDA(h, launch_interleave(Cm, h->Lbuf, h->dtype, h->CLbuf, (size_t)h->Da * h->Db, h->sm_count,
                                     h->stream));
        SV_CUDA(h, launch_pool_grad_l(h->CLbuf, h->dtype, (const uint32_t *)h->pool_lists.buf, h->pool_lists.dinfo,
                                      n_pool, h->Da, h->Db, h->dout + 2, h->stream));
        h->launches += 2;
    } else if (n_pool > 0) {
        void *d_ops = h->partials + 3 * (size_t)h->Db;
        SV_CUDA(h, cudaMemcpyAsync(d_ops, host_ops.data(), host_ops.size(), cudaMemcpyHostToDevice, h->stream));
        SV_CUDA(h, launch_pool_grad(Cm, h->Lbuf, h->dtype, d_ops, n_pool, h->str_sa, h->str_sb, h->str_a,
                                    h->str_b, h->rank_a, h->rank_b, h->Da, h->Db, h->dout + 2, h->stream));
        h->launches++;
    }
    SV_CUDA(h, cudaMemcpyAsync(h->hpinned, h->dout, (2 + (size_t)n_pool) * sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream));
    SV_CUDA(h, cudaStreamSynchronize(h->stream));
    SV_TRY(check_kernel_flag(h));
    const double nrm = h->hpinned[1];
    if (e_out) *e_out = c + h->hpinned[0] / nrm;
    for (int k = 0; k < n_pool; ++k) grad_out[k] = 2.0 * h->hpinned[2 + k] / nrm;
    return SV_OK;
}

sv_status sv_rdm1(sv_handle h, double *re_out, double *im_out) {
    SV_TRY(check_ready(h));
    if (!re_out) return fail(h, SV_ERR_ARG, "NULL re_out");
    DeviceGuard g(h->device);
    NvtxClose nvtx_close{h};
    if (h->storage == 1 || h->rdm_variant != 1 || !is_complex(h->dtype)) {
        // string rows: on the state itself (sector storage) or on its compact copy
        SV_TRY(ensure_strings(h));
        SV_TRY(ensure_rdm_lists(h));
        const int n_el = rdm_rows_elements(h->n);
        const int grid = rdm_rows_grid(h->Db, h->sm_count, h->rdm_bps);
        SV_TRY(ensure_partials(h, (size_t)2 * n_el * grid));
        SV_TRY(ensure_out(h, 2 * (size_t)n_el));
        SV_TRY(mark(h, 0, "sv_rdm1"));
        const void *Cm = h->psi;
        if (h->storage == 0) {
            SV_CUDA(h, launch_compact(h->psi, h->Cbuf, h->dtype, h->str_sa_s, h->str_sb_s, h->Da, h->Db, h->sm_count,
                                      h->stream));
            h->launches++;
            Cm = h->Cbuf;
        }
        const void *src = nullptr;
        int ff_form = 0;
        SV_TRY(rdm_input(h, Cm, &src, &ff_form));
        SV_CUDA(h, launch_rdm_rows(src, h->dtype, ff_form, h->n, h->str_sa, h->str_sb, h->str_a, h->str_b, h->rank_a,
                                   h->rank_b, h->Da, h->Db, grid, (const uint32_t *)h->rdm_lists.buf,
                                   h->rdm_lists.dinfo, h->partials, h->stream));
        h->launches++;
        SV_CUDA(h, launch_reduce_rows(h->partials, 2 * n_el, grid, h->dout, h->stream));
        h->launches++;
        SV_TRY(mark(h, 7, nullptr));
        SV_CUDA(h, cudaMemcpyAsync(h->hpinned, h->dout, 2 * (size_t)n_el * sizeof(double), cudaMemcpyDeviceToHost,
                                   h->stream));
        SV_CUDA(h, cudaStreamSynchronize(h->stream));
    } else {
        SV_TRY(ensure_sector(h));
        // element list (host) -> device scratch after the partial sums
        std::vector<uint8_t> host_el;
        const int n_el = rdm_elements_bytes(h->n, h->perm, host_el);
        const int grid = rdm_gather_grid(h->sector_len, h->sm_count);
        const size_t part = (size_t)2 * n_el * grid;
        const size_t el_doubles = (host_el.size() + sizeof(double) - 1) / sizeof(double);
        SV_TRY(ensure_partials(h, part + el_doubles));
        SV_TRY(ensure_out(h, 2 * (size_t)n_el));
        double *d_el = h->partials + part;
        SV_CUDA(h, cudaMemcpyAsync(d_el, host_el.data(), host_el.size(), cudaMemcpyHostToDevice, h->stream));
        SV_TRY(mark(h, 0, "sv_rdm1"));
        SV_CUDA(h, launch_rdm_gather(h->psi, h->dtype, h->sector, h->sector_len, d_el, n_el, grid, h->partials,
                                     h->stream));
        h->launches++;
        SV_CUDA(h, launch_reduce_rows(h->partials, 2 * n_el, grid, h->dout, h->stream));
        h->launches++;
        SV_TRY(mark(h, 7, nullptr));
        SV_CUDA(h, cudaMemcpyAsync(h->hpinned, h->dout, 2 * (size_t)n_el * sizeof(double), cudaMemcpyDeviceToHost,
                                   h->stream));
        SV_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    if (h->profile) h->phase_ms[5] = elapsed(h, 0, 7);
    const int n = h->n, N = n / 2;
    const double *o = h->hpinned;
    const double nrm = o[0];
    for (int s = 0; s < 2; ++s)
        for (int p = 0; p < N; ++p) {
            re_out[(s * N + p) * N + p] = o[2 * (1 + 2 * p + s)] / nrm;
            if (im_out) im_out[(s * N + p) * N + p] = 0.0;
        }
    int e = 1 + n;
    for (int s = 0; s < 2; ++s)
        for (int p = 0; p < N; ++p)
            for (int q = p + 1; q < N; ++q, ++e) {
                double re = o[2 * e] / nrm, im = o[2 * e + 1] / nrm;
                re_out[(s * N + p) * N + q] = re;
                re_out[(s * N + q) * N + p] = re;
                if (im_out) {
                    im_out[(s * N + p) * N + q] = im;
                    im_out[(s * N + q) * N + p] = -im;
                }
            }
    return SV_OK;
}

sv_status sv_autotune(sv_handle h, sv_ham_handle ham, const sv_excitation *ops, int n_ops, const double *theta) {
    SV_TRY(check_ready(h));
    SV_TRY(check_ham(h, ham));
    std::vector<OpDesc> d;
    SV_TRY(build_ops(h, ops, n_ops, theta, d));
    DeviceGuard g(h->device);
    L2FetchScope l2(h);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SV_CUDA(h, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(e0);
        return fail(h, SV_ERR_CUDA, "autotune: event creation failed");
    }
    h->at_ref = false;
    const sv_status st = autotune_impl(h, ham, d, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

sv_status sv_get_option(sv_handle h, sv_option opt, int64_t *value) {
    if (!h || !value) return fail(h, SV_ERR_ARG, "NULL argument");
    switch (opt) {
        case SV_OPT_CHECKPOINT_INTERVAL: *value = h->ckpt_interval; return SV_OK;
        case SV_OPT_MAX_BYTES: *value = h->max_bytes; return SV_OK;
        case SV_OPT_EXPECT_VARIANT: *value = h->expect_variant; return SV_OK;
        case SV_OPT_RDM_VARIANT: *value = h->rdm_variant; return SV_OK;
        case SV_OPT_PROFILE: *value = h->profile ? 1 : 0; return SV_OK;
        case SV_OPT_LAYOUT_AUTO: *value = h->layout_auto ? 1 : 0; return SV_OK;
        case SV_OPT_AB_CHUNK: *value = h->ab_chunk; return SV_OK;
        case SV_OPT_ROT_BLOCKS_PER_SM: *value = h->rot_bps; return SV_OK;
        case SV_OPT_SECT_BLOCKS_PER_SM: *value = h->sect_bps; return SV_OK;
        case SV_OPT_RDM_BLOCKS_PER_SM: *value = h->rdm_bps; return SV_OK;
        case SV_OPT_POOL_VARIANT: *value = h->pool_variant; return SV_OK;
        case SV_OPT_L2_FETCH: *value = h->l2_fetch; return SV_OK;
        case SV_OPT_REVERSE_INTERLEAVED: *value = h->rev_inter; return SV_OK;
        case SV_OPT_WAIT_POLLS: *value = h->wait_polls; return SV_OK;
        case SV_OPT_SECTOR_SWEEP: *value = h->sweep_mode; return SV_OK;
        case SV_OPT_SWEEP_BLOCKS_PER_SM: *value = h->sweep_bps; return SV_OK;
        case SV_OPT_TEST_STALL: *value = h->test_stall; return SV_OK;
    }
    return fail(h, SV_ERR_ARG, "unknown option");
}

sv_status sv_set_layout(sv_handle h, const int32_t *storage_of_qubit) {
    if (!h || !storage_of_qubit) return fail(h, SV_ERR_ARG, "NULL argument");
    int np[32];
    uint32_t seen = 0;
    for (int q = 0; q < h->n; ++q) {
        int b = storage_of_qubit[q];
        if (b < 0 || b >= h->n || ((seen >> b) & 1u)) return fail(h, SV_ERR_ARG, "layout is not a permutation of [0, n)");
        seen |= 1u << b;
        np[q] = b;
    }
    if (h->storage == 1) {
        for (int q = 0; q < h->n; ++q)
            if (np[q] != q) return fail(h, SV_ERR_ARG, "sector storage has no address layout (identity only)");
        return SV_OK;
    }
    DeviceGuard g(h->device);
    h->layout_auto = false;
    return relayout(h, np);
}

sv_status sv_get_layout(sv_handle h, int32_t *storage_of_qubit) {
    if (!h || !storage_of_qubit) return fail(h, SV_ERR_ARG, "NULL argument");
    for (int q = 0; q < h->n; ++q) storage_of_qubit[q] = h->perm[q];
    return SV_OK;
}

sv_status sv_phase_times(sv_handle h, double *ms_out, int n_out) {
    if (!h || !ms_out || n_out < 0) return fail(h, SV_ERR_ARG, "bad arguments");
    for (int i = 0; i < n_out && i < SV_PHASES; ++i) ms_out[i] = h->phase_ms[i];
    return SV_OK;
}

sv_status sv_set_option(sv_handle h, sv_option opt, int64_t value) {
    if (!h) return fail(nullptr, SV_ERR_ARG, "NULL handle");
    switch (opt) {
        case SV_OPT_CHECKPOINT_INTERVAL:
            if (value < 0) return fail(h, SV_ERR_ARG, "checkpoint interval < 0");
            h->ckpt_interval = value;
            return SV_OK;
        case SV_OPT_MAX_BYTES:
            if (value < 0) return fail(h, SV_ERR_ARG, "max bytes < 0");
            h->max_bytes = value;
            return SV_OK;
        case SV_OPT_EXPECT_VARIANT:
            if (value < 0 || value > 6) return fail(h, SV_ERR_ARG, "expect variant must be 0 to 6");
            h->expect_variant = (int)value;
            return SV_OK;
        case SV_OPT_RDM_VARIANT:
            if (value < 0 || value > 3) return fail(h, SV_ERR_ARG, "rdm variant must be 0 to 3");
            h->rdm_variant = (int)value;
            return SV_OK;
        case SV_OPT_SWEEP_BLOCKS_PER_SM:
            if (value < 1 || value > 64) return fail(h, SV_ERR_ARG, "blocks per SM must be in [1, 64]");
            h->sweep_bps = (int)value;
            return SV_OK;
        case SV_OPT_SECTOR_SWEEP:
            if (value != 0 && value != 1) return fail(h, SV_ERR_ARG, "sector sweep mode must be 0 or 1");
            h->sweep_mode = (int)value;
            return SV_OK;
        case SV_OPT_WAIT_POLLS:
            if (value < 1 || value > (int64_t)1 << 30) return fail(h, SV_ERR_ARG, "wait polls must be in [1, 2^30]");
            h->wait_polls = value;
            return SV_OK;
        case SV_OPT_TEST_STALL:
            if (value < 0 || value > 3) return fail(h, SV_ERR_ARG, "test stall must be in [0, 3]");
            h->test_stall = (int)value;
            return SV_OK;
        case SV_OPT_REVERSE_INTERLEAVED:
            if (value != 0 && value != 1) return fail(h, SV_ERR_ARG, "reverse-sweep interleaving must be 0 or 1");
            h->rev_inter = (int)value;
            return SV_OK;
        case SV_OPT_L2_FETCH:
            if (value != 0 && value != 32 && value != 64 && value != 128)
                return fail(h, SV_ERR_ARG, "L2 fetch granularity must be 0, 32, 64 or 128");
            h->l2_fetch = (int)value;
            return SV_OK;
        case SV_OPT_POOL_VARIANT:
            if (value < 0 || value > 2) return fail(h, SV_ERR_ARG, "pool variant must be 0, 1 or 2");
            h->pool_variant = (int)value;
            return SV_OK;
        case SV_OPT_PROFILE:
            h->profile = value != 0;
            return SV_OK;
        case SV_OPT_LAYOUT_AUTO:
            h->layout_auto = value != 0;
            return SV_OK;
        case SV_OPT_AB_CHUNK:
            if (value < 0 || value > 8) return fail(h, SV_ERR_ARG, "alpha-beta chunk must be in [0, 8]");
            h->ab_chunk = value;
            return SV_OK;
        case SV_OPT_ROT_BLOCKS_PER_SM:
        case SV_OPT_SECT_BLOCKS_PER_SM:
        case SV_OPT_RDM_BLOCKS_PER_SM:
            if (value < 1 || value > 64) return fail(h, SV_ERR_ARG, "blocks per SM must be in [1, 64]");
            (opt == SV_OPT_ROT_BLOCKS_PER_SM ? h->rot_bps : opt == SV_OPT_SECT_BLOCKS_PER_SM ? h->sect_bps
                                                                                           : h->rdm_bps) = (int)value;
            return SV_OK;
    }
    return fail(h, SV_ERR_ARG, "unknown option");
}

}  // extern "C"
