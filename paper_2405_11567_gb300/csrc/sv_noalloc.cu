// sv_noalloc.cu -- a 1-RDM entry point that allocates no device memory.
//
// Some callers cannot allocate device memory at the moment they need a
// density matrix: a process whose device memory is already entirely owned by
// another allocator (a framework's caching allocator, a memory pool sized to the
// whole GPU), or a caller that must not trigger the device-wide synchronisation
// that cudaFree implies in the middle of its own pipelined work.  For them,
// sv_rdm1_noalloc computes the same spin-resolved 1-RDM as sv_rdm1, for a state
// the caller holds in device memory, with every piece of scratch -- the sector
// list, the element table, the per-block partial sums and the reduced sums -- in
// one file-scope device array of fixed size (kNoallocBytes, reserved by every
// GPU that loads the library until the process exits).  Larger problems are
// rejected with SV_ERR_ARG.
//
// Host code may not use the array's name as a device address, so the first call
// on each device looks the address up with cudaGetSymbolAddress (with that
// device current) and keeps it, together with the identity of the CUDA context
// it belongs to; that first call should come before any stream capture.  The
// address is looked up again only when the device's current context is another
// one (after cudaDeviceReset the module is loaded anew and the array may move).
// All calls share the one array: a call overwrites everything it reads back (the
// kernel writes every partial it later sums), and two calls whose work overlaps
// on the GPU race on it.
#include <cuda.h>          // CUcontext / CUresult types; the driver calls are looked up through the runtime
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sv_internal.h"

namespace svk {
int rdm_gather_grid(uint64_t count, int sm_count);
int rdm_elements_bytes(int n, const int *perm, std::vector<uint8_t> &out);
cudaError_t launch_rdm_gather(const void *psi, int dtype, const uint32_t *sector, uint64_t count,
                              const void *elems, int n_el, int grid, double *partial, cudaStream_t st);
cudaError_t launch_reduce_rows(const double *partials, int rows, int cols, double *out, cudaStream_t st);
void set_thread_error(const std::string &m);
}  // namespace svk

using namespace svk;

namespace {

constexpr size_t kNoallocBytes = size_t(8) << 20;  // 8 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_mu;
// per device: the array's device address and the id of the context it was looked up in
void *g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};

typedef CUresult (*ctx_current_fn)(CUcontext *);
typedef CUresult (*ctx_id_fn)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current CUDA context (0 when it cannot be read:
// the address is then looked up on every call).  Caller holds g_mu.
unsigned long long current_context_id() {
    static bool resolved = false;
    static ctx_current_fn get_current = nullptr;
    static ctx_id_fn get_id = nullptr;
    if (!resolved) {
        resolved = true;
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = (ctx_current_fn)f;
            get_id = (ctx_id_fn)g;
        } else {
            cudaGetLastError();
        }
    }
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

sv_status nfail(sv_status s, const std::string &m) {
    set_thread_error(m);
    return s;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" sv_status sv_rdm1_noalloc(const void *psi_dev, int n_qubits, sv_dtype dtype, int n_alpha, int n_beta,
                                     void *cuda_stream, double *re_out, double *im_out) {
    if (!psi_dev || !re_out) return nfail(SV_ERR_ARG, "NULL state or output");
    if (n_qubits < 2 || n_qubits > SV_MAX_QUBITS || (n_qubits & 1))
        return nfail(SV_ERR_ARG, "n_qubits must be even and in [2, 32]");
    if (dtype != SV_C64 && dtype != SV_C128) return nfail(SV_ERR_ARG, "dtype must be SV_C64 or SV_C128");
    const int n = n_qubits, N = n / 2;
    if (n_alpha < 0 || n_beta < 0 || n_alpha > N || n_beta > N) return nfail(SV_ERR_ARG, "bad electron counts");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nfail(SV_ERR_CUDA, "no usable current CUDA device");
    }
    // sector list (qubit order: the caller's state is not permuted), host side
    std::vector<uint32_t> sa, sb, list;
    for (uint32_t s = 0; s < (1u << N); ++s) {
        int c = __builtin_popcount(s);
        uint32_t xa = 0, xb = 0;
        for (int p = 0; p < N; ++p)
            if ((s >> p) & 1u) {
                xa |= 1u << (2 * p);
                xb |= 1u << (2 * p + 1);
            }
        if (c == n_alpha) sa.push_back(xa);
        if (c == n_beta) sb.push_back(xb);
    }
    const uint64_t count = (uint64_t)sa.size() * sb.size();
    int ident[32];
    for (int q = 0; q < 32; ++q) ident[q] = q;
    std::vector<uint8_t> el;
    const int n_el = rdm_elements_bytes(n, ident, el);
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = rdm_gather_grid(count, sms);
    // scratch plan inside the static array
    const size_t off_list = 0;
    const size_t off_el = round256(off_list + count * sizeof(uint32_t));
    const size_t off_part = round256(off_el + el.size());
    const size_t off_out = round256(off_part + sizeof(double) * 2 * (size_t)n_el * grid);
    const size_t need = off_out + sizeof(double) * 2 * (size_t)n_el;
    if (need > kNoallocBytes)
        return nfail(SV_ERR_ARG, "sector too large for the fixed 8 MiB scratch of sv_rdm1_noalloc (" +
                                     std::to_string(count) + " determinants); use sv_rdm1");
    for (uint32_t a : sa)
        for (uint32_t b : sb) list.push_back(a | b);
    std::sort(list.begin(), list.end());
    // device address of the static scratch: once per device and context
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        // ctx is 0 on a thread without a current context yet: look the address up (which
        // makes the device's primary context current) and record that context's id
        const unsigned long long ctx = current_context_id();
        if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
            g_scratch_addr[dev] = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                g_scratch_addr[dev] = nullptr;
                return nfail(SV_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
            g_scratch_ctx[dev] = current_context_id();
        }
        base = g_scratch_addr[dev];
    }
    unsigned char *p = (unsigned char *)base;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    double host_sums[2 * 273];  // 2 * (1 + 32 + 240) elements at most (n <= 32)
    cudaError_t e = cudaSuccess;
    if (count) e = cudaMemcpyAsync(p + off_list, list.data(), count * sizeof(uint32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p + off_el, el.data(), el.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_rdm_gather(psi_dev, dtype, (const uint32_t *)(p + off_list), count, p + off_el, n_el, grid,
                              (double *)(p + off_part), st);
    if (e == cudaSuccess)
        e = launch_reduce_rows((const double *)(p + off_part), 2 * n_el, grid, (double *)(p + off_out), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(host_sums, p + off_out, sizeof(double) * 2 * n_el, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nfail(SV_ERR_CUDA, std::string("sv_rdm1_noalloc: ") + cudaGetErrorString(e));
    }
    const double nrm = host_sums[0];
    for (int s = 0; s < 2; ++s)
        for (int q = 0; q < N; ++q) {
            re_out[(s * N + q) * N + q] = host_sums[2 * (1 + 2 * q + s)] / nrm;
            if (im_out) im_out[(s * N + q) * N + q] = 0.0;
        }
    int k = 1 + n;
    for (int s = 0; s < 2; ++s)
        for (int a = 0; a < N; ++a)
            for (int b = a + 1; b < N; ++b, ++k) {
                const double re = host_sums[2 * k] / nrm, im = host_sums[2 * k + 1] / nrm;
                re_out[(s * N + a) * N + b] = re;
                re_out[(s * N + b) * N + a] = re;
                if (im_out) {
                    im_out[(s * N + a) * N + b] = im;
                    im_out[(s * N + b) * N + a] = -im;
                }
            }
    return SV_OK;
}
