// k_batch.cu -- many independent small problems (uneven qubit counts) in one
// persistent, graph-captured launch: reference preparation, the fermionic
// ansatz, sigma = (H - c) psi and the energy, and the adjoint sweep for the
// gradient, per instance ("Computational Details": ADAPT-VQE runs on many small
// systems; the emulator's workload for every optimiser step).
//
// Each block takes instances from a work queue (one atomicAdd per instance, no
// device-side waiting) in descending order of estimated cost, and runs the whole
// pipeline for it on a compact state: the amplitudes of the instance's
// (N_alpha, N_beta) sector in the string-row order C[rank(b)][rank(a)] (at 20
// qubits and 6 electrons 14,400 amplitudes instead of 2^20), in a per-block
// scratch slot that stays in L2.  The rotations pair every determinant that has
// the excitation's "from" pattern with its partner (found by string ranks), the
// sigma element is the same closed-form X-mask evaluation as the string-row
// kernel (sv_sigma.cuh), and the gradient sums are float64 with fixed-order block
// reductions, so an instance's results do not depend on which block ran it.
//
// An optional time budget makes every block stop taking new instances once the
// budget is spent (checked with %globaltimer before each instance); the host then
// reports SV_ERR_TIMEOUT and leaves the outputs of skipped instances as NaN.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "sv_internal.h"
#include "sv_sigma.cuh"

namespace svk {

struct BatchOp {
    uint32_t m, from, sm;  // qubit-space flip mask, "from" pattern, sign mask
    uint32_t mab;          // low 16 bits: alpha-string flip mask, high 16: beta-string flip mask
    uint32_t fab;          // the same for the "from" pattern
};

struct BatchInst {
    int n, N, Da, Db, L;
    uint32_t hf;                 // compact index of the reference determinant
    double shift;                // c of lambda = (H - c) psi
    double e_shift;              // E_nuc - c
    long long ops, cs;           // offsets into the op and (cos, sin) arrays
    long long eri, hm, dt, jt;   // offsets into the state-precision integral arena
    long long hd, jp;            // offsets into the float64 arena
    long long sa, sb;            // offsets into the uint32 spread arena
    long long stra, strb, ra, rb;  // offsets into the uint16 string arena
    long long out;               // E at out, gradient at out + 1 ...
    int fast;                    // 1: sigma by the string-blocked tables (both string counts <= kBatchSmax)
    int na, nb;                  // electrons per spin
};

// Largest string count per spin for which an instance's sigma runs from per-block
// dense same-spin matrices and excitation tables (matrices of kBatchSmax^2 values).
constexpr int kBatchSmax = 512;
// Dynamic shared memory the launch may take for the string-blocked sigma's data (the
// kernel's static shared memory stays below 8 KB, the block limit is 227 KB).
constexpr size_t kBatchSmemCap = 200 * 1024;

template <typename R>
struct BatchArgs {
    const BatchInst *inst;
    const int *order;
    int count;
    const BatchOp *ops;
    const cplx<R> *cs;           // (cos, sin) per op
    const R *rarena;
    const double *darena;
    const uint32_t *u32;
    const uint16_t *u16;
    double *out;
    cplx<R> *scratch;            // per block: psi then lambda, Dmax each
    int Dmax;
    unsigned char *work;         // per block: the string-blocked sigma's work area (fast instances)
    size_t work_stride;          // its bytes per block
    int Smax, Xmax;              // its sizes: strings per spin, table entries per string
    int smem_mode;               // 1: C~, the integrals and the tables in dynamic shared memory
    int Lmax;                    // most operators of a fast instance (its per-operator pair lists)
    int Dfast, Nmax;             // largest sector and orbital count of the fast instances
    int *ctrl;                   // [0] work counter, [1] timeout flag
    unsigned long long budget_ns;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- string-blocked sigma
//
// For an instance whose string counts are at most kBatchSmax, sigma is taken in the
// string-blocked basis (all alpha creators before all beta creators; amplitudes
// C~ = phi C with phi(a, b) = (-1)^popc(a & pp(b)), pp = prefix parity), where an
// alpha excitation's sign depends on the alpha string alone and a beta excitation's
// on the beta string alone:
//   sigma~[b][a] = (E_nuc - c + dA[a] + dB[b]) C~[b][a]
//                + sum_a' Ma[a][a'] C~[b][a'] + sum_b' Mb[b][b'] C~[b'][a]
//                + sum_k sum_j s_j s_k (q_j p_j | s_k r_k) C~[b'_k][a'_j]
// Ma holds the alpha singles' string-only coefficient h_qp + sum_{o in a} ((qp|oo) -
// (qo|op)) and the alpha-alpha doubles (a dense Da x Da matrix: at 20 qubits 84 of
// its 120 entries per row are nonzero), dA the alpha one-spin diagonal energy; Mb and
// dB the same for beta.  j runs over the alpha single excitations p -> q of a and,
// as "diagonal" entries p = q, over the occupied alpha orbitals; k likewise for b.
// A diagonal entry on one side and an excitation on the other gives the singles'
// dependence on the other spin's string (sum_{o in b} (qp|oo)); two diagonal entries
// give the alpha-beta part of the diagonal energy, sum (pp|qq).  Table entry:
// partner rank | sign << 14 | (q N + p) << 16.  sigma = phi sigma~.
__host__ __device__ constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Per-block work area: C~ [Dmax], Ma and Mb [Smax^2 each], the alpha and beta tables
// [Smax x Xmax each], dA and dB [Smax each, float64], then each operator's alpha and
// beta pair lists [Lmax x Smax each] and their lengths [2 Lmax].
__host__ __device__ constexpr size_t blocked_work_bytes(int Dmax, int Smax, int Xmax, int Lmax, size_t real) {
    return align256(2 * real * (size_t)Dmax) + 2 * align256(real * (size_t)Smax * Smax) +
           2 * align256(4 * (size_t)Smax * Xmax) + 2 * align256(8 * (size_t)Smax) +
           2 * align256(4 * (size_t)Lmax * Smax) + align256(8 * (size_t)Lmax);
}

// Dynamic shared memory of the shared-memory mode: C~ [Dfast], the integrals
// [Nmax^4] and both tables [Xmax x Smax], each from a 16-byte boundary.
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) / 16 * 16; }
__host__ __device__ constexpr size_t blocked_smem_bytes(int Dfast, int Nmax, int Smax, int Xmax, size_t real) {
    return align16(2 * real * (size_t)Dfast) + align16(real * (size_t)Nmax * Nmax * Nmax * Nmax) +
           2 * align16(4 * (size_t)Smax * Xmax);
}

template <typename R>
struct BlockedWork {
    cplx<R> *ct;
    const R *eri;      // the instance's (pq|rs): its shared copy in shared-memory mode
    R *eri_s;          // that copy (nullptr otherwise)
    R *Ma, *Mb;
    uint32_t *xa, *xb; // entry j of string I at x[j * D + I]
    double *dA, *dB;
    uint32_t *la, *lb; // operator k's alpha / beta pair list at l[k * Smax]: rank | sign << 14 | partner << 16
    int *lc;           // their lengths: lc[2 k], lc[2 k + 1]
};

template <typename R>
__device__ __forceinline__ BlockedWork<R> blocked_work(const BatchArgs<R> &B, const R *eri_g, unsigned char *smem) {
    unsigned char *w = B.work + (size_t)blockIdx.x * B.work_stride;
    const size_t S2 = align256(sizeof(R) * (size_t)B.Smax * B.Smax), X = align256(4 * (size_t)B.Smax * B.Xmax),
                 Sd = align256(8 * (size_t)B.Smax);
    BlockedWork<R> W;
    W.ct = reinterpret_cast<cplx<R> *>(w);
    w += align256(2 * sizeof(R) * (size_t)B.Dmax);
    W.Ma = reinterpret_cast<R *>(w);
    W.Mb = reinterpret_cast<R *>(w + S2);
    w += 2 * S2;
    W.xa = reinterpret_cast<uint32_t *>(w);
    W.xb = reinterpret_cast<uint32_t *>(w + X);
    w += 2 * X;
    W.dA = reinterpret_cast<double *>(w);
    W.dB = reinterpret_cast<double *>(w + Sd);
    w += 2 * Sd;
    const size_t Lb = align256(4 * (size_t)B.Lmax * B.Smax);
    W.la = reinterpret_cast<uint32_t *>(w);
    W.lb = reinterpret_cast<uint32_t *>(w + Lb);
    W.lc = reinterpret_cast<int *>(w + 2 * Lb);
    W.eri = eri_g;
    W.eri_s = nullptr;
    if (B.smem_mode) {
        const size_t n4 = (size_t)B.Nmax * B.Nmax * B.Nmax * B.Nmax;
        W.ct = reinterpret_cast<cplx<R> *>(smem);
        smem += align16(2 * sizeof(R) * (size_t)B.Dfast);
        W.eri_s = reinterpret_cast<R *>(smem);
        W.eri = W.eri_s;
        smem += align16(sizeof(R) * n4);
        W.xa = reinterpret_cast<uint32_t *>(smem);
        W.xb = reinterpret_cast<uint32_t *>(smem + align16(4 * (size_t)B.Smax * B.Xmax));
    }
    return W;
}

// Index of the u-th set bit of x (u counts from 0; x has more than u set bits).
__device__ __forceinline__ int nth_bit(uint32_t x, int u) {
    for (; u > 0; --u) x &= x - 1u;
    return __ffs(x) - 1;
}

// One spin's matrix M (D x D, row = output string), excitation table X (entry u of
// string I at X[u D + I], so a warp's strings read consecutive words) and one-spin
// diagonal dS, by the whole block.  M must be zero on entry.
template <typename R>
__device__ void build_spin_tables(const SigmaTables<R> &T, int spin, int D, int ne, R *M, uint32_t *X, double *dS) {
    const uint16_t *str = spin ? T.strb : T.stra, *rk = spin ? T.rb : T.ra;
    const int N = T.N, nv = N - ne, nsg = ne * nv, npo = ne * (ne - 1) / 2, npe = nv * (nv - 1) / 2;
    const int items = nsg + npo * npe + ne;
    for (int t = threadIdx.x; t < D * items; t += blockDim.x) {
        const int I = t / items, u = t - I * items;
        const uint32_t a = str[I], e = ~a & T.maskN, pps = prefix_parity(a);
        if (u < nsg) {  // single p -> q: matrix entry (own-string part) and table entry
            const int p = nth_bit(a, u / nv), q = nth_bit(e, u % nv);
            const uint32_t m = (1u << p) | (1u << q), sg = (uint32_t)par(pps & m) ^ (uint32_t)(p < q);
            const int J = rk[a ^ m];
            R v = T.hm[q * N + p];
            const R *dt = T.Dt + (q * N + p) * N;
            for (uint32_t o = a; o; o &= o - 1u) v += dt[__ffs(o) - 1];
            M[(size_t)I * D + J] = sg ? -v : v;
            X[(size_t)u * D + I] = (uint32_t)J | (sg << 14) | ((uint32_t)(q * N + p) << 16);
        } else if (u < nsg + npo * npe) {  // same-spin double p1 < p2 -> q1 < q2
            int io = (u - nsg) / npe, ie = (u - nsg) % npe, i1 = 0, e1 = 0;
            while (io >= ne - 1 - i1) io -= ne - 1 - i1++;
            while (ie >= nv - 1 - e1) ie -= nv - 1 - e1++;
            const int p1 = nth_bit(a, i1), p2 = nth_bit(a, i1 + 1 + io), q1 = nth_bit(e, e1), q2 = nth_bit(e, e1 + 1 + ie);
            const uint32_t m = (1u << p1) | (1u << p2) | (1u << q1) | (1u << q2);
            const uint32_t sg = (uint32_t)par(pps & m) ^ double_order_sign(p1, p2, q1, q2);
            const R v = eri4<R>(T, q1, p1, q2, p2) - eri4<R>(T, q1, p2, q2, p1);
            M[(size_t)I * D + rk[a ^ m]] = sg ? -v : v;
        } else {  // occupied orbital o: diagonal table entry
            const int o = nth_bit(a, u - nsg - npo * npe);
            X[(size_t)(nsg + (u - nsg - npo * npe)) * D + I] = (uint32_t)I | ((uint32_t)(o * N + o) << 16);
        }
    }
    for (int I = threadIdx.x; I < D; I += blockDim.x) {
        double d = 0.0;
        for (uint32_t o = str[I]; o; o &= o - 1u) {
            const int k = 2 * (__ffs(o) - 1) + spin;
            d += T.hdiag[k];
            for (uint32_t o2 = o & (o - 1u); o2; o2 &= o2 - 1u) d += T.Jp[k * T.n + 2 * (__ffs(o2) - 1) + spin];
        }
        dS[I] = d;
    }
}

// sigma~ at (Ia, Ib) from C~ (W.ct) and the instance's tables.
template <typename R>
__device__ __forceinline__ cplx<R> sigma_blocked(const SigmaTables<R> &T, const BlockedWork<R> &W, int Ia, int Ib,
                                                 int Db, int nxa, int nxb) {
    const int Da = T.Da, NN = T.N * T.N;
    const cplx<R> *ct = W.ct;
    const cplx<R> c0 = ct[(size_t)Ib * Da + Ia];
    const double d = T.e_shift + W.dA[Ia] + W.dB[Ib];
    R ar = (R)d * c0.x, ai = (R)d * c0.y;
    const cplx<R> *row = ct + (size_t)Ib * Da;
    for (int j = 0; j < Da; ++j) {  // alpha same-spin: Ma symmetric, read by column for coalescing
        const R w = W.Ma[(size_t)j * Da + Ia];
        const cplx<R> c = row[j];
        ar = fma(w, c.x, ar);
        ai = fma(w, c.y, ai);
    }
    const R *mb = W.Mb + (size_t)Ib * Db;
    for (int k = 0; k < Db; ++k) {  // beta same-spin
        const R w = mb[k];
        const cplx<R> c = ct[(size_t)k * Da + Ia];
        ar = fma(w, c.x, ar);
        ai = fma(w, c.y, ai);
    }
    const uint32_t *xa = W.xa + Ia, *xb = W.xb + Ib;
    for (int k = 0; k < nxb; ++k) {  // alpha-beta, singles' cross-spin parts, alpha-beta diagonal
        const uint32_t eb = xb[(size_t)k * Db];
        const cplx<R> *prow = ct + (size_t)(eb & 0x3FFFu) * Da;
        const R *er = W.eri + (eb >> 16);
        R tr = 0, ti = 0;
        for (int j = 0; j < nxa; ++j) {
            const uint32_t ea = xa[(size_t)j * Da];
            R w = er[(size_t)(ea >> 16) * NN];
            if ((ea >> 14) & 1u) w = -w;
            const cplx<R> c = prow[ea & 0x3FFFu];
            tr = fma(w, c.x, tr);
            ti = fma(w, c.y, ti);
        }
        if ((eb >> 14) & 1u) {
            tr = -tr;
            ti = -ti;
        }
        ar += tr;
        ai += ti;
    }
    return mk<R>(ar, ai);
}

// (cos, sin) of every instance's angles, in float64, then to the state precision: the
// first node of the batch graph (the host only copies the angles).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_batch_sincos(const double *__restrict__ theta, cplx<R> *__restrict__ cs,
                                                          long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double sn, cn;
        sincos(theta[k], &sn, &cn);
        cs[k] = mk<R>((R)cn, (R)sn);
    }
}

template <typename R, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_batch(BatchArgs<R> B) {
    extern __shared__ __align__(16) unsigned char batch_smem[];
    __shared__ int s_inst;
    __shared__ double red[2 * NT / 32];
    __shared__ unsigned long long s_t0;
    cplx<R> *psi = B.scratch + (size_t)blockIdx.x * 2 * B.Dmax;
    cplx<R> *lam = psi + B.Dmax;
    if (threadIdx.x == 0) s_t0 = global_ns();
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) {
            int next = -1;
            if (B.budget_ns && global_ns() - s_t0 > B.budget_ns) {
                atomicExch(&B.ctrl[1], 1);
            } else {
                int k = atomicAdd(&B.ctrl[0], 1);
                if (k < B.count) next = B.order[k];
            }
            s_inst = next;
        }
        __syncthreads();
        const int ii = s_inst;
        if (ii < 0) break;
        const BatchInst I = B.inst[ii];
        SigmaTables<R> T;
        T.sa = B.u32 + I.sa; T.sb = B.u32 + I.sb;
        T.stra = B.u16 + I.stra; T.strb = B.u16 + I.strb; T.ra = B.u16 + I.ra; T.rb = B.u16 + I.rb;
        T.eri = B.rarena + I.eri; T.hm = B.rarena + I.hm; T.Dt = B.rarena + I.dt; T.Jt = B.rarena + I.jt;
        T.hdiag = B.darena + I.hd; T.Jp = B.darena + I.jp; T.e_shift = I.e_shift;
        T.N = I.N; T.n = I.n; T.Da = I.Da; T.maskN = (1u << I.N) - 1u;
        const int Da = I.Da, D = I.Da * I.Db;
        // reference determinant
        for (int i = threadIdx.x; i < D; i += blockDim.x) psi[i] = mk<R>(0, 0);
        __syncthreads();
        if (threadIdx.x == 0) psi[I.hf] = mk<R>(1, 0);
        __syncthreads();
        const BlockedWork<R> W = blocked_work<R>(B, T.eri, batch_smem);
        if (I.fast) {
            // every operator's pair lists (alpha strings matching its alpha pattern x beta
            // strings matching its beta pattern), one warp per operator and spin, in rank
            // order by ballot compaction
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
            for (int t = warp; t < 2 * I.L; t += nwarp) {
                const int k = t >> 1, spin = t & 1;
                const BatchOp op = B.ops[I.ops + k];
                const uint32_t m = spin ? (op.mab >> 16) : (op.mab & 0xFFFFu), f = spin ? (op.fab >> 16) : (op.fab & 0xFFFFu);
                const int Ds = spin ? I.Db : Da;
                const uint16_t *str = spin ? T.strb : T.stra, *rk = spin ? T.rb : T.ra;
                const uint32_t *spr = spin ? T.sb : T.sa;
                uint32_t *dst = (spin ? W.lb : W.la) + (size_t)k * B.Smax;
                int cnt = 0;
                for (int base = 0; base < Ds; base += 32) {
                    const int Is = base + lane;
                    uint32_t sv = 0;
                    bool hit = false;
                    if (Is < Ds) {
                        sv = str[Is];
                        hit = (sv & m) == f;
                    }
                    const uint32_t bal = __ballot_sync(0xffffffffu, hit);
                    if (hit)
                        dst[cnt + __popc(bal & ((1u << lane) - 1u))] =
                            (uint32_t)Is | ((uint32_t)par(spr[Is] & op.sm) << 14) | ((uint32_t)rk[sv ^ m] << 16);
                    cnt += __popc(bal);
                }
                if (lane == 0) W.lc[t] = cnt;
            }
            __syncthreads();
        }
        // forward sweep
        for (int k = 0; k < I.L && I.fast; ++k) {  // over the operator's pairs
            const cplx<R> csk = B.cs[I.cs + k];
            const uint32_t *LA = W.la + (size_t)k * B.Smax, *LB = W.lb + (size_t)k * B.Smax;
            const int nA = W.lc[2 * k], np = nA * W.lc[2 * k + 1];
            for (int q = threadIdx.x; q < np; q += blockDim.x) {
                const int ib = q / nA;
                const uint32_t ea = LA[q - ib * nA], eb = LB[ib];
                const int i = (int)(eb & 0x3FFFu) * Da + (int)(ea & 0x3FFFu), j = (int)(eb >> 16) * Da + (int)(ea >> 16);
                const R ss = ((ea ^ eb) >> 14) & 1u ? -csk.y : csk.y;
                const cplx<R> u = psi[i], v = psi[j];
                psi[i] = mk<R>(csk.x * u.x - ss * v.x, csk.x * u.y - ss * v.y);
                psi[j] = mk<R>(csk.x * v.x + ss * u.x, csk.x * v.y + ss * u.y);
            }
            __syncthreads();
        }
        for (int k = 0; k < I.L && !I.fast; ++k) {
            const BatchOp op = B.ops[I.ops + k];
            const cplx<R> csk = B.cs[I.cs + k];
            for (int i = threadIdx.x; i < D; i += blockDim.x) {
                const int Ib = i / Da, Ia = i - Ib * Da;
                const uint32_t x = T.sa[Ia] | T.sb[Ib];
                if ((x & op.m) != op.from) continue;
                const int j = (int)T.rb[T.strb[Ib] ^ (op.mab >> 16)] * Da + T.ra[T.stra[Ia] ^ (op.mab & 0xFFFFu)];
                const R ss = par(x & op.sm) ? -csk.y : csk.y;
                const cplx<R> u = psi[i], v = psi[j];
                psi[i] = mk<R>(csk.x * u.x - ss * v.x, csk.x * u.y - ss * v.y);
                psi[j] = mk<R>(csk.x * v.x + ss * u.x, csk.x * v.y + ss * u.y);
            }
            __syncthreads();
        }
        // sigma and the energy
        double e_acc = 0.0, n_acc = 0.0;
        if (I.fast) {
            const int Db = I.Db, nxa = I.na * (I.N - I.na) + I.na, nxb = I.nb * (I.N - I.nb) + I.nb;
            for (int i = threadIdx.x; i < Da * Da; i += blockDim.x) W.Ma[i] = (R)0;
            for (int i = threadIdx.x; i < Db * Db; i += blockDim.x) W.Mb[i] = (R)0;
            if (W.eri_s)
                for (int i = threadIdx.x; i < I.N * I.N * I.N * I.N; i += blockDim.x) W.eri_s[i] = T.eri[i];
            for (int i = threadIdx.x; i < D; i += blockDim.x) {  // C~ = phi C
                const int Ib = i / Da, Ia = i - Ib * Da;
                const cplx<R> c = psi[i];
                W.ct[i] = par(T.stra[Ia] & prefix_parity(T.strb[Ib])) ? mk<R>(-c.x, -c.y) : c;
            }
            __syncthreads();
            build_spin_tables<R>(T, 0, Da, I.na, W.Ma, W.xa, W.dA);
            build_spin_tables<R>(T, 1, Db, I.nb, W.Mb, W.xb, W.dB);
            __syncthreads();
            for (int i = threadIdx.x; i < D; i += blockDim.x) {
                const int Ib = i / Da, Ia = i - Ib * Da;
                const cplx<R> c0 = W.ct[i];
                const cplx<R> s = sigma_blocked<R>(T, W, Ia, Ib, Db, nxa, nxb);
                lam[i] = par(T.stra[Ia] & prefix_parity(T.strb[Ib])) ? mk<R>(-s.x, -s.y) : s;
                e_acc += (double)c0.x * (double)s.x + (double)c0.y * (double)s.y;
                n_acc += (double)c0.x * (double)c0.x + (double)c0.y * (double)c0.y;
            }
        } else {
            for (int i = threadIdx.x; i < D; i += blockDim.x) {
                const int Ib = i / Da, Ia = i - Ib * Da;
                const cplx<R> c0 = psi[i];
                const cplx<R> s = sigma_at<R>(T, psi, Ia, Ib, c0);
                lam[i] = s;
                e_acc += (double)c0.x * (double)s.x + (double)c0.y * (double)s.y;
                n_acc += (double)c0.x * (double)c0.x + (double)c0.y * (double)c0.y;
            }
        }
        block_sum2_nt<NT>(e_acc, n_acc, red);  // contains the barrier that publishes lambda
        __shared__ double s_norm;
        if (threadIdx.x == 0) {
            s_norm = n_acc;
            B.out[I.out] = I.shift + e_acc / n_acc;
        }
        __syncthreads();
        const double nrm = s_norm;
        // reverse sweep
        for (int k = I.L - 1; k >= 0; --k) {
            const BatchOp op = B.ops[I.ops + k];
            const cplx<R> csk = B.cs[I.cs + k];
            double g = 0.0;
            const uint32_t *LA = W.la + (size_t)k * B.Smax, *LB = W.lb + (size_t)k * B.Smax;
            const int nA = I.fast ? W.lc[2 * k] : 0, np = I.fast ? nA * W.lc[2 * k + 1] : D;
            for (int q = threadIdx.x; q < np; q += blockDim.x) {
                int i, j;
                bool neg;
                if (I.fast) {  // over the operator's pairs
                    const int ib = q / nA;
                    const uint32_t ea = LA[q - ib * nA], eb = LB[ib];
                    i = (int)(eb & 0x3FFFu) * Da + (int)(ea & 0x3FFFu);
                    j = (int)(eb >> 16) * Da + (int)(ea >> 16);
                    neg = ((ea ^ eb) >> 14) & 1u;
                } else {  // every determinant, with the op's "from" test
                    i = q;
                    const int Ib = i / Da, Ia = i - Ib * Da;
                    const uint32_t x = T.sa[Ia] | T.sb[Ib];
                    if ((x & op.m) != op.from) continue;
                    j = (int)T.rb[T.strb[Ib] ^ (op.mab >> 16)] * Da + T.ra[T.stra[Ia] ^ (op.mab & 0xFFFFu)];
                    neg = par(x & op.sm);
                }
                const cplx<R> u = psi[i], v = psi[j], lu = lam[i], lv = lam[j];
                const R t = (lv.x * u.x + lv.y * u.y) - (lu.x * v.x + lu.y * v.y);
                g += (double)(neg ? -t : t);
                const R ss = neg ? -csk.y : csk.y;
                psi[i] = mk<R>(csk.x * u.x + ss * v.x, csk.x * u.y + ss * v.y);
                psi[j] = mk<R>(csk.x * v.x - ss * u.x, csk.x * v.y - ss * u.y);
                lam[i] = mk<R>(csk.x * lu.x + ss * lv.x, csk.x * lu.y + ss * lv.y);
                lam[j] = mk<R>(csk.x * lv.x - ss * lu.x, csk.x * lv.y - ss * lu.y);
            }
            const double gs = block_sum_nt<NT>(g, red);
            if (threadIdx.x == 0) B.out[I.out + 1 + k] = 2.0 * gs / nrm;
        }
        __syncthreads();
    }
}

}  // namespace svk

using namespace svk;

namespace svk {
void set_thread_error(const std::string &m);  // sv_api.cu: the message sv_last_error(NULL) returns
}

namespace {
sv_status bfail(sv_status s, const std::string &m) {
    set_thread_error(m);
    return s;
}

}  // namespace

struct sv_batch {
    int n_inst = 0;
    sv_dtype dtype = SV_C64;
    cudaStream_t stream = nullptr;
    int device = 0, sm_count = 148, grid = 0, grid_max = 0, Dmax = 0;
    int Smax = 0, Xmax = 0;      // the string-blocked sigma's sizes (0: no instance takes it)
    int Dfast = 0, Nmax = 0;     // largest sector / orbital count among those instances
    int Lmax = 0;                // most operators among them
    size_t work_stride = 0, smem = 0;  // dynamic shared memory of the launch (0: global-memory mode)
    void *d_work = nullptr;
    int threads = kThreads;  // block size of the persistent kernel: 256, 512 or 1024
    std::vector<int> L;
    std::vector<long long> cs_off, out_off;
    long long total_ops = 0, total_out = 0;
    std::vector<void *> dev;  // every device allocation
    BatchInst *d_inst = nullptr;
    int *d_order = nullptr, *d_ctrl = nullptr;
    BatchOp *d_ops = nullptr;
    void *d_cs = nullptr, *d_r = nullptr, *d_scratch = nullptr;
    double *d_theta = nullptr;
    double *d_d = nullptr, *d_out = nullptr;
    uint32_t *d_u32 = nullptr;
    uint16_t *d_u16 = nullptr;
    void *h_cs = nullptr;  // pinned: the angles of the next launch (float64)
    double *h_out = nullptr;
    int *h_ctrl = nullptr;
    unsigned long long budget_ns = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool own_stream = false;
    uint64_t launches = 0;
};

namespace {

template <typename R>
struct HostArena {
    std::vector<R> r;
    std::vector<double> d;
    std::vector<uint32_t> u32;
    std::vector<uint16_t> u16;
};

// String table set for (N, k electrons of one spin, spin offset 0 alpha / 1 beta).
struct StrSet {
    long long str, rank, spread;
    int count;
};

template <typename R>
sv_status build_plan(sv_batch *b, int n_inst, const sv_instance *inst) {
    HostArena<R> A;
    std::vector<BatchInst> hi(n_inst);
    std::vector<BatchOp> hops;
    std::vector<double> cost(n_inst);
    std::map<std::string, StrSet> sets;
    auto strset = [&](int N, int k, int spin) -> StrSet {
        std::string key = std::to_string(N) + "/" + std::to_string(k) + "/" + std::to_string(spin);
        auto it = sets.find(key);
        if (it != sets.end()) return it->second;
        StrSet s;
        s.rank = (long long)A.u16.size();
        A.u16.resize(A.u16.size() + ((size_t)1 << N), 0xFFFFu);
        std::vector<uint16_t> strs;
        for (uint32_t v = 0; v < (1u << N); ++v)
            if (__builtin_popcount(v) == k) {
                A.u16[s.rank + v] = (uint16_t)strs.size();
                strs.push_back((uint16_t)v);
            }
        s.str = (long long)A.u16.size();
        A.u16.insert(A.u16.end(), strs.begin(), strs.end());
        s.spread = (long long)A.u32.size();
        for (uint16_t v : strs) {
            uint32_t x = 0;
            for (int p = 0; p < N; ++p)
                if ((v >> p) & 1u) x |= 1u << (2 * p + spin);
            A.u32.push_back(x);
        }
        s.count = (int)strs.size();
        sets[key] = s;
        return s;
    };
    long long cs = 0, out = 0;
    b->L.resize(n_inst);
    b->cs_off.resize(n_inst);
    b->out_off.resize(n_inst);
    b->Dmax = 1;
    for (int t = 0; t < n_inst; ++t) {
        const sv_instance &in = inst[t];
        const int n = in.n_qubits, N = n / 2;
        if (n < 2 || n > 32 || (n & 1)) return bfail(SV_ERR_ARG, "instance qubit count must be even, 2..32");
        if (N > 16) return bfail(SV_ERR_ARG, "instance too large for the batched kernel");
        if (!in.h || !in.eri || (in.n_ops > 0 && !in.ops) || in.n_ops < 0 || in.n_occ < 0 || in.n_occ > n ||
            (in.n_occ > 0 && !in.occ))
            return bfail(SV_ERR_ARG, "bad instance description");
        uint32_t ref = 0;
        int na = 0, nb = 0;
        for (int k = 0; k < in.n_occ; ++k) {
            int j = in.occ[k];
            if (j < 0 || j >= n || ((ref >> j) & 1u)) return bfail(SV_ERR_ARG, "bad reference occupation");
            ref |= 1u << j;
            (j & 1) ? ++nb : ++na;
        }
        StrSet sa = strset(N, na, 0), sb = strset(N, nb, 1);
        const long long D = (long long)sa.count * sb.count;
        if (D > (1 << 22)) return bfail(SV_ERR_ARG, "instance sector too large for the batched kernel");
        b->Dmax = std::max<int>(b->Dmax, (int)D);
        BatchInst I{};
        I.n = n; I.N = N; I.Da = sa.count; I.Db = sb.count; I.L = in.n_ops;
        I.na = na; I.nb = nb;
        I.fast = sa.count <= kBatchSmax && sb.count <= kBatchSmax;
        if (I.fast) {
            b->Dfast = std::max<int>(b->Dfast, (int)D);
            b->Nmax = std::max(b->Nmax, N);
            b->Smax = std::max(b->Smax, std::max(sa.count, sb.count));
            b->Xmax = std::max(b->Xmax, std::max(na * (N - na) + na, nb * (N - nb) + nb));
            b->Lmax = std::max(b->Lmax, in.n_ops);
        }
        I.sa = sa.spread; I.sb = sb.spread; I.stra = sa.str; I.strb = sb.str; I.ra = sa.rank; I.rb = sb.rank;
        // reference index
        uint32_t ra_str = 0, rb_str = 0;
        for (int p = 0; p < N; ++p) {
            if ((ref >> (2 * p)) & 1u) ra_str |= 1u << p;
            if ((ref >> (2 * p + 1)) & 1u) rb_str |= 1u << p;
        }
        I.hf = (uint32_t)A.u16[sb.rank + rb_str] * sa.count + A.u16[sa.rank + ra_str];
        // integrals: validated like sv_ham_create, then cast
        sv_ham H;
        H.n_orb = N;
        H.e_nuc = in.e_nuc;
        H.h.assign(in.h, in.h + (size_t)N * N);
        H.eri.assign(in.eri, in.eri + (size_t)N * N * N * N);
        for (int p = 0; p < N; ++p)
            for (int q = 0; q < N; ++q)
                if (std::fabs(H.h[p * N + q] - H.h[q * N + p]) > 1e-12 * std::max(1.0, std::fabs(H.h[p * N + q])))
                    return bfail(SV_ERR_ARG, "instance h is not symmetric");
        auto E = [&](int p, int q, int r, int s) { return H.eri[(((size_t)p * N + q) * N + r) * N + s]; };
        for (int p = 0; p < N; ++p)
            for (int q = 0; q < N; ++q)
                for (int r = 0; r < N; ++r)
                    for (int s = 0; s < N; ++s) {
                        double v = E(p, q, r, s), tol = 1e-12 * std::max(1.0, std::fabs(v));
                        if (!std::isfinite(v) || std::fabs(v - E(q, p, r, s)) > tol || std::fabs(v - E(p, q, s, r)) > tol ||
                            std::fabs(v - E(r, s, p, q)) > tol)
                            return bfail(SV_ERR_ARG, "instance eri lacks the 8-fold symmetry");
                    }
        I.shift = diag_energy(H, ref, n);
        I.e_shift = in.e_nuc - I.shift;
        I.eri = (long long)A.r.size();
        for (double v : H.eri) A.r.push_back((R)v);
        I.hm = (long long)A.r.size();
        for (double v : H.h) A.r.push_back((R)v);
        I.dt = (long long)A.r.size();
        for (int q = 0; q < N; ++q)
            for (int p = 0; p < N; ++p)
                for (int k = 0; k < N; ++k) A.r.push_back((R)(E(q, p, k, k) - E(q, k, k, p)));
        I.jt = (long long)A.r.size();
        for (int q = 0; q < N; ++q)
            for (int p = 0; p < N; ++p)
                for (int k = 0; k < N; ++k) A.r.push_back((R)E(q, p, k, k));
        HostTables<double> ht;
        build_tables<double>(H, n, ht);
        I.hd = (long long)A.d.size();
        A.d.insert(A.d.end(), ht.hdiag.begin(), ht.hdiag.end());
        I.jp = (long long)A.d.size();
        A.d.insert(A.d.end(), ht.Jp.begin(), ht.Jp.end());
        // operators, qubit space
        I.ops = (long long)hops.size();
        const int ident[32] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15,
                               16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31};
        for (int k = 0; k < in.n_ops; ++k) {
            OpDesc d;
            std::string why;
            if (!make_op(in.ops[k], n, ident, d, why)) return bfail(SV_ERR_ARG, "instance op: " + why);
            uint32_t ma = 0, mb = 0;
            for (int p = 0; p < N; ++p) {
                if ((d.m >> (2 * p)) & 1u) ma |= 1u << p;
                if ((d.m >> (2 * p + 1)) & 1u) mb |= 1u << p;
            }
            uint32_t fa = 0, fb = 0;
            for (int p = 0; p < N; ++p) {
                if ((d.from >> (2 * p)) & 1u) fa |= 1u << p;
                if ((d.from >> (2 * p + 1)) & 1u) fb |= 1u << p;
            }
            hops.push_back(BatchOp{d.m, d.from, d.sm, ma | (mb << 16), fa | (fb << 16)});
        }
        I.cs = cs;
        b->cs_off[t] = cs;
        cs += in.n_ops;
        I.out = out;
        b->out_off[t] = out;
        out += 1 + in.n_ops;
        b->L[t] = in.n_ops;
        hi[t] = I;
        // cost: sector size x (connections + 3 sweeps over the operators)
        const double conn = (double)na * (N - na) + (double)nb * (N - nb);
        cost[t] = (double)D * (conn * conn + 3.0 * in.n_ops + 1.0);
    }
    b->total_ops = cs;
    b->total_out = out;
    std::vector<int> order(n_inst);
    for (int t = 0; t < n_inst; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    // device arenas
    auto up = [&](void **dst, const void *src, size_t bytes) -> sv_status {
        cudaError_t e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bfail(SV_ERR_OOM, "batch arena allocation failed");
        }
        b->dev.push_back(*dst);
        if (bytes && src) {
            e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return bfail(SV_ERR_CUDA, cudaGetErrorString(e));
        }
        return SV_OK;
    };
    sv_status s;
    if ((s = up((void **)&b->d_inst, hi.data(), hi.size() * sizeof(BatchInst))) != SV_OK) return s;
    if ((s = up((void **)&b->d_order, order.data(), order.size() * sizeof(int))) != SV_OK) return s;
    if ((s = up((void **)&b->d_ops, hops.data(), hops.size() * sizeof(BatchOp))) != SV_OK) return s;
    if ((s = up(&b->d_r, A.r.data(), A.r.size() * sizeof(R))) != SV_OK) return s;
    if ((s = up((void **)&b->d_d, A.d.data(), A.d.size() * sizeof(double))) != SV_OK) return s;
    if ((s = up((void **)&b->d_u32, A.u32.data(), A.u32.size() * sizeof(uint32_t))) != SV_OK) return s;
    if ((s = up((void **)&b->d_u16, A.u16.data(), A.u16.size() * sizeof(uint16_t))) != SV_OK) return s;
    if ((s = up(&b->d_cs, nullptr, std::max<long long>(cs, 1) * sizeof(cplx<R>))) != SV_OK) return s;
    if ((s = up((void **)&b->d_theta, nullptr, std::max<long long>(cs, 1) * sizeof(double))) != SV_OK) return s;
    if ((s = up((void **)&b->d_out, nullptr, std::max<long long>(out, 1) * sizeof(double))) != SV_OK) return s;
    if ((s = up((void **)&b->d_ctrl, nullptr, 2 * sizeof(int))) != SV_OK) return s;
    // scratch slots for the largest grid sv_batch_autotune may try (4 blocks per SM)
    b->grid_max = std::max(1, std::min(n_inst, b->sm_count * 4));
    b->grid = std::max(1, std::min(n_inst, b->sm_count * 2));
    if ((s = up(&b->d_scratch, nullptr, (size_t)b->grid_max * 2 * b->Dmax * sizeof(cplx<R>))) != SV_OK) return s;
    b->work_stride = b->Smax > 0 ? blocked_work_bytes(b->Dmax, b->Smax, b->Xmax, b->Lmax, sizeof(R)) : 0;
    {   // C~, the integrals and the tables in shared memory when they fit beside the static part
        const size_t sm = b->Smax > 0 ? blocked_smem_bytes(b->Dfast, b->Nmax, b->Smax, b->Xmax, sizeof(R)) : 0;
        b->smem = (sm > 0 && sm <= kBatchSmemCap) ? sm : 0;
    }
    if ((s = up(&b->d_work, nullptr, (size_t)b->grid_max * b->work_stride)) != SV_OK) return s;
    if (cudaMallocHost(&b->h_cs, std::max<long long>(cs, 1) * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_out, std::max<long long>(out, 1) * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_ctrl, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return bfail(SV_ERR_OOM, "pinned host allocation failed");
    }
    return SV_OK;
}

template <typename R>
sv_status capture(sv_batch *b) {
    BatchArgs<R> a;
    a.inst = b->d_inst; a.order = b->d_order; a.count = b->n_inst; a.ops = b->d_ops;
    a.cs = (const cplx<R> *)b->d_cs; a.rarena = (const R *)b->d_r; a.darena = b->d_d;
    a.u32 = b->d_u32; a.u16 = b->d_u16; a.out = b->d_out; a.scratch = (cplx<R> *)b->d_scratch;
    a.Dmax = b->Dmax; a.ctrl = b->d_ctrl; a.budget_ns = b->budget_ns;
    a.work = (unsigned char *)b->d_work; a.work_stride = b->work_stride; a.Smax = b->Smax; a.Xmax = b->Xmax;
    a.smem_mode = b->smem > 0; a.Dfast = b->Dfast; a.Nmax = b->Nmax; a.Lmax = b->Lmax;
    cudaStream_t st = b->stream;
    cudaError_t e = cudaSuccess;
    if (b->smem > 48 * 1024) {  // dynamic shared memory above the default limit
        e = b->threads == 1024 ? cudaFuncSetAttribute(k_batch<R, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem)
            : b->threads == 512 ? cudaFuncSetAttribute(k_batch<R, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem)
                                : cudaFuncSetAttribute(k_batch<R, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bfail(SV_ERR_CUDA, std::string("batch shared memory: ") + cudaGetErrorString(e));
        }
    }
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(SV_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    cudaMemcpyAsync(b->d_theta, b->h_cs, std::max<long long>(b->total_ops, 1) * sizeof(double), cudaMemcpyHostToDevice,
                    st);
    if (b->total_ops > 0) {
        const long long g = std::min<long long>((b->total_ops + kThreads - 1) / kThreads, (long long)b->sm_count * 4);
        k_batch_sincos<R><<<(int)g, kThreads, 0, st>>>(b->d_theta, (cplx<R> *)b->d_cs, b->total_ops);
    }
    cudaMemsetAsync(b->d_ctrl, 0, 2 * sizeof(int), st);
    if (b->threads == 1024) k_batch<R, 1024><<<b->grid, 1024, b->smem, st>>>(a);
    else if (b->threads == 512) k_batch<R, 512><<<b->grid, 512, b->smem, st>>>(a);
    else k_batch<R, 256><<<b->grid, 256, b->smem, st>>>(a);
    cudaMemcpyAsync(b->h_out, b->d_out, std::max<long long>(b->total_out, 1) * sizeof(double), cudaMemcpyDeviceToHost,
                    st);
    cudaMemcpyAsync(b->h_ctrl, b->d_ctrl, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    e = cudaStreamEndCapture(st, &b->graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(SV_ERR_CUDA, std::string("capture end: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(SV_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return SV_OK;
}

template <typename R>
void fill_cs(sv_batch *b, const double *theta) {
    if (b->total_ops > 0) std::memcpy(b->h_cs, theta, (size_t)b->total_ops * sizeof(double));
}

}  // namespace

extern "C" {

sv_status sv_batch_create(int n_inst, const sv_instance *inst, sv_dtype dtype, void *cuda_stream,
                          sv_batch_handle *out) {
    if (!out) return bfail(SV_ERR_ARG, "NULL output handle pointer");
    *out = nullptr;
    if (n_inst < 1 || !inst) return bfail(SV_ERR_ARG, "need at least one instance");
    if (dtype != SV_C64 && dtype != SV_C128) return bfail(SV_ERR_ARG, "bad dtype");
    sv_batch *b = new sv_batch();
    b->n_inst = n_inst;
    b->dtype = dtype;
    b->stream = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return bfail(SV_ERR_CUDA, "no CUDA device");
    }
    if (!b->stream) {  // graph capture needs a stream other than the legacy default stream
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return bfail(SV_ERR_CUDA, "stream creation failed");
        }
        b->own_stream = true;
    }
    cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, b->device);
    sv_status s = dtype == SV_C64 ? build_plan<float>(b, n_inst, inst) : build_plan<double>(b, n_inst, inst);
    if (s != SV_OK) {
        sv_batch_destroy(b);
        return s;
    }
    *out = b;
    return SV_OK;
}

sv_status sv_batch_set_time_limit(sv_batch_handle b, double ms) {
    if (!b || !(ms >= 0.0) || !std::isfinite(ms)) return bfail(SV_ERR_ARG, "bad time limit");
    b->budget_ns = (unsigned long long)(ms * 1e6);
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    return SV_OK;
}

sv_status sv_batch_energy_grad(sv_batch_handle b, const double *theta, double *e_out, double *grad_out) {
    if (!b) return bfail(SV_ERR_ARG, "NULL batch handle");
    if (b->total_ops > 0 && !theta) return bfail(SV_ERR_ARG, "NULL theta");
    for (long long k = 0; k < b->total_ops; ++k)
        if (!std::isfinite(theta[k])) return bfail(SV_ERR_ARG, "non-finite theta");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    sv_status s = SV_OK;
    if (b->dtype == SV_C64) fill_cs<float>(b, theta);
    else fill_cs<double>(b, theta);
    for (long long k = 0; k < b->total_out; ++k) b->h_out[k] = std::nan("");
    if (!b->exec) s = b->dtype == SV_C64 ? capture<float>(b) : capture<double>(b);
    if (s == SV_OK) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s = bfail(SV_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
        } else {
            b->launches += b->total_ops > 0 ? 2 : 1;
        }
    }
    if (s == SV_OK) {
        for (int t = 0; t < b->n_inst; ++t) {
            const double *o = b->h_out + b->out_off[t];
            if (e_out) e_out[t] = o[0];
            if (grad_out)
                for (int k = 0; k < b->L[t]; ++k) grad_out[b->cs_off[t] + k] = o[1 + k];
        }
        if (b->h_ctrl[1]) s = bfail(SV_ERR_TIMEOUT, "batch time limit reached; unfinished instances are NaN");
    }
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return s;
}

uint64_t sv_batch_launch_count(sv_batch_handle b) { return b ? b->launches : 0; }

static void drop_graph(sv_batch_handle b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

sv_status sv_batch_autotune(sv_batch_handle b, const double *theta, int *grid_out) {
    if (!b) return bfail(SV_ERR_ARG, "NULL batch handle");
    if (b->total_ops > 0 && !theta) return bfail(SV_ERR_ARG, "NULL theta");
    for (long long k = 0; k < b->total_ops; ++k)
        if (!std::isfinite(theta[k])) return bfail(SV_ERR_ARG, "non-finite theta");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    if (b->dtype == SV_C64) fill_cs<float>(b, theta);
    else fill_cs<double>(b, theta);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sv_status s = SV_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = bfail(SV_ERR_CUDA, "event creation failed");
    const int keep = b->grid, keep_t = b->threads;
    int best = keep, best_threads = keep_t;
    float best_t = -1.f;
    // (threads per block, blocks per SM): at most 2048 resident threads per SM
    const int cands[][2] = {{256, 1}, {256, 2}, {256, 4}, {512, 1}, {512, 2}, {1024, 1}, {1024, 2}};
    for (const auto &cd : cands) {
        if (s != SV_OK) break;
        const int g = std::max(1, std::min(b->n_inst, b->sm_count * cd[1]));
        if (g > b->grid_max) continue;
        drop_graph(b);
        b->grid = g;
        b->threads = cd[0];
        s = b->dtype == SV_C64 ? capture<float>(b) : capture<double>(b);
        float ms = 0.f;
        for (int r = 0; s == SV_OK && r < 2; ++r) {  // the second run is timed
            cudaError_t e = cudaEventRecord(e0, b->stream);
            if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                cudaGetLastError();
                s = bfail(SV_ERR_CUDA, std::string("batch autotune launch: ") + cudaGetErrorString(e));
            } else {
                b->launches += b->total_ops > 0 ? 2 : 1;
            }
        }
        if (s == SV_OK && (best_t < 0.f || ms < best_t)) {
            best_t = ms;
            best = g;
            best_threads = cd[0];
        }
    }
    drop_graph(b);
    b->grid = s == SV_OK ? best : keep;
    b->threads = s == SV_OK ? best_threads : keep_t;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (grid_out) *grid_out = b->grid;
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return s;
}

sv_status sv_batch_destroy(sv_batch_handle b) {
    if (!b) return SV_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (void *p : b->dev) cudaFree(p);
    if (b->h_cs) cudaFreeHost(b->h_cs);
    if (b->h_out) cudaFreeHost(b->h_out);
    if (b->h_ctrl) cudaFreeHost(b->h_ctrl);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
    return SV_OK;
}

}  // extern "C"
