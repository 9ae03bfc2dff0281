/*
 * sv_oracle.c -- plain CPU reference ("route A") for the state-vector path of
 * arXiv:2405.11567 (the emulator that stands in for the QPU: Fig. 1; Methodology,
 * "GPU-accelerated QPU emulation"; Methodology, "Computational Details").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or call
 * this file; only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg use it.  It shares no code, header or table with the CUDA path.
 *
 * What it computes, all in complex128 / float64, written as the plain
 * definitions (no blocking, no fusion, no closed-form shortcuts):
 *
 *   * A determinant |x> is an occupation-number basis state; bit j of x is the
 *     occupation of spin-orbital j, one spin-orbital per qubit (introduction;
 *     Methodology, Strategy 2: the n_{pq,sigma} equation and the Jordan-Wigner
 *     mapping named with it).
 *     Spin-orbital j = 2p + sigma (sigma = 0 alpha, 1 beta): interleaved ordering.
 *   * Jordan-Wigner rule for one operator on one determinant: a_j or a_j^dagger
 *     on |x> gives (-1)^(number of occupied spin-orbitals with index < j) times
 *     the determinant with bit j flipped, or zero if bit j is already empty /
 *     already full.  Products of operators are applied right-most first.
 *   * The state lives in the fixed (N_alpha, N_beta) sector: the HF start and
 *     every operator used here conserve both numbers, so all other amplitudes
 *     are identically zero and are not stored.  Determinants are kept as a
 *     sorted list; a determinant's position is found by binary search.
 *   * Excitation generator G = T - T^dagger with T = a+_a a_i (single) or
 *     T = a+_a a+_b a_j a_i (double, i<j, a<b).  U = exp(theta G).  Because
 *     G^2 = -P, where P projects onto the determinants that T or T^dagger
 *     do not annihilate, exp(theta G) = 1 + (cos theta - 1) P + sin theta G
 *     (the series of the exponential summed in closed form).
 *   * Hamiltonian (FCIDUMP chemist convention, "Computational Details": integrals passed as
 *     h_pq and (pq|rs)):
 *        H = E_nuc + sum_{PQ} h[PQ] a+_P a_Q
 *                  + 1/2 sum_{PQRS} [PQ|RS] a+_P a+_R a_S a_Q
 *     with h[PQ] = h_pq delta(sP,sQ) and [PQ|RS] = (pq|rs) delta(sP,sQ) delta(sR,sS).
 *     Every term is applied literally to every determinant.
 *   * One-particle density matrix n_{pq,sigma} = <psi| a+_{p sigma} a_{q sigma} |psi>
 *     (Methodology, Strategy 2, equation for n_{pq,sigma}).
 *
 * Build: gcc -O2 -fopenmp -fPIC -shared (oracle/build.py).  OpenMP parallel
 * loops run over output entries only (gather form), so results do not depend
 * on the thread count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <complex.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* ---- Jordan-Wigner action of one operator on one determinant ------------- */

/* a_j |x>: returns 0 if bit j is empty, else +-1 and clears bit j of *x. */
static int jw_annihilate(uint64_t *x, int j)
{
    uint64_t bit = 1ULL << j;
    if (!(*x & bit)) return 0;
    int below = __builtin_popcountll(*x & (bit - 1ULL));
    *x &= ~bit;
    return (below & 1) ? -1 : 1;
}

/* a+_j |x>: returns 0 if bit j is full, else +-1 and sets bit j of *x. */
static int jw_create(uint64_t *x, int j)
{
    uint64_t bit = 1ULL << j;
    if (*x & bit) return 0;
    int below = __builtin_popcountll(*x & (bit - 1ULL));
    *x |= bit;
    return (below & 1) ? -1 : 1;
}

/* ---- the sector of determinants ----------------------------------------- */

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Number of determinants with na alpha and nb beta electrons among n/2 spatial orbitals. */
int64_t orc_sector_dim(int n, int na, int nb)
{
    int N = n / 2;
    if (n < 2 || (n & 1) || n > 62 || na < 0 || nb < 0 || na > N || nb > N) return -1;
    double ca = 1.0, cb = 1.0;
    for (int k = 0; k < na; ++k) ca = ca * (N - k) / (k + 1);
    for (int k = 0; k < nb; ++k) cb = cb * (N - k) / (k + 1);
    return (int64_t)llround(ca) * (int64_t)llround(cb);
}

/* All determinants of the sector in ascending order of x.  Returns the count. */
int64_t orc_sector_list(int n, int na, int nb, uint64_t *out)
{
    int N = n / 2;
    int64_t D = orc_sector_dim(n, na, nb);
    if (D < 0) return -1;
    if (N > 24) return -1;
    /* every N-bit string with the right number of set bits, for each spin */
    uint64_t *sa = malloc(sizeof(uint64_t) * (size_t)(1ULL << N));
    uint64_t *sb = malloc(sizeof(uint64_t) * (size_t)(1ULL << N));
    int64_t A = 0, B = 0;
    for (uint64_t s = 0; s < (1ULL << N); ++s) {
        int c = __builtin_popcountll(s);
        if (c == na) sa[A++] = s;
        if (c == nb) sb[B++] = s;
    }
    int64_t k = 0;
    for (int64_t ia = 0; ia < A; ++ia) {
        for (int64_t ib = 0; ib < B; ++ib) {
            uint64_t x = 0;
            for (int p = 0; p < N; ++p) {
                if ((sa[ia] >> p) & 1ULL) x |= 1ULL << (2 * p);      /* alpha of orbital p */
                if ((sb[ib] >> p) & 1ULL) x |= 1ULL << (2 * p + 1);  /* beta of orbital p  */
            }
            out[k++] = x;
        }
    }
    free(sa);
    free(sb);
    qsort(out, (size_t)k, sizeof(uint64_t), cmp_u64);
    return k;
}

/* Position of determinant x in the sorted list, or -1 when absent. */
static int64_t det_index(const uint64_t *dets, int64_t D, uint64_t x)
{
    int64_t lo = 0, hi = D - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (dets[mid] == x) return mid;
        if (dets[mid] < x) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

int64_t orc_det_index(const uint64_t *dets, int64_t D, uint64_t x) { return det_index(dets, D, x); }

/* ---- excitation operators ------------------------------------------------ */
/* op[0] = kind (1 single, 2 double: fermionic; 3 single, 4 double: qubit
 * excitations); op[1..2] = occupied i, j; op[3..4] = virtual a, b.
 * A qubit excitation ("Computational Details": the qubit-excitation-based pool)
 * uses the qubit lowering / raising operators |0><1|, |1><0| on each qubit with
 * no Jordan-Wigner string: the same determinants are connected, always with +1. */

/* Apply a product of operators to |x>, right-most first: kinds[k] = 1 for a+,
 * 0 for a; modes[k] the spin-orbital.  Returns the accumulated sign (0 if the
 * product annihilates |x>) and leaves the resulting determinant in *y.          */
static int apply_product(int count, const int *kinds, const int *modes, uint64_t x, uint64_t *y)
{
    int s = 1;
    *y = x;
    for (int k = count - 1; k >= 0; --k) {
        int t = kinds[k] ? jw_create(y, modes[k]) : jw_annihilate(y, modes[k]);
        if (!t) return 0;
        s *= t;
    }
    return s;
}

/* The same product with qubit operators: a qubit flip that must find the bit in
 * the right state, no sign. */
static int apply_qubit_product(int count, const int *kinds, const int *modes, uint64_t x, uint64_t *y)
{
    *y = x;
    for (int k = count - 1; k >= 0; --k) {
        uint64_t bit = 1ULL << modes[k];
        if (kinds[k]) { if (*y & bit) return 0; *y |= bit; }
        else          { if (!(*y & bit)) return 0; *y &= ~bit; }
    }
    return 1;
}

/* T |x> : returns the sign (0 if annihilated) and the resulting determinant in *y. */
static int exc_T(const int32_t *op, uint64_t x, uint64_t *y)
{
    int (*apply)(int, const int *, const int *, uint64_t, uint64_t *) =
        op[0] >= 3 ? apply_qubit_product : apply_product;
    if (op[0] == 1 || op[0] == 3) {         /* a+_a a_i */
        const int kinds[2] = {1, 0}, modes[2] = {op[3], op[1]};
        return apply(2, kinds, modes, x, y);
    }
    /* a+_a a+_b a_j a_i */
    const int kinds[4] = {1, 1, 0, 0}, modes[4] = {op[3], op[4], op[2], op[1]};
    return apply(4, kinds, modes, x, y);
}

/* T^dagger |x> : (a+_a a_i)^dagger = a+_i a_a ; (a+_a a+_b a_j a_i)^dagger = a+_i a+_j a_b a_a. */
static int exc_Tdag(const int32_t *op, uint64_t x, uint64_t *y)
{
    int (*apply)(int, const int *, const int *, uint64_t, uint64_t *) =
        op[0] >= 3 ? apply_qubit_product : apply_product;
    if (op[0] == 1 || op[0] == 3) {
        const int kinds[2] = {1, 0}, modes[2] = {op[1], op[3]};
        return apply(2, kinds, modes, x, y);
    }
    const int kinds[4] = {1, 1, 0, 0}, modes[4] = {op[1], op[2], op[4], op[3]};
    return apply(4, kinds, modes, x, y);
}

/* Sign and target of T|x> for one determinant, exported for the sign-table tests. */
int orc_exc_apply(const int32_t *op, uint64_t x, uint64_t *y) { return exc_T(op, x, y); }

/* out = G psi with G = T - T^dagger.
 * (G psi)[x] = sum_y <x|T|y> psi[y] - sum_y <x|T^dagger|y> psi[y].
 * T and T^dagger have real +-1 matrix elements, so <x|T|y> = <y|T^dagger|x> and
 * <x|T^dagger|y> = <y|T|x>: the y that contribute are T^dagger|x> and T|x>.      */
void orc_generator_apply(const uint64_t *dets, int64_t D, const int32_t *op,
                         const cplx *psi, cplx *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t ix = 0; ix < D; ++ix) {
        uint64_t y;
        cplx acc = 0.0;
        int s = exc_Tdag(op, dets[ix], &y);         /* <x|T|y> = s */
        if (s) { int64_t jx = det_index(dets, D, y); if (jx >= 0) acc += s * psi[jx]; }
        s = exc_T(op, dets[ix], &y);                /* <x|T^dagger|y> = s */
        if (s) { int64_t jx = det_index(dets, D, y); if (jx >= 0) acc -= s * psi[jx]; }
        out[ix] = acc;
    }
}

/* out = exp(theta G) psi = psi + (cos theta - 1) P psi + sin theta G psi. */
void orc_rotate(const uint64_t *dets, int64_t D, const int32_t *op, double theta,
                const cplx *psi, cplx *out)
{
    double c = cos(theta), sn = sin(theta);
#pragma omp parallel for schedule(static)
    for (int64_t ix = 0; ix < D; ++ix) {
        uint64_t y;
        cplx g = 0.0;
        int in_p = 0;
        int s = exc_Tdag(op, dets[ix], &y);
        if (s) { int64_t jx = det_index(dets, D, y); if (jx >= 0) { g += s * psi[jx]; in_p = 1; } }
        s = exc_T(op, dets[ix], &y);
        if (s) { int64_t jx = det_index(dets, D, y); if (jx >= 0) { g -= s * psi[jx]; in_p = 1; } }
        out[ix] = in_p ? (psi[ix] + (c - 1.0) * psi[ix] + sn * g) : psi[ix];
    }
}

/* ---- Hamiltonian --------------------------------------------------------- */

/* sigma[r] = (H psi)[rows[r]] for r < nrows (rows == NULL: every determinant).
 * H|x> = sum_y <y|H|x> |y> is obtained by applying every term of H to |x>.
 * H is real symmetric (real h_pq = h_qp and (pq|rs) with the 8-fold symmetry),
 * so (H psi)[x] = sum_y <x|H|y> psi[y] = sum_y <y|H|x> psi[y].                   */
void orc_hamiltonian_apply(int n, const uint64_t *dets, int64_t D,
                           const double *h, const double *eri, double e_nuc,
                           const cplx *psi, cplx *sigma,
                           const int64_t *rows, int64_t nrows)
{
    int N = n / 2;
    int64_t R = rows ? nrows : D;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < R; ++r) {
        int64_t ix = rows ? rows[r] : r;
        uint64_t x = dets[ix];
        cplx acc = e_nuc * psi[ix];
        /* one-body: h[PQ] a+_P a_Q */
        for (int Q = 0; Q < n; ++Q) {
            for (int p = 0; p < N; ++p) {
                int P = 2 * p + (Q & 1);
                uint64_t y = x;
                int s1 = jw_annihilate(&y, Q);
                if (!s1) continue;
                int s2 = jw_create(&y, P);
                if (!s2) continue;
                int64_t jx = det_index(dets, D, y);
                if (jx < 0) continue;
                acc += h[p * N + (Q >> 1)] * (double)(s1 * s2) * psi[jx];
            }
        }
        /* two-body: 1/2 [PQ|RS] a+_P a+_R a_S a_Q */
        for (int Q = 0; Q < n; ++Q) {
            uint64_t y1 = x;
            int s1 = jw_annihilate(&y1, Q);
            if (!s1) continue;
            for (int S = 0; S < n; ++S) {
                uint64_t y2 = y1;
                int s2 = jw_annihilate(&y2, S);
                if (!s2) continue;
                for (int rr = 0; rr < N; ++rr) {
                    int Rr = 2 * rr + (S & 1);
                    uint64_t y3 = y2;
                    int s3 = jw_create(&y3, Rr);
                    if (!s3) continue;
                    for (int p = 0; p < N; ++p) {
                        int P = 2 * p + (Q & 1);
                        uint64_t y4 = y3;
                        int s4 = jw_create(&y4, P);
                        if (!s4) continue;
                        int64_t jx = det_index(dets, D, y4);
                        if (jx < 0) continue;
                        size_t e = (((size_t)p * N + (Q >> 1)) * N + rr) * N + (S >> 1);
                        acc += 0.5 * eri[e] * (double)(s1 * s2 * s3 * s4) * psi[jx];
                    }
                }
            }
        }
        sigma[r] = acc;
    }
}

/* ---- one-particle density matrix ----------------------------------------- */

/* out[sigma][p][q] = <psi| a+_{p sigma} a_{q sigma} |psi> = sum_x conj(psi[y]) <y|a+_P a_Q|x> psi[x],
 * y = a+_P a_Q x.  out is complex [2][N][N]. */
void orc_rdm1(int n, const uint64_t *dets, int64_t D, const cplx *psi, cplx *out)
{
    int N = n / 2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int e = 0; e < 2 * N * N; ++e) {
        int sg = e / (N * N), p = (e / N) % N, q = e % N;
        int P = 2 * p + sg, Q = 2 * q + sg;
        cplx acc = 0.0;
        for (int64_t ix = 0; ix < D; ++ix) {
            uint64_t y = dets[ix];
            int s1 = jw_annihilate(&y, Q);
            if (!s1) continue;
            int s2 = jw_create(&y, P);
            if (!s2) continue;
            int64_t jx = det_index(dets, D, y);
            if (jx < 0) continue;
            acc += conj(psi[jx]) * (double)(s1 * s2) * psi[ix];
        }
        out[e] = acc;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
