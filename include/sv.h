/*
 * sv.h -- C-ABI of the GB300 (sm_103a) state-vector library for the hot path
 * of arXiv:2405.11567: the emulator that stands in for the QPU (Fig. 1;
 * Methodology, "GPU-accelerated QPU emulation").  It prepares the
 * Jordan-Wigner Hartree-Fock reference, applies a fermionic-excitation
 * (UCCSD / ADAPT-VQE) ansatz, and returns the energy <psi|H|psi> of the
 * second-quantised Hamiltonian, its exact gradient with respect to the ansatz
 * angles, and the spin-resolved one-particle density matrix n_{pq,sigma}.
 *
 * Conventions (fixed by this library where the paper is silent):
 *   - qubit j = spin-orbital j = 2p + sigma (sigma 0 = alpha, 1 = beta);
 *     bit j of a basis index x is the occupation of spin-orbital j.
 *   - Jordan-Wigner: a_j^(+) on |x> carries (-1)^(number of occupied
 *     spin-orbitals with index < j) (Methodology, Strategy 2: the
 *     Jordan-Wigner mapping used for n_{pq,sigma}).
 *   - excitation: single T = a+_a a_i; double T = a+_a a+_b a_j a_i with
 *     i < j and a < b; U = exp(theta (T - T^dagger)); the ansatz is
 *     U_L ... U_1 |ref>, ops[0] acting first ("Computational Details":
 *     ADAPT-VQE with an operator pool).
 *   - Hamiltonian (FCIDUMP chemist notation, "Computational Details"):
 *     H = E_nuc + sum h_pq a+_{p s} a_{q s}
 *               + 1/2 sum (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s}.
 *   - E = <psi|H|psi> / <psi|psi>; dE/dtheta_k in Hartree per radian.
 *
 * State storage: one dense vector of 2^n amplitudes in device memory, index =
 * basis index x (sv_create), or only the amplitudes of one (N_alpha, N_beta)
 * sector (sv_create_sector); complex amplitudes interleaved (re, im) in float
 * (SV_C64) or double (SV_C128), or real amplitudes (SV_R32, SV_R64).  Every
 * reduction (energy, gradient, norm, density matrix) is accumulated and returned
 * in float64 whatever the state precision.
 *
 * Ownership: the caller owns every host array passed in and out; the library
 * copies what it keeps.  Device buffers are owned by the library unless they
 * are passed to sv_create_with_buffers, in which case the caller owns them and
 * must keep them alive until sv_destroy.
 *
 * Errors: every call returns an sv_status; nothing aborts or throws across
 * this boundary.  SV_ERR_ARG = invalid argument (nothing was changed on the
 * device); SV_ERR_OOM = a device allocation failed; SV_ERR_CUDA = a CUDA call
 * failed (the handle becomes unusable: SV_ERR_STATE on later calls until
 * sv_prepare_hf / sv_prepare_state succeeds); SV_ERR_TIMEOUT = a bounded
 * device-side wait expired (batched launch only); SV_ERR_STATE = the call
 * needs a prepared state and there is none.  sv_last_error() returns a
 * message for the last failing call on a handle (or, with NULL, on this
 * thread).
 *
 * Streams: all device work of a handle is ordered on the stream given at
 * creation (NULL = the legacy default stream).  Calls that return host values
 * synchronise that stream before returning.
 */
#ifndef SV_GB300_H
#define SV_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sv_ctx *sv_handle;
typedef struct sv_ham *sv_ham_handle;

typedef enum {
    SV_OK = 0,
    SV_ERR_ARG = 1,
    SV_ERR_OOM = 2,
    SV_ERR_CUDA = 3,
    SV_ERR_TIMEOUT = 4,
    SV_ERR_STATE = 5
} sv_status;

/* State precision.  SV_C64 / SV_C128: complex amplitudes (float / double pairs).
 * SV_R32 / SV_R64: real amplitudes (float / double) -- the states of the paper's
 * real-angle ansatz on a real reference stay real (real integrals, real generators
 * T - T^dagger), so half the bytes and products suffice; host arrays of such a handle
 * hold one real per amplitude.  Real states: sv_create, sv_create_sector and every
 * state call; not the batched launch nor sv_rdm1_noalloc (SV_ERR_ARG). */
typedef enum { SV_C64 = 0, SV_C128 = 1, SV_R32 = 2, SV_R64 = 3 } sv_dtype;

/* One excitation operator.  kind 1: single, occ[0] -> vir[0] (occ[1], vir[1]
 * ignored); kind 2: double, occ[0] < occ[1], vir[0] < vir[1].  Kinds 3 and 4
 * are the same single and double as qubit excitations (the qubit-excitation-
 * based pool of "Computational Details"): products of qubit raising / lowering
 * operators with no Jordan-Wigner string, i.e. the same pairs of basis states
 * rotated with sign +1.  Indices are spin-orbitals in [0, n_qubits); the four
 * (two) indices are distinct and the operator conserves S_z (same number of
 * alpha spin-orbitals among occ and vir).  Anything else is SV_ERR_ARG. */
typedef struct {
    int32_t kind;
    int32_t occ[2];
    int32_t vir[2];
} sv_excitation;

/* Largest qubit count accepted (basis indices fit in 32 bits). */
#define SV_MAX_QUBITS 32

/* ---- state handles ------------------------------------------------------ */

/* Create a handle for an n_qubits state (2 <= n_qubits <= SV_MAX_QUBITS, even)
 * in precision dtype on the current CUDA device, ordered on cuda_stream
 * (a cudaStream_t, may be NULL).  Allocates the state vector (2^n amplitudes);
 * further buffers (the adjoint vector, checkpoints, reduction scratch) are
 * allocated on first use.  The state is unprepared until sv_prepare_hf or
 * sv_prepare_state.  Paper: the emulator's state vector (Fig. 1;
 * "Computational Details": state-vector emulation up to 32 qubits). */
sv_status sv_create(int n_qubits, sv_dtype dtype, void *cuda_stream, sv_handle *out);

/* As sv_create, but the state vector and the adjoint vector live in caller-owned
 * device buffers of 2^n amplitudes each (psi_dev required, lam_dev may be NULL:
 * then the library allocates it on first use).  Lets a caller allocate with its
 * own allocator (e.g. PyTorch's).  Both must be 256-byte aligned. */
sv_status sv_create_with_buffers(int n_qubits, sv_dtype dtype, void *cuda_stream,
                                 void *psi_dev, void *lam_dev, sv_handle *out);

/* Create a handle whose state keeps only the amplitudes of one particle-number
 * sector: n_alpha alpha and n_beta beta electrons among N = n_qubits/2 spatial
 * orbitals, C(N, n_alpha) * C(N, n_beta) amplitudes instead of 2^n (9,018,009
 * at 30 qubits and 5 + 5 electrons: 72 MB in complex64, held in L2).  Every
 * operator of the method (the excitations, H, a+_{p s} a_{q s}) conserves both
 * counts (Methodology: the spin-conserving UCCSD / ADAPT-VQE excitations and
 * the second-quantised H), so the result of every call equals that of a dense
 * handle (sv_create) on the same inputs.
 *
 * Device order of the amplitudes (sv_state_device_ptr): row-major matrix
 * C[rank(beta string)][rank(alpha string)], where the alpha (beta) string of
 * basis state x is its bits 2p (2p + 1), p = 0..N-1, packed into an N-bit
 * integer, and rank = position among the strings of the same popcount in
 * ascending order.  Host views are unchanged: sv_prepare_state and sv_get_state
 * take / give the dense 2^n qubit-order vector (zero outside the sector),
 * sv_get_amplitudes returns 0 for basis states outside the sector.
 * sv_prepare_hf and sv_prepare_state reject states of another sector
 * (SV_ERR_ARG); sv_set_layout accepts only the identity; there is no
 * sv_create_with_buffers form.  Errors: SV_ERR_ARG for n_qubits outside
 * [2, 32] or odd, counts outside [0, N], a bad dtype or NULL out; SV_ERR_OOM,
 * SV_ERR_CUDA as for sv_create.  No counterpart in the paper: a storage choice of
 * this library. */
sv_status sv_create_sector(int n_qubits, int n_alpha, int n_beta, sv_dtype dtype, void *cuda_stream,
                           sv_handle *out);

/* Release the handle and every device buffer it owns.  NULL is accepted. */
sv_status sv_destroy(sv_handle h);

/* Prepare the Hartree-Fock reference |x_HF>: the spin-orbitals listed in occ
 * (n_occ distinct indices in [0, n), any order) are occupied, all others
 * empty ("Computational Details": computations start from a HF state).  The
 * handle records this reference for sv_energy_grad. */
sv_status sv_prepare_hf(sv_handle h, const int32_t *occ, int n_occ);

/* Prepare an arbitrary initial state from host memory: 2^n amplitudes of the
 * handle's dtype (interleaved re, im for complex dtypes, one real each for real
 * dtypes), which must vanish (exactly) outside the
 * sector with n_alpha alpha and n_beta beta electrons (SV_ERR_ARG otherwise).
 * The handle keeps a device copy as the reference for sv_energy_grad (a
 * multi-determinant start such as the CIPSI states of "Computational
 * Details"). */
sv_status sv_prepare_state(sv_handle h, const void *amplitudes_host, int n_alpha, int n_beta);

/* Copy the current state (2^n amplitudes, dtype of the handle) to host memory. */
sv_status sv_get_state(sv_handle h, void *amplitudes_host);

/* Amplitudes of `count` basis states (indices in qubit order, each < 2^n) of the
 * current state, written to host memory (count amplitudes of the handle's dtype):
 * sampling a large state without copying all of it. */
sv_status sv_get_amplitudes(sv_handle h, const uint64_t *basis, int count, void *amplitudes_host);

/* Device pointer of the state vector (2^n amplitudes), for callers that read
 * it on the GPU.  Valid until sv_destroy.  Amplitudes are stored in the handle's
 * layout (sv_get_layout): the amplitude of basis state x sits at the address
 * whose bit storage_of_qubit[q] is bit q of x. */
sv_status sv_state_device_ptr(sv_handle h, void **psi_dev);

/* Storage layout: bit storage_of_qubit[q] of an amplitude's device address holds
 * qubit q (a permutation of [0, n); identity after sv_create).  A rotation whose
 * lowest address bit is b moves runs of 2^b consecutive amplitudes, so placing
 * rarely excited qubits on the low bits keeps the streaming kernels' runs long.
 * sv_set_layout moves the current state (and a stored reference) to the new
 * layout on the device and turns SV_OPT_LAYOUT_AUTO off.  Host-side views
 * (sv_prepare_state, sv_get_state, every returned value) are always in qubit
 * order.  No counterpart in the paper: a storage choice of this library. */
sv_status sv_set_layout(sv_handle h, const int32_t *storage_of_qubit);
sv_status sv_get_layout(sv_handle h, int32_t *storage_of_qubit);

/* ---- Hamiltonian handles -------------------------------------------------- */

/* Build a Hamiltonian from integrals in the FCIDUMP chemist convention
 * ("Computational Details"): h[p*n_orb+q] (symmetric), eri[((p*n_orb+q)*n_orb+r)*n_orb+s]
 * = (pq|rs) with the 8-fold symmetry of real orbitals (checked to 1e-12,
 * SV_ERR_ARG otherwise), e_nuc.  1 <= n_orb <= SV_MAX_QUBITS/2.  The X-mask
 * tables (every group of Pauli strings sharing a flip pattern, evaluated in
 * closed form) and the string tables of the expectation are built lazily per
 * state size and precision and cached in the handle. */
sv_status sv_ham_create(int n_orb, const double *h, const double *eri, double e_nuc,
                        sv_ham_handle *out);
sv_status sv_ham_destroy(sv_ham_handle ham);

/* ---- the hot path ---------------------------------------------------------- */

/* psi <- U_L ... U_1 psi with U_k = exp(theta[k] (T_k - T_k^dagger)), ops[0] first.
 * cos/sin of theta are taken on the host in float64.  One kernel per operator (dense
 * storage; sector storage: one cooperative launch for the whole list, SV_OPT_SECTOR_SWEEP).
 * On a state still equal to the determinant sv_prepare_hf wrote, with SV_OPT_LAYOUT_AUTO
 * on, the storage layout first becomes the one the operator list prefers. */
sv_status sv_apply_ansatz(sv_handle h, const sv_excitation *ops, int n_ops, const double *theta);

/* *e_out = <psi|H|psi> / <psi|psi> of the current state (Fig. 1: the QPU/GPU
 * returns <H>; FCI energy functional of Methodology).  n_orb of the
 * Hamiltonian must equal n_qubits / 2. */
sv_status sv_energy(sv_handle h, sv_ham_handle ham, double *e_out);

/* Energy and exact gradient of E(theta) for psi(theta) = U_L..U_1 |ref>, where
 * |ref> is the reference recorded by the last sv_prepare_hf / sv_prepare_state.
 * grad_out[k] = dE/dtheta_k (n_ops values).  Adjoint method: one forward sweep,
 * lambda = (H - c) psi, one reverse sweep that uncomputes psi and lambda gate by
 * gate (the constant c does not change the gradient of a unitary ansatz).  On
 * return the handle holds psi(theta).  Either output may be NULL. */
sv_status sv_energy_grad(sv_handle h, sv_ham_handle ham, const sv_excitation *ops, int n_ops,
                         const double *theta, double *e_out, double *grad_out);

/* ADAPT-VQE operator screening ("Computational Details": the ansatz grows by the
 * pool operator with the largest energy gradient): for the current state psi,
 * grad_out[k] = dE/dtheta at theta = 0 of exp(theta G_k) psi = 2 Re <psi|H G_k|psi>
 * / <psi|psi> for each of the n_pool pool operators (any kinds), and *e_out (may
 * be NULL) = E(psi).  One expectation pass writing lambda = (H - c) psi in compact
 * form, then one block per pool operator (SV_OPT_POOL_VARIANT). */
sv_status sv_pool_gradients(sv_handle h, sv_ham_handle ham, const sv_excitation *pool, int n_pool, double *e_out,
                            double *grad_out);

/* Spin-resolved one-particle density matrix of the current state,
 * n_{pq,sigma} = <psi|a+_{p sigma} a_{q sigma}|psi> / <psi|psi> (Methodology,
 * Strategy 2, equation for n_{pq,sigma}).  re_out[(sigma*N + p)*N + q] = Re n,
 * im_out likewise Im n (im_out may be NULL), N = n_qubits/2, sigma 0 = alpha. */
sv_status sv_rdm1(sv_handle h, double *re_out, double *im_out);

/* ---- no device allocation ------------------------------------------------------ */

/* The spin-resolved 1-RDM (same values and layout as sv_rdm1) of a state the
 * caller holds in device memory, computed without allocating any device memory:
 * for callers whose device memory is entirely owned by another allocator, or who
 * must not trigger the device-wide synchronisation cudaFree implies.  psi_dev:
 * 2^n_qubits amplitudes of dtype in qubit order (address bit q = qubit q), zero
 * outside the sector with n_alpha alpha and n_beta beta electrons.  All scratch
 * lives in one fixed 8 MiB device array that the library reserves on every GPU
 * that loads it, until the process exits; it holds 4 bytes per sector
 * determinant plus about 1.4 MB of partial sums, so sectors above roughly 1.7
 * million determinants are rejected with SV_ERR_ARG (use sv_rdm1).  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and keeps it for that device's CUDA context; make that first call before any
 * stream capture.  After the context changes (cudaDeviceReset) the next call
 * looks it up again.  Every call reuses the same array, so calls whose work
 * overlaps on the GPU (other streams, other threads) race: serialise them.
 * Ordering: the call reads psi_dev on cuda_stream (may be NULL, the legacy
 * default stream) and synchronises that stream only; work on another stream that
 * writes psi_dev (a handle created on a non-blocking stream, for instance) must
 * be ordered before it by the caller (an event the stream waits on, or a
 * synchronisation).  No counterpart in the paper: an operational variant of
 * sv_rdm1. */
sv_status sv_rdm1_noalloc(const void *psi_dev, int n_qubits, sv_dtype dtype, int n_alpha, int n_beta,
                          void *cuda_stream, double *re_out, double *im_out);

/* ---- many small problems in one launch --------------------------------------- */

typedef struct sv_batch *sv_batch_handle;

/* One independent problem of a batch.  n_qubits even, 2..32 (n_qubits/2 <= 16
 * orbitals and a sector of at most 2^22 determinants); occ: the reference
 * determinant's occupied spin-orbitals; h, eri, e_nuc: integrals as for
 * sv_ham_create (checked the same way); ops: its ansatz (rules of sv_excitation).
 * The library copies everything at sv_batch_create. */
typedef struct {
    int32_t n_qubits;
    const int32_t *occ;
    int32_t n_occ;
    const double *h;
    const double *eri;
    double e_nuc;
    const sv_excitation *ops;
    int32_t n_ops;
} sv_instance;

/* Plan a batch: tables, integrals and operators of every instance move to the
 * device once; states are kept per block in compact (N_alpha, N_beta)-sector form.
 * Work is ordered by estimated cost (largest first) and taken by the blocks of one
 * persistent kernel.  cuda_stream may be NULL (the plan then owns a stream; the
 * launch is captured in a CUDA graph, which the legacy default stream cannot
 * hold).  No counterpart in the paper beyond running many emulations; the
 * batched configuration of this library's workload list. */
sv_status sv_batch_create(int n_inst, const sv_instance *inst, sv_dtype dtype, void *cuda_stream,
                          sv_batch_handle *out);

/* Energy and gradient of every instance for the angles theta (concatenated in
 * instance order, sum of n_ops values): e_out[i] = E_i, grad_out (same layout as
 * theta) = dE_i/dtheta.  One graph launch (angles up, their cosines and sines in
 * float64 on the device, the batched kernel, results down), then
 * a stream synchronisation.  SV_ERR_TIMEOUT when the time limit stopped the
 * kernel early: the outputs of instances not run are NaN. */
sv_status sv_batch_energy_grad(sv_batch_handle b, const double *theta, double *e_out, double *grad_out);

/* Device-side time budget (ms, 0 = none): blocks stop taking new instances once it
 * is spent (checked before each instance; no block ever waits on another). */
sv_status sv_batch_set_time_limit(sv_batch_handle b, double ms);

/* Kernels launched by this batch so far (two per sv_batch_energy_grad: the angles'
 * cosines and sines, then the batched kernel; one when the instances have no
 * operators). */
uint64_t sv_batch_launch_count(sv_batch_handle b);

/* Autotuner for the persistent batched launch: times the captured launch (angles
 * up, kernel, results down) at the angles theta (as for sv_batch_energy_grad) with
 * 256, 512 and 1024 threads per block and 1, 2 or 4 blocks per SM (at most 2048
 * threads per SM; grids capped by the instance count) and keeps the fastest for later
 * calls; *grid_out (may be NULL) receives the grid.  Each instance runs whole in one
 * block with fixed-order sums, so results depend on the block size only through the
 * order of those sums (rounding) and reruns with one choice are bit-identical.  No
 * counterpart in the paper. */
sv_status sv_batch_autotune(sv_batch_handle b, const double *theta, int *grid_out);

sv_status sv_batch_destroy(sv_batch_handle b);

/* ---- options ------------------------------------------------------------------ */

typedef enum {
    SV_OPT_CHECKPOINT_INTERVAL = 1, /* store psi every C gates in the forward sweep of
                                       sv_energy_grad and restore it in the reverse sweep
                                       (0 = none; default 0) */
    SV_OPT_MAX_BYTES = 2,           /* cap on device bytes this handle may allocate
                                       (0 = no cap); checkpoints are dropped to fit */
    SV_OPT_EXPECT_VARIANT = 3,      /* 0 auto (= 5 for complex64 / real float32 states
                                       of at least 2^20 sector determinants whose
                                       same-spin couplings fill at least 5% of a string
                                       space of at most 4096 strings, where variant 5's
                                       limits hold and its planes take at most 16 GiB
                                       within the byte cap, else 4 for those states;
                                       = 6 for complex128 / real float64 states where
                                       the split form's rows fit in shared memory (3
                                       when its two work matrices do not fit the byte
                                       cap); else 3 where its rows fit in shared
                                       memory; else 2); 1 record scan:
                                       one thread per sector determinant tests every mask
                                       group (dense storage only); 2 string rows: compact
                                       alpha/beta-string matrix, one block per beta
                                       string; 3 string rows split: the alpha-beta
                                       doubles in a second kernel that stages partner rows
                                       in shared memory; 4 (single precision; float64
                                       states take 3): split, with the same-spin part as
                                       two dense products in the string-blocked basis,
                                       Ma X + X Mb^T, on the tensor cores (tcgen05 bf16
                                       MMAs on operands split into three bf16 pieces, six
                                       products: float32-level accuracy; TMA copies; a
                                       bounded wait that runs out makes the next
                                       synchronising call fail with SV_ERR_CUDA); Ma, Mb are
                                       built once per Hamiltonian and sector (4 (Da^2 +
                                       Db^2) bytes plus their bf16 pieces); 5 (single
                                       precision, N <= 16 spatial orbitals, at most 4096
                                       strings per spin; else 4): as 4, with the
                                       alpha-beta part too as tensor-core products, one
                                       per (alpha tile, partner beta string), into
                                       planes of planes x Db x (nb (N - nb) + 1) x Da
                                       floats (3.7 GB at 30 qubits, complex64) gathered
                                       in a fixed order; 6 (float64 states; single
                                       precision takes 3): the split form of 3 with every
                                       product and sum of an amplitude's connections in
                                       float-float arithmetic (a float64 value as the
                                       unevaluated sum of two float32 words, 48-bit
                                       significand; error-free transformations) on the
                                       FP32 pipe instead of GB300's much narrower FP64
                                       pipe; the amplitudes are converted once per call
                                       and sigma written back as float64 (two work
                                       matrices of 16 Da Db bytes, complex) */
    SV_OPT_RDM_VARIANT = 4,         /* 0 auto (3 for float64 states, else 2); 1 sector
                                       gather: one thread per sector determinant (dense
                                       storage only); 2 string rows: one block per beta
                                       string of the compact matrix, in the state's own
                                       arithmetic; 3 string rows in float-float arithmetic
                                       (float64 states, on the FP32 pipe: the compact
                                       matrix converted once per call into a work matrix
                                       of Da Db x 16 or 8 bytes; single-precision states
                                       take 2).  The automatic choice keeps 2 where that
                                       matrix cannot be allocated */
    SV_OPT_PROFILE = 5,             /* 1: record CUDA events around each phase (sv_phase_times) */
    SV_OPT_LAYOUT_AUTO = 6,         /* 1 (default): sv_energy_grad chooses the storage layout
                                       from its operator list (sv_set_layout), and so does
                                       sv_apply_ansatz while the state is still the
                                       determinant sv_prepare_hf wrote (re-written in the new
                                       layout); 0: keep it (sv_set_layout sets 0) */
    SV_OPT_AB_CHUNK = 7,            /* variant 3: partner rows staged per chunk (complex64:
                                       2, 4, 6 or 8; complex128: 1, 2, 3 or 4; another value
                                       takes the largest compiled size below it; 0 = the
                                       fastest estimate among the sizes that fit) */
    SV_OPT_ROT_BLOCKS_PER_SM = 8,   /* launch geometry of the dense rotation and adjoint
                                       kernels: at most this many blocks per SM (1..64,
                                       default 32) */
    SV_OPT_SECT_BLOCKS_PER_SM = 9,  /* the same for the sector rotation / adjoint kernels
                                       (default 8) */
    SV_OPT_RDM_BLOCKS_PER_SM = 10,  /* the same for the string-row 1-RDM (default 4) */
    SV_OPT_POOL_VARIANT = 11,       /* sv_pool_gradients: 0 auto (= 2); 1 string scan: one
                                       block per operator tests every alpha / beta string;
                                       2 pair lists: per-operator pair lists built once per
                                       pool (kept while the pool's operators are unchanged),
                                       amplitudes and lambda read interleaved */
    SV_OPT_L2_FETCH = 12,           /* dense storage: while sv_apply_ansatz, sv_energy_grad
                                       and sv_autotune run, the CUDA context's maximum L2
                                       fetch granularity (cudaLimitMaxL2FetchGranularity,
                                       a limit of the whole context) is this many bytes
                                       (32, 64 or 128; default 32); each of those calls
                                       puts the context's previous value back when it
                                       returns (sv_apply_ansatz returns before its
                                       kernels finish: the limit is a hint, so only
                                       their speed can depend on when it changes back).
                                       0 leaves the context's value alone, and so do
                                       states smaller than four times the device's L2
                                       (served from L2; a change of the limit costs about
                                       half a millisecond of host time).  Rotations of
                                       excitations on low address bits touch runs of
                                       32-64 bytes, which larger fetches double */
    SV_OPT_REVERSE_INTERLEAVED = 14, /* dense storage: 1 (default) sv_energy_grad runs its
                                       reverse sweep on psi(theta) and lambda interleaved
                                       by amplitude in one buffer (element x holds psi[x]
                                       then lambda[x]), so an excitation's touched runs
                                       are twice as long as in two separate vectors; used
                                       where the handle's adjoint vector and working copy
                                       are one allocation (not with a caller-provided
                                       adjoint vector, checkpoints or the record-scan
                                       expectation); 0 two separate vectors */
    SV_OPT_WAIT_POLLS = 15,         /* polls of each bounded wait before a kernel gives up
                                       (a poll: in k_ab_tc an mbarrier try-wait that
                                       suspends the thread for at most 64 ns; in k_same_tc
                                       a try-wait and a 32 ns sleep; at a grid barrier a
                                       read of its counter and a 32 ns sleep): the
                                       tensor-core expectation kernels' mbarrier waits
                                       (variants 4 and 5: the kernel then waits, bounded,
                                       for its copies and MMAs in flight, frees its
                                       tensor memory and returns) and the grid barriers
                                       of the whole-sweep launches (SV_OPT_SECTOR_SWEEP);
                                       the call then fails with SV_ERR_CUDA and the
                                       handle needs sv_prepare_hf / sv_prepare_state.
                                       1..2^30, default 2^22 */
    SV_OPT_TEST_STALL = 16,         /* failure-detection test hook, 0 (default) off: bit 0
                                       makes k_same_tc's producer issue no copy, bit 1
                                       makes k_ab_tc's builders stage and write nothing,
                                       so that the consumers' first bounded waits run out
                                       with no copy or MMA in flight (the path of a stuck
                                       producer).  No fault and no hang: the call reports
                                       SV_ERR_CUDA */
    SV_OPT_SECTOR_SWEEP = 17,       /* sector storage: 1 (default) each forward and reverse
                                       sweep is one cooperative launch that walks the
                                       operators in order with a grid-wide barrier
                                       between them (every barrier wait bounded by
                                       SV_OPT_WAIT_POLLS: past it the call fails with
                                       SV_ERR_CUDA); used where no checkpoint copy falls
                                       inside the sweep and the device accepts the
                                       cooperative launch, else one launch per operator
                                       (0 always) */
    SV_OPT_SWEEP_BLOCKS_PER_SM = 18 /* launch geometry of the whole-sweep launches: at most
                                       this many blocks per SM, no more than can be
                                       resident (1..64, default 2; sv_autotune times
                                       1, 2, 4, 8) */
} sv_option;

/* Options change launch choices or summation order only: results agree within the
 * precision's rounding.  SV_ERR_ARG for an unknown option or a value out of range. */
sv_status sv_set_option(sv_handle h, sv_option opt, int64_t value);

/* Current value of an option (after sv_autotune: the values it chose). */
sv_status sv_get_option(sv_handle h, sv_option opt, int64_t *value);

/* Autotuner: time, on this handle's device with CUDA events, the candidate launch
 * choices for the given Hamiltonian and ansatz (ops/theta as for sv_energy_grad)
 * and keep the fastest -- the expectation's form and partner-row chunk size
 * (SV_OPT_EXPECT_VARIANT 2 to 5, SV_OPT_AB_CHUNK), the rotation and adjoint kernels'
 * blocks per SM (4, 8, 16, 32; dense storage, or sector storage with one launch per
 * operator), the whole-sweep launches' (1, 2, 4, 8; sector storage,
 * SV_OPT_SWEEP_BLOCKS_PER_SM) and the 1-RDM's (2, 4, 8, 16).
 * Needs a prepared state; the state itself is left unchanged (candidates run on
 * copies in the adjoint vector and the saved-state buffer, which sv_energy_grad
 * allocates anyway).  Takes tens of launches of each kernel: call it once per problem
 * shape, outside any timed region.  No counterpart in the paper. */
sv_status sv_autotune(sv_handle h, sv_ham_handle ham, const sv_excitation *ops, int n_ops, const double *theta);

/* ---- introspection ------------------------------------------------------------ */

/* Number of phases reported by sv_phase_times. */
#define SV_PHASES 8

/* Device time (ms) of each phase of the last sv_energy_grad / sv_rdm1 call,
 * measured with CUDA events on the handle's stream while SV_OPT_PROFILE is 1:
 * [0] reference preparation, [1] forward sweep (one rotation kernel per op),
 * [2] expectation (sigma and energy), [3] reverse sweep (one adjoint kernel per
 * op plus the gradient reduction), [4] restoring psi(theta), [5] the last
 * sv_rdm1; inside [2], for the tensor-core expectation forms (variants 4 and 5):
 * [6] the same-spin products (k_transpose_pieces + k_same_tc), [7] the
 * alpha-beta products (k_ab_tc, variant 5).  Writes min(n_out, SV_PHASES)
 * values; phases not run are 0. */
sv_status sv_phase_times(sv_handle h, double *ms_out, int n_out);

/* Message of the last failing call on h (h == NULL: on this thread). Never NULL. */
const char *sv_last_error(sv_handle h);

/* Number of kernels this handle has launched since creation. */
uint64_t sv_launch_count(sv_handle h);

/* Library version string. */
const char *sv_version(void);

/* The checked build (libsv_gb300_check.so: the kernels compiled with SV_CHECK, which test
 * every index they compute from a host-built table against the size of the buffer it
 * addresses and, for a bad one, skip the access and record it instead of faulting): the
 * kinds of out-of-range index seen since the last call on the current device, then
 * cleared.  Byte 0: the sector kernels (sweeps, 1-RDM rows), byte 1: the string-row
 * expectation (alpha-beta plane offsets), byte 2: the alpha-beta tensor-core products
 * (gather offsets), bits 24-27: pool screening (pair addresses); within a byte 1 pair address, 2 string rank, 4 gather offset, 8 plane
 * offset; bit 31 where a word could not be read.  The default build returns 0.  Only the
 * kernels built on host tables are checked; the dense kernels' addresses are formed by
 * bit insertion and stay in range by construction. */
uint32_t sv_check_status(void);

#ifdef __cplusplus
}
#endif
#endif /* SV_GB300_H */
