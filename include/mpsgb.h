/* mpsgb -- grouped-qubit MPS TEBD of the 2D transverse-field Ising model on one GB300.
 *
 * C ABI of the CUDA library (libmpsgb.so).  Method: Mandra et al., "A Heuristic for
 * Matrix Product State Simulation of Out-of-Equilibrium Dynamics of Two-Dimensional
 * Quantum Spin Systems":
 *   Sec. II   Eq. hamiltonian  H = J sum_<ij> Z_i Z_j + h sum_i X_i (periodic square lattice)
 *             Eq. trotter_step U(dt) = e^{-i dt H_X/2} e^{-i dt H_ZZ} e^{-i dt H_X/2}
 *             Eq. initial_state prod_j (cos(theta/2)|0> + sin(theta/2)|1>), theta = theta_min + dtheta
 *             Eq. z2_tot  <Z_tot^2> = (1/n^2) sum_{j,k} <Z_j Z_k>
 *   Sec. III  TEBD on a grouped-qubit MPS (each row split in two groups fused into one
 *             block, snake order); in-block gates update one block; inter-block gates act
 *             as rank-2 MPOs that double the spanned bonds, which are truncated back to
 *             chi by SVD with the orthogonality centre on the bond; the state is
 *             renormalised after each truncation and F_MPS is the product of the
 *             truncation fidelities; Eq. Z_tot; Eq. Z_tot_via_F; Eq. z2_tot_rescaled;
 *             Table gamma_scaling.
 *
 * Conventions
 *   - Qubit (r, c) of an Lx x Ly grid has index r*Ly + c; |0> is Z = +1.
 *   - Gate angles are literal: the X layer is prod_j exp(-i alpha X_j), the ZZ layer
 *     prod_<ij> exp(-i phi Z_i Z_j) (phi = J dt; alpha = h dt/2 for second order).
 *   - Every function returns an mpsgb_status (0 on success).  On failure the message of
 *     mpsgb_last_error() (per calling thread) says what went wrong.  No exception or
 *     CUDA error crosses the ABI; a CUDA error reports MPSGB_EDEVICE.
 *   - Ownership: a handle owns all device memory of its MPS (blocks and workspace) and
 *     frees it in mpsgb_destroy.  The CUDA stream and the allocator passed at creation
 *     are borrowed and must outlive the handle.  Output pointers are caller-owned host
 *     memory.  Calls on one handle are not thread-safe; distinct handles are.
 *   - Device waits inside the library are bounded; none spins without a limit.
 */
#ifndef MPSGB_H
#define MPSGB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpsgb_mps* mpsgb_handle;

typedef enum {
  MPSGB_OK = 0,
  MPSGB_EINVAL = -1,    /* bad argument (size, enum, NaN angle, null pointer) */
  MPSGB_ENOMEM = -2,    /* the allocator returned NULL */
  MPSGB_ETIMEDOUT = -3, /* a bounded device wait ran out */
  MPSGB_EDEVICE = -4,   /* a CUDA call failed */
  MPSGB_ESTATE = -5     /* the handle is in a state that does not allow the call */
} mpsgb_status;

/* Arithmetic of the path.
 *   FP64         complex128 storage, every contraction in FP64; every spanned bond is truncated by
 *                the SVD of the centre block (one-sided Jacobi, no Gram matrix), which resolves
 *                Schmidt values down to the rounding floor.  The accuracy reference.
 *   SPLIT_TF32X3 as SPLIT_BF16X3 with TF32 splits on the tensor cores (tcgen05 kind::tf32): x_hi =
 *                tf32(x), x_lo = tf32(x - x_hi), 22 significant bits, at half the BF16 tensor rate.
 *   SPLIT_BF16X3 complex64 storage; the block-sized contractions (Grams, left factors, new blocks,
 *                transfer and environment products) on the tcgen05 tensor cores: every FP32
 *                component is split into two BF16 terms (hi + lo, 16 significant bits) and a
 *                real product is hi*hi + hi*lo + lo*hi with FP32 accumulation; the truncation core
 *                in FP32 on CUDA cores: the left Gram factorised by Cholesky (its eigenvectors when
 *                it is numerically singular), one Hermitian eigensolve of the 2 chi x 2 chi core;
 *                weights and F in FP64.
 *   FP32         complex64 storage, all contractions on FP32 CUDA cores (reference form for
 *                the split forms). */
typedef enum { MPSGB_FP64 = 0, MPSGB_SPLIT_TF32X3 = 1, MPSGB_SPLIT_BF16X3 = 2, MPSGB_FP32 = 3 } mpsgb_precision;
/* Non-adjacent gates: MPO route (Sec. III: the rank-2 MPO spans the bonds between the two blocks,
 * each truncated in turn) or SWAP routing (block q is moved next to block p by two-site SWAP updates,
 * the gate is one two-site update, and the block is moved back; every two-site update is an SVD
 * truncation).  SWAP routing needs chi * d <= 4096 (EINVAL at creation otherwise). */
typedef enum { MPSGB_ROUTE_MPO = 0, MPSGB_ROUTE_SWAP = 1 } mpsgb_route;
/* LAYER_ZSTAG: prod_j exp(-i angle s_j Z_j), the staggered field H_Z = sum_j s_j Z_j of Eq. xy_init,
 * s_j = (-1)^(sum of the qubit's lattice coordinates) (checkerboard). */
typedef enum { MPSGB_LAYER_X = 0, MPSGB_LAYER_ZZ = 1, MPSGB_LAYER_ZSTAG = 2 } mpsgb_layer;
/* X_STAG2: <X_stag^2> = (1/n^2) sum_{j,k} s_j s_k <X_j X_k> (Eq. xy_signal, the XY workload's signal,
 * s_j as for LAYER_ZSTAG); defined on every lattice. */
typedef enum { MPSGB_Z_TOT = 0, MPSGB_Z_TOT2 = 1, MPSGB_X_TOT = 2, MPSGB_X_STAG2 = 3 } mpsgb_obs;

/* Lattice and its mapping onto MPS sites.
 *   LATTICE_2D_GROUPED  the paper's main setting (Sec. II-III, Fig. mps_drawing): an Lx x Ly grid,
 *                       periodic in both directions; each row split into two groups of ceil(Ly/2)
 *                       and floor(Ly/2) qubits, each group one MPS block (d = 2^k), blocks along a
 *                       row snake.  Lz must be 0 or 1.
 *   LATTICE_3D_SITES    the 3D variant of the Supplemental Material (section "3D Transverse Field
 *                       Ising Model", Fig. 3D_snake): an Lx x Ly x Lz cubic grid with open
 *                       boundaries, one qubit per MPS site (d = 2), sites along a 3D snake (layer
 *                       z = 0 .. Lz-1; the rows x of a layer run forward in even layers and backward
 *                       in odd ones; each row y runs forward or backward in turn along the path, so
 *                       that consecutive sites are lattice neighbours).  Qubit (x, y, z) has the
 *                       global index (z Lx + x) Ly + y.  2 <= Lx, Ly, Lz <= 16, Lx Ly Lz <= 512. */
/*   LATTICE_2D_SITES    the XY workload's setting (Supplemental Material, section "XY Model"): an
 *                       Lx x Ly grid with open boundaries, one qubit per MPS site along a row snake
 *                       (row r runs forward for even r, backward for odd r); qubit (r, c) has index
 *                       r Ly + c.  2 <= Lx, Ly <= 16, Lx Ly <= 256.  Lz must be 0 or 1. */
typedef enum { MPSGB_LATTICE_2D_GROUPED = 0, MPSGB_LATTICE_3D_SITES = 1, MPSGB_LATTICE_2D_SITES = 2 } mpsgb_lattice;

/* Hamiltonian.
 *   MODEL_TFIM  Eq. hamiltonian, H = J sum_<ij> Z_i Z_j + h sum_i X_i, from the product state of Eq.
 *               initial_state (cfg.theta); any lattice; both routes.
 *   MODEL_XY    Eq. XY_hamiltonian, H_XY = (g/2) sum_<ij> (X_i X_j + Y_i Y_j) with g = cfg.J (and
 *               the J argument of mpsgb_step); LATTICE_2D_SITES, ROUTE_SWAP and trotter_order 2 only
 *               (EINVAL otherwise).  The handle starts in |Neel>, the ground state of H_Z =
 *               sum_j s_j Z_j (qubit j in |1> where s_j = +1); a step is Eq. xy_trotter_step (the
 *               depth-7 product over the bond sets A, B: horizontal bonds starting on even / odd
 *               columns, C, D: vertical bonds starting on even / odd rows), each two-qubit factor
 *               exp(-i theta (X X + Y Y)) applied by SWAP routing with a two-site update that
 *               carries the whole 4 x 4 gate.  Eq. xy_init is mpsgb_step(h, g, 0, dtau, 2, m)
 *               followed by mpsgb_apply_layer(h, MPSGB_LAYER_ZSTAG, pi / 8). */
typedef enum { MPSGB_MODEL_TFIM = 0, MPSGB_MODEL_XY = 1 } mpsgb_model;

typedef struct {
  int Lx, Ly;          /* 2D grid: Lx rows of Ly qubits, periodic in both directions; 2 <= Lx <= 16,
                          2 <= Ly <= 10 (blocks of at most 2^5 states), Lx * Ly <= 160.
                          3D grid: see mpsgb_lattice */
  int chi_max;         /* maximum bond dimension chi (>= 1) */
  double theta;        /* absolute initial angle of Eq. initial_state (use mpsgb_initial_theta) */
  mpsgb_precision prec;
  mpsgb_route route;
  unsigned long long seed; /* recorded only: the method draws no random numbers */
  double J, h, dt;     /* evolution parameters used by mpsgb_batch_step */
  int trotter_order;   /* 1: X then ZZ per step; 2: Eq. trotter_step */
  mpsgb_lattice lattice;
  int Lz;              /* layers of the 3D lattice (0 or 1 for the 2D lattices) */
  mpsgb_model model;
} mpsgb_config;

/* Device allocator used for every allocation of a handle.  alloc returns NULL on failure.
 * Pass NULL to mpsgb_create to use cudaMallocAsync / cudaFreeAsync on the handle's stream. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, void* stream, void* ctx);
  void* ctx;
} mpsgb_allocator;

/* Create the product state of Eq. initial_state with all bonds 1 and F_MPS = 1.
 * cfg: read only, copied.  alloc: borrowed or NULL.  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream) on which all work of the handle is issued.  *out receives the handle.
 * Errors: EINVAL for an unsupported grid / chi / precision, ENOMEM, EDEVICE. */
int mpsgb_create(const mpsgb_config* cfg, const mpsgb_allocator* alloc, void* cuda_stream, mpsgb_handle* out);

/* Apply one Trotter layer (Sec. III): LAYER_X applies prod_j exp(-i angle X_j) block by block
 * (no truncation); LAYER_ZZ applies prod_<ij> exp(-i angle Z_i Z_j): in-block pairs as diagonal
 * phases, then every inter-block gate, in the fixed order of the schedule, as a rank-2 MPO
 * followed by truncation of each spanned bond to chi_max; F_MPS is multiplied by each
 * truncation fidelity; LAYER_ZSTAG applies prod_j exp(-i angle s_j Z_j) block by block (no
 * truncation; the last factor of Eq. xy_init).  On MODEL_XY handles LAYER_X and LAYER_ZZ are
 * EINVAL (its layers are the bond sets of mpsgb_step).  Errors: EINVAL (NaN angle / bad layer),
 * EDEVICE. */
int mpsgb_apply_layer(mpsgb_handle h, mpsgb_layer layer, double angle);

/* Apply only the inter-block gates first .. first+count-1 of the ZZ layer's schedule (the order of
 * mpsgb_schedule_gates), each exp(-i phi Z_i Z_j) as a rank-2 MPO followed by the truncation of every
 * bond it spans (Sec. III); in-block phases are not applied.  A ZZ layer is the in-block phases
 * followed by all gates of the schedule.  For checks of single bond updates and for timing them.
 * Errors: EINVAL for a range outside the schedule or a NaN angle, EDEVICE, ETIMEDOUT. */
int mpsgb_apply_gates(mpsgb_handle h, int first, int count, double phi);

/* nsteps Trotter steps: order 2 = X(h dt/2) ZZ(J dt) X(h dt/2) (Eq. trotter_step), order 1 =
 * X(h dt) then ZZ(J dt).  Equivalent to the corresponding apply_layer calls.  MODEL_XY: nsteps
 * applications of Eq. xy_trotter_step with g = J (hx unused, order must be 2); a set of duration s
 * applies exp(-i (g s / 2)(X X + Y Y)) to each of its bonds, in the order of their (first site,
 * second site) positions. */
int mpsgb_step(mpsgb_handle h, double J, double hx, double dt, int trotter_order, int nsteps);

/* Re-compress the whole MPS to bond dimension chi <= chi_max by a left-to-right sequential SVD
 * sweep: the truncation of Sec. III (keep the chi largest singular values of each bond with the
 * orthogonality centre on it, renormalise) applied bond by bond without a gate; multiplies F_MPS
 * by every truncation fidelity.  Errors: EINVAL for chi < 1 or > chi_max. */
int mpsgb_truncate(mpsgb_handle h, int chi);

/* Expectation value (Eq. Z_tot, Eq. z2_tot, <X_tot> = (1/n) sum_j <X_j>, or <X_stag^2> of Eq.
 * xy_signal) of the current, normalised MPS, written to the host double *out.  Synchronises the
 * handle's stream. */
int mpsgb_expect(mpsgb_handle h, mpsgb_obs obs, double* out);

/* All three observables and the squared norm in one environment sweep:
 * out[0] = <Z_tot>, out[1] = <Z_tot^2>, out[2] = <X_tot>, out[3] = <psi|psi>. Host pointer. */
int mpsgb_observables(mpsgb_handle h, double out[4]);

/* F_MPS (Sec. III), the product of all truncation fidelities so far, to the host double *F. */
int mpsgb_fidelity(mpsgb_handle h, double* F);

/* Schmidt values across bond `bond` (0 .. nblocks-2, between blocks bond and bond+1), descending,
 * written to out[0 .. min(cap, n)-1]; *n receives the bond dimension.  These are the singular
 * values of Sec. III whose discarded squares make up 1 - F at a truncation.  Moves the
 * orthogonality centre (the state is unchanged).  Errors: EINVAL for a bad bond or null pointer. */
int mpsgb_singular_values(mpsgb_handle h, int bond, double* out, int cap, int* n);

/* Current bond dimensions (nblocks-1 values) to out[0 .. cap-1]; *n receives nblocks-1. */
int mpsgb_bond_dims(mpsgb_handle h, int* out, int cap, int* n);

/* Device memory a handle of this config holds for its blocks, chi^2 * dmax * nblocks * element
 * size, to the host *bytes.  Not from the paper: the admission figure of the serving loop (the
 * paper keeps its MPS sites in host RAM and moves them to the GPU as needed).  Host only. */
int mpsgb_footprint_bytes(const mpsgb_config* cfg, size_t* bytes);

/* Batched advance of many independent MPS (the task's batched workload; the paper evolves one MPS
 * at a time): every handle in hs[0 .. count-1] applies nlayers Trotter layers U(dt) (Eq.
 * trotter_step for order 2, X then ZZ for order 1) with the J, h, dt and order of its own config.
 * Handles advance concurrently, one host thread and the handle's own CUDA stream each, so their
 * kernels overlap on the device (handles that share a stream, e.g. the legacy default stream,
 * serialise there).  use_graph = 1: the fixed launch sequences inside a layer (Cholesky
 * factorisations, eigenvector back-transformations) are recorded once per size and buffer set as
 * CUDA graphs and replayed, on handles whose stream is not the legacy default stream; use_graph = 0
 * issues every launch directly.  A whole layer is not one graph: the truncation decisions (kept
 * counts, fidelities) are read back to the host after every eigensolve or SVD and decide the
 * shapes of what follows.  The handles must be distinct; use_graph other than 0 or 1 is EINVAL.
 * Returns the first failing status (with the handle's index in the message). */
int mpsgb_batch_step(mpsgb_handle* hs, int count, int nlayers, int use_graph);

/* Write / read a checkpoint: config, bond dims, centre, F_MPS, counters and all blocks.  Not from
 * the paper: persistence of this library (file layout: "MPSGBv2\0", the config struct, four ints
 * {element bytes, blocks, centre, 0}, F as a double, five 64-bit counters, the bond dims as ints,
 * then every block (left, d, right) row-major complex in the form's element type).
 * mpsgb_load creates a new handle (alloc and stream as in mpsgb_create).  Errors: EINVAL for an
 * unreadable or mismatched file, ENOMEM, EDEVICE. */
int mpsgb_save(mpsgb_handle h, const char* path);
int mpsgb_load(const char* path, const mpsgb_allocator* alloc, void* cuda_stream, mpsgb_handle* out);

/* Free the handle and all its device memory (synchronises its stream).  NULL is ignored. */
void mpsgb_destroy(mpsgb_handle h);

/* Message of the last failed call on this thread ("" if none).  Valid until the next call. */
const char* mpsgb_last_error(void);

/* Counters of a handle: out[0] bond truncations, out[1] inter-block gates, out[2] centre moves,
 * out[3] eigensolver calls, out[4] eigensolver sweeps.  Host pointer, 5 entries. */
int mpsgb_stats(mpsgb_handle h, long long out[5]);

/* Cycle limit (SM clock cycles) of the library's bounded device waits on other CTAs: the grid
 * barriers of the Householder reduction.  A wait that runs out records an error word and lets the
 * kernel finish; the call then returns MPSGB_ETIMEDOUT and the CUDA context stays usable.  The
 * default, 4e9 cycles (about 2 s), is far above any legitimate wait; tests lower it to exercise the
 * timeout path.  cycles <= 0 restores the default.  Process-wide; returns the previous limit.
 * Not from the paper: a robustness control of this library. */
long long mpsgb_set_wait_limit(long long cycles);

/* All counters of a handle, in this order: bond truncations, inter-block gates, centre moves,
 * eigensolver or SVD calls, their sweeps, Gram matrices factorised by Cholesky (complex64 forms),
 * Gram matrices too close to singular for Cholesky (the eigenvector factor was taken).  Up to cap
 * values to out; *n receives the number of counters (7).  Not from the paper: diagnostics. */
int mpsgb_counters(mpsgb_handle h, long long* out, int cap, int* n);

/* Number of CUDA kernels the library has launched in this process (all handles). */
unsigned long long mpsgb_launch_count(void);

/* Device-time measurement of the library's launch sites with CUDA events on their own streams.
 * mpsgb_kernel_timing(1) resets the totals and starts recording (0 stops); mpsgb_kernel_times
 * synchronises on the recorded events and returns, for launch site `site` (0 .. 10, see
 * mpsgb_kernel_site_name), the summed device time in ms, the launch count and the useful work of
 * those launches (real flops for arithmetic sites -- 16 n^3 / 3 for the Householder reduction of an
 * n x n Hermitian matrix; bytes moved for the in-block gate; 0 for the Jacobi SVD, whose work
 * depends on the data).
 * Recording adds two event records per launch; it is off by default. */
int mpsgb_kernel_timing(int enable);
int mpsgb_kernel_times(int site, double* ms, long long* launches, double* work);
const char* mpsgb_kernel_site_name(int site);

/* Self-test of the tensor-core split GEMM (no paper counterpart; a kernel check): multiplies seeded
 * random complex64 matrices, op(A) (M x K) times op(B) (K x N) with op(A) = A^H if mode bit 0 and
 * op(B) = B^T if mode bit 1, on the tensor cores (BF16 splits, or TF32 splits if mode bit 2) and
 * on FP32 CUDA cores, and writes
 * max |difference| / max |CUDA-core result| to *rel_err.  Allocates its own device memory. */
int mpsgb_tc_gemm_selftest(int M, int N, int K, int mode, unsigned long long seed, double* rel_err);

/* Self-test of the Hermitian eigensolver (no paper counterpart; a kernel check): a seeded n x n
 * Hermitian complex matrix is decomposed in FP64 (fp64 != 0) or FP32.  kind 0: X X^H with graded
 * columns of X (spectrum over many decades); kind 1: X X^H of rank n/2 (n - n/2 exact zeros);
 * kind 2: [[I, P Q^H], [Q P^H, I]] with n/8 columns in P and Q (eigenvalue 1 with multiplicity
 * n - 2(n/8) inside the spectrum).  out[0] outer sweeps, or the eigensolver's negative status,
 * out[1] device ms, out[2] max |A V - V diag(w)| / max |w|, out[3] max |V^H V - I| over sampled
 * columns, out[4] 1 if w is descending, out[5] max |w|.  Allocates its own device memory. */
int mpsgb_eig_selftest(int n, int fp64, int kind, unsigned long long seed, double out[6]);

/* Self-test of the one-sided Jacobi SVD of the FP64 form's truncation (no paper counterpart; a kernel
 * check): X is a host p x q complex matrix (row-major, interleaved re / im doubles; converted to
 * complex64 if fp64 == 0), decomposed on the GPU as X = U diag(s) Vh.  s: host, p values,
 * descending.  out[0] sweeps (negative: the solver's error status), out[1] device ms, out[2]
 * max |U diag(s) Vh - X| / max |X|, out[3] max |U^H U - I|, out[4] max |Vh Vh^H - I| over the rows
 * above the numerical-rank cut, out[5] that rank.  Allocates its own device memory. */
int mpsgb_svd_selftest(int p, int q, int fp64, const double* X, double* s, double out[6]);

/* Allocation-free Hermitian eigendecomposition (the paper has no counterpart: this is a service
 * for callers that cannot allocate device memory at the point of the call, e.g. code that runs
 * under a frozen or request-scoped allocator, or a thread that must not enter the CUDA allocator).
 * A: n x n Hermitian matrix on the device, row-major with leading dimension lda, complex128 if
 * fp64 != 0 else complex64 (read only).  w: n eigenvalues, descending (double / float, device).
 * V: eigenvectors as columns, row-major n x n with leading dimension ldv (device); A = V diag(w) V^H.
 * Work is issued on cuda_stream; the call blocks the calling host thread until that stream has
 * finished it (including the last kernel), so when it returns the shared array is free again.
 * Nothing is allocated: the solver's workspace is one fixed device array of 1 MiB per device, so
 * n is limited to 1..128 (EINVAL beyond, before anything is launched).  The first call on a device
 * resolves that array's device address (cudaGetSymbolAddress) and caches it for the process; make
 * that first call before any stream capture begins.  The cached address does not survive
 * cudaDeviceReset.  Every call on a device shares the array and leaves its contents behind (each
 * call re-initialises what it reads); calls that overlap on the GPU, from several host threads at
 * once, race on it and must be serialised by the caller.  Errors: EINVAL, ETIMEDOUT (sweep
 * limit), EDEVICE (a launch failed or the stream reported an error). */
int mpsgb_eigh_noalloc(int n, int fp64, const void* A, long long lda, void* w, void* V, long long ldv,
                       void* cuda_stream);

/* Host-only schedule facts of an Lx x Ly grid (no GPU needed): out[0] blocks, out[1] ZZ bonds,
 * out[2] in-block bonds, out[3] inter-block gates, out[4] bond truncations per ZZ layer,
 * out[5] largest local dimension.  Errors: EINVAL for an unsupported grid. */
int mpsgb_schedule_info(int Lx, int Ly, long long out[6]);

/* Host-only: the inter-block gates of the ZZ layer in application order, 6 ints each
 * (p, q, qubit_i, qubit_j, bit_i, bit_j), at most cap gates; *n receives the gate count. */
int mpsgb_schedule_gates(int Lx, int Ly, int* out, int cap, int* n);

/* The same two queries for the lattice of a config (cfg->lattice, Lx, Ly, Lz; host only).  For
 * LATTICE_3D_SITES every site holds one qubit (bit positions 0) and every ZZ bond is an
 * inter-site gate.  Errors: EINVAL for an unsupported lattice. */
int mpsgb_config_schedule_info(const mpsgb_config* cfg, long long out[6]);
int mpsgb_config_schedule_gates(const mpsgb_config* cfg, int* out, int cap, int* n);

/* Host-only: theta_min + dtheta with theta_min = asin(h / (4 J)) (Sec. II; 4 = neighbours of a
 * site of the square lattice). */
double mpsgb_initial_theta(double J, double hx, double dtheta);

/* Host-only: theta_min + dtheta for a lattice, theta_min = asin(h / (z J)) with z the number of
 * neighbours of a site: 4 for LATTICE_2D_GROUPED (Sec. II), 6 for LATTICE_3D_SITES (the 3D
 * variant starts from the same product state, Eq. initial_state; z = 6 is the cubic lattice's
 * coordination, the mean-field minimum of the bulk).  NaN for an unknown lattice. */
double mpsgb_initial_theta_lattice(mpsgb_lattice lattice, double J, double hx, double dtheta);

/* Host-only: gamma_fit = a log2(chi)/n + b of Table gamma_scaling; temperature 0 = low
 * (dtheta = 0), 1 = mid (2 pi/9), 2 = high (3 pi/9).  Returns NaN for another temperature. */
double mpsgb_gamma_fit(int temperature, int chi, int n);

/* Host-only: gamma_fit for a lattice: LATTICE_2D_GROUPED as mpsgb_gamma_fit; LATTICE_3D_SITES from
 * Table 3d_gamma_scaling of the Supplemental Material's 3D section (a = 2.654, 2.153, 1.5104 for
 * dtheta = 0, pi/9, 2 pi/9; b = 0).  NaN for another lattice, temperature outside 0..2 or
 * chi, n < 1. */
double mpsgb_gamma_fit_lattice(mpsgb_lattice lattice, int temperature, int chi, int n);

/* Host-only rescaling (Eq. Z_tot_via_F and Eq. z2_tot_rescaled): out[0] = F * z,
 * out[1] = z2 * F^gamma. */
int mpsgb_rescale(double z, double z2, double F, double gamma, double out[2]);

#ifdef __cplusplus
}
#endif
#endif /* MPSGB_H */
