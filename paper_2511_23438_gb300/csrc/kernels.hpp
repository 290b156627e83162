// Host-callable wrappers of the library's CUDA kernels (internal API).
#pragma once
#include <functional>

#include "common.cuh"

namespace mpsgb {

// ---------------------------------------------------------------- graph replay (graph.cu)
// Identity of a fixed launch sequence: what it does (tag), its sizes and its buffers and stream.
struct GraphKey {
  long long v[12];
  bool operator==(const GraphKey& o) const {
    for (int i = 0; i < 12; ++i)
      if (v[i] != o.v[i]) return false;
    return true;
  }
};
// Issue the launch sequence `issue` (which returns 0, or non-zero on a failed call) on st: on a
// capturable stream it is recorded once per key as a CUDA graph and replayed; otherwise issued
// directly.  Returns 0, or -4 if a call or the capture failed.
// Runs issue(s) once: directly on st (s = st), or the first time for `key` recorded as a CUDA graph on
// a capture stream private to the calling thread (s = that stream, so that no other thread's work on
// st can enter the recording) and launched on st; later calls with the same key launch the graph.
int replay_or_issue(cudaStream_t st, const GraphKey& key, const std::function<int(cudaStream_t)>& issue);
// graph cache of one handle; GraphScope makes it the calling thread's cache for its lifetime
struct GraphCache;
GraphCache* new_graph_cache();
void free_graph_cache(GraphCache* c);  // waits for the cached graphs' last launches
struct GraphScope {
  explicit GraphScope(GraphCache* c);
  ~GraphScope();
  GraphCache* prev;
};
// graph replay for the calling host thread (on by default)
void set_graphs_enabled(bool on);
bool graphs_enabled();

// ---------------------------------------------------------------- GEMM (gemm.cu)
template <typename R>
void gemm(cudaStream_t st, int M, int N, int K, Cx<R> alpha, View<R> A, View<R> B, Cx<R> beta, View<R> C,
          int batch = 1, long long sA = 0, long long sB = 0, long long sC = 0);

// As gemm (batch 1), with K split over CTAs into the workspace ws (ws_elems complex elements) and
// reduced in a fixed order when the output alone has too few tiles to fill the GPU.
template <typename R>
void gemm_splitk(cudaStream_t st, int M, int N, int K, Cx<R> alpha, View<R> A, View<R> B, Cx<R> beta, View<R> C,
                 Cx<R>* ws, size_t ws_elems);
// C = alpha op(A) op(B) + beta C on row-major real matrices (op(X) = X^T if tX); ws (ws_elems
// elements, may be null) lets long-K products split K over CTAs with a fixed-order reduction.
template <typename R>
void rgemm(cudaStream_t st, int M, int N, int K, R alpha, const R* A, long long lda, bool ta, const R* B, long long ldb,
           bool tb, R beta, R* C, long long ldc, R* ws, size_t ws_elems);

// ---------------------------------------------------------------- eigensolver (eig.cu)
// Hermitian eigendecomposition of `batch` n x n matrices (row-major, leading dim
// lda, batch stride sA, read only).  Eigenvalues go to w (descending, stride sw),
// eigenvectors to the columns of V (row-major n x n, leading dim ldv, stride sV):
// A = V diag(w) V^H.  n <= 32: warp-level cyclic Jacobi; 33 <= n <= 64: blocked Jacobi
// (16-wide blocks, 32 x 32 pair problems solved by warps, tile updates of the full matrix);
// n >= kTridiagMinN: Householder tridiagonalisation, bisection and inverse iteration on the
// unreduced blocks, orthonormalisation and back-transformation (tridiag.cu).
// Returns the number of outer sweeps (1 for the tridiagonal route), or < 0: -1 Jacobi sweep
// limit hit, -2 a bounded grid barrier of the reduction timed out, -3 the eigenvectors of the
// tridiagonal matrix could not be orthonormalised (dependent vectors), -4 launch or device error.
// nvec > 0: all eigenvalues, but on the tridiagonal route only the eigenvectors of the nvec
// largest (the first nvec columns of V; the other columns are left undefined).
size_t eigh_workspace_bytes(int n, int batch, int real_bytes);
// n above which eigh() uses the Householder-tridiagonal solver (tridiag.cu) instead of Jacobi
constexpr int kTridiagMinN = 65;
size_t tri_workspace_bytes(int n, int real_bytes);
template <typename R>
int eigh_tridiag(cudaStream_t st, int n, const Cx<R>* A, long long lda, R* w, Cx<R>* V, long long ldv, void* workspace,
                 int nvec = 0);
template <typename R>
int eigh(cudaStream_t st, int n, const Cx<R>* A, long long lda, long long sA, R* w, long long sw, Cx<R>* V,
         long long ldv, long long sV, int batch, void* workspace, int nvec = 0);

// ---------------------------------------------------------------- Cholesky (chol.cu)
// A = C C^H for the n x n Hermitian matrix A (row-major, lda), in place: A becomes the lower-
// triangular C (strict upper triangle zeroed) and Ci (row-major, ldi) the lower-triangular C^{-1}.
// ws: chol_workspace_bytes(n).  flag (device int) is set non-zero if a pivot fell to or below
// rel * A_jj (its column's diagonal): A is then treated as numerically singular.  Returns 0, or -4
// for a launch error.  Does not synchronise.
size_t chol_workspace_bytes(int n, int real_bytes);
template <typename R>
int chol_inv(cudaStream_t st, int n, Cx<R>* A, long long lda, Cx<R>* Ci, long long ldi, double rel, void* ws,
             int* flag);

// ---------------------------------------------------------------- Jacobi SVD (svd.cu)
// SVD of `batch` p x q complex matrices X (row-major, leading dim ldx, batch stride sX; read only) by
// one-sided Jacobi rotations of the rows: X = U diag(s) Vh with s descending (FP64, device s and/or
// host s_host, either may be null), Vh (p x q, orthonormal rows where s > 0, zero rows where s == 0)
// and U (p x p, unitary); Vh or U may be null.  Returns the number of sweeps, -1 if the sweep limit
// was reached, -2 if a bounded grid barrier timed out, -4 for a launch or device error, -5 if a
// singular value came out non-finite (non-finite input; s_host must be given to detect it).
// Synchronises the stream.
size_t svd_rows_workspace_bytes(int p, int q, int batch, int real_bytes);
template <typename R>
int svd_rows(cudaStream_t st, int p, int q, const Cx<R>* X, long long ldx, double* s, double* s_host, Cx<R>* Vh,
             long long ldvh, Cx<R>* U, long long ldu, void* workspace, int batch = 1, long long sX = 0,
             long long sVh = 0, long long sU = 0);
// Block expanded by the rank-2 MPO cos(phi) I I - i sin(phi) Z_i Z_j (the bond index of the MPO is the
// slow half of a doubled bond): mode 0 block p (l, d, r) -> (l, d, 2r); mode 1 a block in between
// (l, d, r) -> (2l, d, 2r), block diagonal; mode 2 block q (l, d, r) -> (2l, d, r).  shift: position
// of the gate's qubit in the physical index counted from the least significant bit.
template <typename R>
void mpo_expand(cudaStream_t st, int mode, int l, int d, int r, const Cx<R>* in, Cx<R>* out, double phi, int shift);
// X[i, :cols] *= c s[i] for i < rows (s: device FP64)
template <typename R>
void scale_rows(cudaStream_t st, int rows, int cols, Cx<R>* X, long long ld, const double* s, double c);
// theta (l, da, db, r) *= exp(-i phi z_a z_b), z_a = 1 - 2 bit shift_a of the first physical index,
// z_b likewise of the second (the gate of a two-site update)
template <typename R>
void two_site_phase(cudaStream_t st, int l, int da, int db, int r, Cx<R>* th, double phi, int shift_a, int shift_b);
// a 4 x 4 two-qubit gate (row-major, index 2 x + y with x the first qubit's bit), by value
struct Gate4 {
  double re[16], im[16];
};
template <typename R>
void two_site_gate(cudaStream_t st, int l, int da, int db, int r, Cx<R>* th, const Gate4& u, int shift_a, int shift_b);
// X[:rows, j] *= c s[j] for j < cols (s: device FP64)
template <typename R>
void scale_cols(cudaStream_t st, int rows, int cols, Cx<R>* X, long long ld, const double* s, double c);

// ---------------------------------------------------------------- tensor-core split GEMM (tcgemm.cu)
// C = alpha op(A) op(B) + beta C on complex64 views with 2-term splits on tcgen05: BF16
// (kind::f16) or, with tf32, TF32 (kind::tf32); FP32 accumulation.  ws: device workspace of
// tc_gemm_workspace_bytes(M, N, K, tf32) bytes; d_err: device word set non-zero if a bounded wait
// of the kernel ran out.  Returns 0, or < 0 if the workspace is too small / the tensor maps
// could not be built.
size_t tc_gemm_workspace_bytes(long long M, long long N, long long K, bool tf32);
int tc_gemm(cudaStream_t st, int M, int N, int K, c64 alpha, View<float> A, View<float> B, c64 beta, View<float> C,
            void* ws, size_t ws_bytes, int* d_err, bool tf32);
int eig_selftest(int n, int fp64, int kind, unsigned long long seed, double* out);
int svd_selftest(int p, int q, int fp64, const double* X, double* s, double* out);
int eigh_noalloc(int n, int fp64, const void* A, long long lda, void* w, void* V, long long ldv, cudaStream_t st);
int tc_selftest(int M, int N, int K, int mode, unsigned long long seed, double* rel_err);

// ---------------------------------------------------------------- small kernels (local.cu)
// blk[a, s, b] <- sum_t U[s, t] blk[a, t, b] for a block of shape (l, d, r); U is d x d row-major on device
template <typename R>
void apply_phys(cudaStream_t st, Cx<R>* blk, int l, int d, int r, const Cx<R>* U);
// product state of Eq. initial_state for one block of k qubits: (1, 2^k, 1)
template <typename R>
void init_product(cudaStream_t st, Cx<R>* blk, int k, double c, double s);
// C = alpha * C over a view
template <typename R>
void scale_view(cudaStream_t st, int M, int N, Cx<R> alpha, View<R> C, int batch = 1, long long sC = 0);
// C = a * X + b * Y (element-wise on M x N views; C may alias X or Y element-for-element)
template <typename R>
void axpby(cudaStream_t st, int M, int N, Cx<R> a, View<R> X, Cx<R> b, View<R> Y, View<R> C);
// copy / convert between precisions: dst(i, j) = src(i, j)
template <typename Rd, typename Rs>
void copy_view(cudaStream_t st, int M, int N, View<Rs> src, View<Rd> dst);
// M[:, j] *= s[j]^p  for p in {+1/2, -1/2} (p2 = +1 or -1), columns j < ncol; rows < nrow
template <typename R>
void scale_cols_pow(cudaStream_t st, int nrow, int ncol, Cx<R>* M, long long ld, const R* s, int p2);
// Z = Y1 + w(s) * Y0 over a block-shaped tensor (l, d, r) with w(s) = sum of z over the block's qubits
// (mode 1), its square (mode 2) or the bit-flip sum X (mode 3, Y1 may be null).
template <typename R>
void weighted_phys(cudaStream_t st, int mode, int l, int d, int r, const Cx<R>* Y1, const Cx<R>* Y0, Cx<R>* Z,
                   double coef);
// Z = Y1 + coef * O(Y0) over (l, d, r): O = identity (mode 0) or sum_t s_t X_t over the block's
// qubits (mode 1; s_t = -1 where bit t of negmask is set, bit 0 = least significant); Y1 may be null
template <typename R>
void stag_x(cudaStream_t st, int mode, int l, int d, int r, const Cx<R>* Y1, const Cx<R>* Y0, Cx<R>* Z, double coef,
            int negmask);
// sum_ij conj(X_ij) * Y_ij accumulated in FP64 into out[0..1] (re, im) -- device pointer
template <typename R>
void dot_fp64(cudaStream_t st, long long n, const Cx<R>* X, const Cx<R>* Y, double* out);
// diagonal sum of an n x n row-major matrix into out (FP64)
template <typename R>
void trace_fp64(cudaStream_t st, int n, const Cx<R>* A, long long lda, double* out);
// set to identity / zero
template <typename R>
void set_identity(cudaStream_t st, int n, Cx<R>* A, long long lda);
template <typename R>
void set_zero(cudaStream_t st, long long count, Cx<R>* A);
// Build the 2r x 2r right environment of an inter-block gate from Y+ and Y- (r x r each):
//   E = [[Y+ + Y-, e^{-2i phi} Y+ + e^{2i phi} Y-], [h.c., Y+ + Y-]]
template <typename R>
void env_from_split_grams(cudaStream_t st, int r, const Cx<R>* Yp, const Cx<R>* Ym, double phi, Cx<R>* E);
// Assemble [[E00, E01], [E01^H, E00]] (2r x 2r) from two r x r blocks
template <typename R>
void env_assemble(cudaStream_t st, int r, const Cx<R>* E00, const Cx<R>* E01, Cx<R>* E);
// Place two r x r matrices on the diagonal of a 2r x 2r zero matrix
template <typename R>
void block_diag2(cudaStream_t st, int r, const Cx<R>* P, const Cx<R>* Q, Cx<R>* G);

}  // namespace mpsgb
