// Cholesky factorisation G = C C^H of a Hermitian positive-definite matrix together with the
// inverse C^{-1}, for the Gram matrices of the Gram-route truncation core and of the centre moves
// (complex64 forms).
//
// In the Gram route a Gram matrix only has to be written as G = Gs Gs^H with an invertible Gs: the
// Schmidt values across the bond are the eigenvalues of H = Gs^H E Gs, the new left isometry is
// L Gs^{-H} V_k and the carry (Gs V_k)^H / sqrt(kept), whatever Gs is; a centre move is the QR
// factorisation M = (M Gs^{-H}) Gs^H of the block.  The eigenvector factor U D^{1/2} needs a full
// Hermitian eigensolve of G; the Cholesky factor costs n^3 / 3 complex MACs and, with its inverse,
// turns every solve into one GEMM.  Both come from one recursion on halves (multiples of 32):
//   C11 = chol(G11), C21 = G21 C11^{-H}, C22 = chol(G22 - C21 C21^H),
//   C^{-1}: (C^{-1})_11 = C11^{-1}, (C^{-1})_22 = C22^{-1}, (C^{-1})_21 = -C22^{-1} C21 C11^{-1},
// whose products are GEMMs; a 32 x 32 diagonal block is factorised and inverted in shared memory.
// A pivot at or below rel * G_jj (the column's own diagonal entry) marks G as numerically singular:
// the caller then takes the eigenvector factor, which handles rank deficiency (structurally
// rank-deficient Grams occur at the chain ends).  The test is per column because Cholesky is
// invariant under diagonal scaling, also in rounding: its accuracy follows the condition of
// D^{-1/2} G D^{-1/2} (D = diag G), not that of G, and Gram matrices of blocks whose columns carry
// Schmidt values of many magnitudes are badly conditioned mostly through that scaling.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "common.cuh"
#include "kernels.hpp"

namespace mpsgb {

namespace {
constexpr int NB = 32;

// Factorise the nb x nb diagonal block at A (leading dim lda) in place (lower triangle = C_kk) and
// write its inverse (lower triangular) into Ci (leading dim ldi).  One CTA of NB x 8 threads.
// flag[0] is set if a pivot d_jj (before the square root) is <= thr[j].
template <typename R>
__global__ void chol_diag_kernel(int nb, Cx<R>* A, long long lda, Cx<R>* Ci, long long ldi, const double* thr,
                                 int* flag) {
  __shared__ Cx<R> S[NB][NB + 1];
  __shared__ Cx<R> I[NB][NB + 1];
  __shared__ int bad;
  const int tx = threadIdx.x, ty = threadIdx.y;  // tx: column 0..31, ty: 0..7
  if (tx == 0 && ty == 0) bad = 0;
  for (int i = ty; i < NB; i += 8) {
    S[i][tx] = (i < nb && tx < nb) ? A[(long long)i * lda + tx] : cmake<R>(i == tx ? R(1) : R(0), R(0));
    I[i][tx] = cmake<R>(0, 0);
  }
  __syncthreads();
  for (int j = 0; j < NB; ++j) {
    const R djj = S[j][j].x;  // pivot: real part of the updated diagonal
    if (j < nb && !((double)djj > thr[j]) && tx == 0 && ty == 0) bad = 1;
    const R d = sqrt(fmax(djj, (R)1e-30));
    __syncthreads();
    if (ty == 0 && tx > j) S[tx][j] = (R(1) / d) * S[tx][j];
    if (ty == 0 && tx == j) S[j][j] = cmake<R>(d, 0);
    __syncthreads();
    // trailing update of the lower triangle: S[i][l] -= S[i][j] conj(S[l][j]) for j < l <= i
    for (int i = j + 1 + ty; i < NB; i += 8)
      if (tx > j && tx <= i) S[i][tx] = S[i][tx] - S[i][j] * conj(S[tx][j]);
    __syncthreads();
  }
  // inverse of the lower-triangular S by forward substitution, one column per thread (ty == 0)
  if (ty == 0) {
    const int c = tx;
    for (int i = 0; i < NB; ++i) {
      Cx<R> acc = cmake<R>(i == c ? R(1) : R(0), R(0));
      for (int k = c; k < i; ++k) acc = acc - S[i][k] * I[k][c];
      I[i][c] = (R(1) / S[i][i].x) * acc;
    }
  }
  __syncthreads();
  for (int i = ty; i < nb; i += 8)
    if (tx <= i) {
      A[(long long)i * lda + tx] = S[i][tx];
      Ci[(long long)i * ldi + tx] = I[i][tx];
    }
  if (tx == 0 && ty == 0 && bad) atomicExch(flag, 1);
}

// per-column pivot thresholds thr[i] = rel * Re A_ii
template <typename R>
__global__ void diag_thr_kernel(int n, const Cx<R>* A, long long lda, double rel, double* thr) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    thr[i] = rel * (double)A[(long long)i * lda + i].x;
}

// zero the strict upper triangle of an n x n row-major matrix
template <typename R>
__global__ void zero_upper_kernel(int n, Cx<R>* A, long long lda) {
  const long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e - i * n;
    if (j > i) A[i * lda + j] = cmake<R>(0, 0);
  }
}

inline int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 65535LL * 8); }

// recursion of the file header on the n x n matrix A (in place) and its inverse Ci (lower part;
// the caller zeroes Ci first); T: scratch of at least n x (n/2 + 32) elements (leading dim ldt)
template <typename R>
void chol_rec(cudaStream_t st, int n, Cx<R>* A, long long lda, Cx<R>* Ci, long long ldi, const double* thr, int* flag,
              Cx<R>* T, long long ldt) {
  if (n <= NB) {
    chol_diag_kernel<R><<<1, dim3(NB, 8), 0, st>>>(n, A, lda, Ci, ldi, thr, flag);
    count_launch();
    return;
  }
  const int n1 = ((n / 2 + NB - 1) / NB) * NB, n2 = n - n1;
  const Cx<R> one = cmake<R>(1, 0), mone = cmake<R>(-1, 0), zero = cmake<R>(0, 0);
  Cx<R>* A21 = A + (long long)n1 * lda;
  Cx<R>* A22 = A21 + n1;
  Cx<R>* Ci21 = Ci + (long long)n1 * ldi;
  Cx<R>* Ci22 = Ci21 + n1;
  chol_rec<R>(st, n1, A, lda, Ci, ldi, thr, flag, T, ldt);
  // C21 = G21 C11^{-H}
  gemm<R>(st, n2, n1, n1, one, rowmajor<R>(A21, lda), transposed<R>(Ci, ldi, true), zero, rowmajor<R>(T, ldt));
  copy_view<R, R>(st, n2, n1, rowmajor<R>(T, ldt), rowmajor<R>(A21, lda));
  // G22 -= C21 C21^H
  gemm<R>(st, n2, n2, n1, mone, rowmajor<R>(A21, lda), transposed<R>(A21, lda, true), one, rowmajor<R>(A22, lda));
  chol_rec<R>(st, n2, A22, lda, Ci22, ldi, thr + n1, flag, T, ldt);
  // (C^{-1})_21 = -C22^{-1} (C21 C11^{-1})
  gemm<R>(st, n2, n1, n1, one, rowmajor<R>(A21, lda), rowmajor<R>(Ci, ldi), zero, rowmajor<R>(T, ldt));
  gemm<R>(st, n2, n1, n2, mone, rowmajor<R>(Ci22, ldi), rowmajor<R>(T, ldt), zero, rowmajor<R>(Ci21, ldi));
}
}  // namespace

size_t chol_workspace_bytes(int n, int real_bytes) {
  return 2 * (size_t)real_bytes * (size_t)n * (size_t)((n + 1) / 2 + NB) + sizeof(double) * (size_t)n + 512;
}

// the whole factorisation as one launch sequence (no host decision inside)
template <typename R>
int chol_issue(cudaStream_t st, int n, Cx<R>* A, long long lda, Cx<R>* Ci, long long ldi, double rel, void* ws,
               int* flag) {
  Cx<R>* T = static_cast<Cx<R>*>(ws);
  const long long ldt = (n + 1) / 2 + NB;
  double* thr = reinterpret_cast<double*>(static_cast<char*>(ws) + sizeof(Cx<R>) * (size_t)n * ldt);
  if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return -4;
  diag_thr_kernel<R><<<(n + 255) / 256, 256, 0, st>>>(n, A, lda, rel, thr);
  count_launch();
  if (cudaMemset2DAsync(Ci, sizeof(Cx<R>) * ldi, 0, sizeof(Cx<R>) * n, n, st) != cudaSuccess) return -4;
  chol_rec<R>(st, n, A, lda, Ci, ldi, thr, flag, T, ldt);
  zero_upper_kernel<R><<<blocks_for((long long)n * n), 256, 0, st>>>(n, A, lda);
  count_launch();
  return 0;
}

template <typename R>
int chol_inv(cudaStream_t st, int n, Cx<R>* A, long long lda, Cx<R>* Ci, long long ldi, double rel, void* ws,
             int* flag) {
  GemmSite site(KT_GEMM_CHOL);
  // a fixed launch sequence for given sizes and buffers: replayed as a CUDA graph where possible
  GraphKey key{{1, n, (long long)sizeof(R), (long long)(uintptr_t)A, lda, (long long)(uintptr_t)Ci, ldi,
                (long long)(uintptr_t)ws, (long long)(uintptr_t)flag, (long long)(rel * 1e18),
                (long long)(uintptr_t)st, 0}};
  return replay_or_issue(st, key, [&](cudaStream_t cs) { return chol_issue<R>(cs, n, A, lda, Ci, ldi, rel, ws, flag); });
}

template int chol_inv<float>(cudaStream_t, int, c64*, long long, c64*, long long, double, void*, int*);
template int chol_inv<double>(cudaStream_t, int, z128*, long long, z128*, long long, double, void*, int*);

}  // namespace mpsgb
