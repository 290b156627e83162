// Hermitian eigensolver: cyclic parallel (round-robin) two-sided Jacobi.
//
// n <= 32 : one warp per matrix, the matrix in shared memory, rotations applied
//           column-wise then row-wise each round (16 disjoint pairs per round).
// n  > 32 : blocked Jacobi.  Indices are cut into 16-wide blocks; a tournament
//           pairs the blocks; each pair's 32 x 32 sub-problem is diagonalised by
//           one warp (the n <= 32 solver), and the resulting 32 x 32 unitaries are
//           applied to the whole matrix (tile updates Q_P^H H_{PP'} Q_P') and to
//           the accumulated eigenvectors.  Sweeps repeat until no pair needs a
//           rotation.
// Rotation rule for a pair (p, q) with entries a = H_pp, c = H_qq, b = H_pq:
// rotate iff |b| > tol * max(sqrt(|a c|), floor) with tol = 8 eps and floor =
// ||H||_F.  As sqrt(|a c|) <= ||H||_F this is a normwise criterion: the sweep stops
// when every off-diagonal entry is below 8 eps ||H||_F, so eigenvalues carry an
// absolute error of order eps ||H|| (rounding noise of the tile updates cannot
// keep the sweeps alive).
// The rotation G = [[cs, sn], [-sn e^{-i beta}, cs e^{-i beta}]], b = |b| e^{i beta},
// with t = sign(z) / (|z| + sqrt(1 + z^2)), z = (c - a) / (2 |b|), zeroes b.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.hpp"

namespace mpsgb {

namespace {
constexpr int LDS = 33;  // padded leading dimension of 32 x 32 shared tiles

__host__ __device__ __forceinline__ int slot_player(int slot, int r, int nb) {
  return slot == 0 ? 0 : 1 + (slot - 1 + r) % (nb - 1);
}

template <typename R> struct Rot { R cs, sn; Cx<R> ph; };

template <typename R> __device__ __forceinline__ R eps_of();
template <typename R> __device__ __forceinline__ R tol_of() { return R(8) * eps_of<R>(); }
// floor of the rotation rule relative to ||H||_F (normwise rule in both precisions: with the
// relative rule the rounding noise of the tile updates keeps re-creating tiny couplings and the
// sweeps never stop)
template <typename R> __device__ __forceinline__ R floor_scale() { return R(1); }
template <> __device__ __forceinline__ double eps_of<double>() { return 2.220446049250313e-16; }
template <> __device__ __forceinline__ float eps_of<float>() { return 1.1920929e-7f; }

template <typename R>
__device__ __forceinline__ bool jacobi_rot(R a, R c, Cx<R> b, R tol, R floor_, Rot<R>& rt) {
  R ab = sqrt(abs2(b));
  R ref = sqrt(fabs(a * c));
  if (ref < floor_) ref = floor_;
  if (!(ab > tol * ref)) { rt.cs = 1; rt.sn = 0; rt.ph = cmake<R>(1, 0); return false; }
  R z = (c - a) / (R(2) * ab);
  R t;
  if (fabs(z) > R(1) / (R(16) * eps_of<R>())) t = R(0.5) / z;
  else t = (z >= 0 ? R(1) : R(-1)) / (fabs(z) + sqrt(z * z + R(1)));
  R cs = R(1) / sqrt(t * t + R(1));
  rt.cs = cs;
  rt.sn = t * cs;
  rt.ph = cmake<R>(b.x / ab, -b.y / ab);
  return true;
}

// Full cyclic Jacobi of the 32 x 32 Hermitian matrix S (shared, ld LDS) by one warp;
// Q accumulates the rotations (S_in = Q S_out Q^H).  Returns whether any rotation happened.
template <typename R>
__device__ bool warp_jacobi(Cx<R>* S, Cx<R>* Q, R tol, R floor_, int max_sweeps, Rot<R>* rots, int* pq) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < 32; ++i) Q[i * LDS + lane] = cmake<R>(i == lane ? R(1) : R(0), R(0));
  bool any = false;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < 31; ++r) {
      __syncwarp();
      if (lane < 16) {
        int p = slot_player(lane, r, 32), q = slot_player(31 - lane, r, 32);
        Rot<R> rt;
        rotated |= jacobi_rot(S[p * LDS + p].x, S[q * LDS + q].x, S[p * LDS + q], tol, floor_, rt) ? 1 : 0;
        rots[lane] = rt;
        pq[2 * lane] = p;
        pq[2 * lane + 1] = q;
      }
      __syncwarp();
      for (int k = 0; k < 16; ++k) {  // columns: S <- S G, Q <- Q G (lane owns a row)
        Rot<R> rt = rots[k];
        if (rt.sn == R(0)) continue;
        int p = pq[2 * k], q = pq[2 * k + 1];
        Cx<R> x = S[lane * LDS + p], y = S[lane * LDS + q] * rt.ph;
        S[lane * LDS + p] = rt.cs * x - rt.sn * y;
        S[lane * LDS + q] = rt.sn * x + rt.cs * y;
        x = Q[lane * LDS + p]; y = Q[lane * LDS + q] * rt.ph;
        Q[lane * LDS + p] = rt.cs * x - rt.sn * y;
        Q[lane * LDS + q] = rt.sn * x + rt.cs * y;
      }
      __syncwarp();
      for (int k = 0; k < 16; ++k) {  // rows: S <- G^H S (lane owns a column)
        Rot<R> rt = rots[k];
        if (rt.sn == R(0)) continue;
        int p = pq[2 * k], q = pq[2 * k + 1];
        Cx<R> x = S[p * LDS + lane], y = conj(rt.ph) * S[q * LDS + lane];
        S[p * LDS + lane] = rt.cs * x - rt.sn * y;
        S[q * LDS + lane] = rt.sn * x + rt.cs * y;
      }
      __syncwarp();
      if (lane < 16 && rots[lane].sn != R(0)) {
        int p = pq[2 * lane], q = pq[2 * lane + 1];
        S[p * LDS + q] = cmake<R>(0, 0);
        S[q * LDS + p] = cmake<R>(0, 0);
        S[p * LDS + p].y = 0;
        S[q * LDS + q].y = 0;
      }
    }
    rotated = __any_sync(0xffffffffu, rotated);
    if (!rotated) break;
    any = true;
  }
  __syncwarp();
  return any;
}

// Same sweep as warp_jacobi with 128 threads: per round the 16 rotations are computed by
// threads 0..15, then the 32 x 16 (row, pair) column updates and the 32 x 16 (column, pair)
// row updates are spread over all threads.
template <typename R>
__device__ bool cta_jacobi32(Cx<R>* S, Cx<R>* Q, R tol, R floor_, int max_sweeps, Rot<R>* rots, int* pq,
                             int* rotated_sm) {
  const int t = threadIdx.x;
  for (int e = t; e < 1024; e += blockDim.x) {
    int i = e >> 5, j = e & 31;
    Q[i * LDS + j] = cmake<R>(i == j ? R(1) : R(0), R(0));
  }
  bool any = false;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (t == 0) *rotated_sm = 0;
    __syncthreads();
    for (int r = 0; r < 31; ++r) {
      if (t < 16) {
        int p = slot_player(t, r, 32), q = slot_player(31 - t, r, 32);
        Rot<R> rt;
        if (jacobi_rot(S[p * LDS + p].x, S[q * LDS + q].x, S[p * LDS + q], tol, floor_, rt)) *rotated_sm = 1;
        rots[t] = rt;
        pq[2 * t] = p;
        pq[2 * t + 1] = q;
      }
      __syncthreads();
      for (int it = t; it < 512; it += blockDim.x) {  // columns: S <- S G, Q <- Q G
        const int row = it & 31, k = it >> 5;
        Rot<R> rt = rots[k];
        if (rt.sn == R(0)) continue;
        const int p = pq[2 * k], q = pq[2 * k + 1];
        Cx<R> x = S[row * LDS + p], y = S[row * LDS + q] * rt.ph;
        S[row * LDS + p] = rt.cs * x - rt.sn * y;
        S[row * LDS + q] = rt.sn * x + rt.cs * y;
        x = Q[row * LDS + p]; y = Q[row * LDS + q] * rt.ph;
        Q[row * LDS + p] = rt.cs * x - rt.sn * y;
        Q[row * LDS + q] = rt.sn * x + rt.cs * y;
      }
      __syncthreads();
      for (int it = t; it < 512; it += blockDim.x) {  // rows: S <- G^H S
        const int col = it & 31, k = it >> 5;
        Rot<R> rt = rots[k];
        if (rt.sn == R(0)) continue;
        const int p = pq[2 * k], q = pq[2 * k + 1];
        Cx<R> x = S[p * LDS + col], y = conj(rt.ph) * S[q * LDS + col];
        S[p * LDS + col] = rt.cs * x - rt.sn * y;
        S[q * LDS + col] = rt.sn * x + rt.cs * y;
      }
      __syncthreads();
      if (t < 16 && rots[t].sn != R(0)) {
        int p = pq[2 * t], q = pq[2 * t + 1];
        S[p * LDS + q] = cmake<R>(0, 0);
        S[q * LDS + p] = cmake<R>(0, 0);
        S[p * LDS + p].y = 0;
        S[q * LDS + q].y = 0;
      }
      __syncthreads();
    }
    const bool rot = *rotated_sm != 0;
    __syncthreads();
    if (!rot) break;
    any = true;
  }
  return any;
}

// ---- n <= 32: one warp per matrix, solve + sort + write
template <typename R>
__global__ void __launch_bounds__(32) eig_small_kernel(int n, const Cx<R>* A, long long lda, long long sA, R* w,
                                                        long long sw, Cx<R>* V, long long ldv, long long sV,
                                                        const double* fro) {
  __shared__ Cx<R> S[32 * LDS];
  __shared__ Cx<R> Q[32 * LDS];
  __shared__ Rot<R> rots[16];
  __shared__ int pq[32];
  __shared__ R dg[32];
  const int lane = threadIdx.x;
  const long long z = blockIdx.x;
  const Cx<R>* Ap = A + z * sA;
  for (int i = 0; i < 32; ++i)
    S[i * LDS + lane] = (i < n && lane < n) ? Ap[i * lda + lane] : cmake<R>(0, 0);
  __syncwarp();
  R fl = (R)sqrt(fro[z]) * floor_scale<R>();
  warp_jacobi<R>(S, Q, tol_of<R>(), fl, 40, rots, pq);
  dg[lane] = S[lane * LDS + lane].x;
  __syncwarp();
  if (lane < n) {
    R d = dg[lane];
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += (dg[j] > d || (dg[j] == d && j < lane)) ? 1 : 0;
    w[z * sw + rank] = d;
    Cx<R>* Vp = V + z * sV;
    for (int i = 0; i < n; ++i) Vp[i * ldv + rank] = Q[i * LDS + lane];
  }
}

// ---- blocked solver kernels
// Working copies: H (np x np), Vw (np x np), Qs (npairs x 32 x 32) per problem.
template <typename R>
__global__ void blk_init_kernel(int n, int np, const Cx<R>* A, long long lda, long long sA, Cx<R>* H, Cx<R>* Vw) {
  long long tot = (long long)np * np;
  const long long z = blockIdx.y;
  const Cx<R>* Ap = A + z * sA;
  Cx<R>* Hp = H + z * tot;
  Cx<R>* Vp = Vw + z * tot;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / np), j = (int)(e - (long long)i * np);
    Hp[e] = (i < n && j < n) ? Ap[i * lda + j] : cmake<R>(0, 0);
    Vp[e] = cmake<R>(i == j ? R(1) : R(0), R(0));
  }
}

template <typename R>
__global__ void __launch_bounds__(128) blk_pair_kernel(int np, int nb, int round, Cx<R>* H, Cx<R>* Qs, int* flag,
                                                        int* ident, const double* fro) {
  __shared__ Cx<R> S[32 * LDS];
  __shared__ Cx<R> Q[32 * LDS];
  __shared__ Rot<R> rots[16];
  __shared__ int pq[32];
  __shared__ int rotated_sm;
  const int t = threadIdx.x;
  const int pair = blockIdx.x;
  const long long z = blockIdx.y;
  const int I = slot_player(pair, round, nb), J = slot_player(nb - 1 - pair, round, nb);
  Cx<R>* Hp = H + z * (long long)np * np;
  // sub-problem indices: 16 of block I then 16 of block J
  for (int e = t; e < 1024; e += blockDim.x) {
    int i = e >> 5, j = e & 31;
    int gi = i < 16 ? I * 16 + i : J * 16 + (i - 16);
    int gj = j < 16 ? I * 16 + j : J * 16 + (j - 16);
    S[i * LDS + j] = Hp[(long long)gi * np + gj];
  }
  __syncthreads();
  R fl = (R)sqrt(fro[z]) * floor_scale<R>();
  bool any = cta_jacobi32<R>(S, Q, tol_of<R>(), fl, 8, rots, pq, &rotated_sm);
  Cx<R>* Qp = Qs + (z * (nb / 2) + pair) * 1024;
  if (any)
    for (int e = t; e < 1024; e += blockDim.x) Qp[e] = Q[(e >> 5) * LDS + (e & 31)];
  if (t == 0) {
    ident[z * (nb / 2) + pair] = any ? 0 : 1;
    if (any) atomicOr(flag + z, 1);
  }
}

// One launch applies the round's rotations: work items [0, np2 * np2) are the tiles
// H_{PP'} <- Q_P^H H_{PP'} Q_P' (P <= P', mirrored for P < P'); the remaining items are
// 32-row slabs of the eigenvector matrix, Vw[rows, cols(P)] <- Vw[rows, cols(P)] Q_P.
// Pairs whose rotation is the identity are skipped.
template <typename R>
__global__ void __launch_bounds__(256) blk_update_kernel(int np, int nb, int round, Cx<R>* H, Cx<R>* Vw,
                                                         const Cx<R>* Qs, const int* ident) {
  const int npairs = nb / 2;
  const long long z = blockIdx.y;
  const int item = blockIdx.x;
  __shared__ Cx<R> T[32 * LDS];
  __shared__ Cx<R> M[32 * LDS];
  const int tid = threadIdx.x;
  const int* id = ident + z * npairs;
  if (item < npairs * npairs) {
    const int P = item / npairs, P2 = item - P * npairs;
    if (P > P2 || (id[P] && id[P2])) return;
    Cx<R>* Hp = H + z * (long long)np * np;
    const Cx<R>* QP = Qs + (z * npairs + P) * 1024;
    const Cx<R>* QP2 = Qs + (z * npairs + P2) * 1024;
    const int I = slot_player(P, round, nb), J = slot_player(nb - 1 - P, round, nb);
    const int I2 = slot_player(P2, round, nb), J2 = slot_player(nb - 1 - P2, round, nb);
    for (int e = tid; e < 1024; e += 256) {
      int i = e >> 5, j = e & 31;
      int gi = i < 16 ? I * 16 + i : J * 16 + (i - 16);
      int gj = j < 16 ? I2 * 16 + j : J2 * 16 + (j - 16);
      T[i * LDS + j] = Hp[(long long)gi * np + gj];
      M[i * LDS + j] = id[P2] ? cmake<R>(i == j ? R(1) : R(0), R(0)) : QP2[e];
    }
    __syncthreads();
    Cx<R> x[4];
    for (int u = 0; u < 4; ++u) {  // X = T Q_P'
      int e = tid + 256 * u, i = e >> 5, j = e & 31;
      Cx<R> acc = cmake<R>(0, 0);
#pragma unroll 8
      for (int k = 0; k < 32; ++k) cfma(acc, T[i * LDS + k], M[k * LDS + j]);
      x[u] = acc;
    }
    __syncthreads();
    for (int u = 0; u < 4; ++u) {
      int e = tid + 256 * u, i = e >> 5, j = e & 31;
      T[i * LDS + j] = x[u];
      M[i * LDS + j] = id[P] ? cmake<R>(i == j ? R(1) : R(0), R(0)) : QP[e];
    }
    __syncthreads();
    for (int u = 0; u < 4; ++u) {  // Y = Q_P^H X
      int e = tid + 256 * u, i = e >> 5, j = e & 31;
      Cx<R> acc = cmake<R>(0, 0);
#pragma unroll 8
      for (int k = 0; k < 32; ++k) cfma(acc, conj(M[k * LDS + i]), T[k * LDS + j]);
      int gi = i < 16 ? I * 16 + i : J * 16 + (i - 16);
      int gj = j < 16 ? I2 * 16 + j : J2 * 16 + (j - 16);
      Hp[(long long)gi * np + gj] = acc;
      if (P != P2) Hp[(long long)gj * np + gi] = conj(acc);
    }
  } else {
    const int v = item - npairs * npairs;
    const int P = v % npairs, rc = v / npairs;
    if (id[P]) return;
    Cx<R>* Vp = Vw + z * (long long)np * np;
    const Cx<R>* QP = Qs + (z * npairs + P) * 1024;
    const int I = slot_player(P, round, nb), J = slot_player(nb - 1 - P, round, nb);
    for (int e = tid; e < 1024; e += 256) {
      int i = e >> 5, j = e & 31;
      int gj = j < 16 ? I * 16 + j : J * 16 + (j - 16);
      T[i * LDS + j] = Vp[(long long)(rc * 32 + i) * np + gj];
      M[i * LDS + j] = QP[e];
    }
    __syncthreads();
    for (int u = 0; u < 4; ++u) {
      int e = tid + 256 * u, i = e >> 5, j = e & 31;
      Cx<R> acc = cmake<R>(0, 0);
#pragma unroll 8
      for (int k = 0; k < 32; ++k) cfma(acc, T[i * LDS + k], M[k * LDS + j]);
      int gj = j < 16 ? I * 16 + j : J * 16 + (j - 16);
      Vp[(long long)(rc * 32 + i) * np + gj] = acc;
    }
  }
}

// diagonal -> descending eigenvalues (rank sort, ties by index) and column gather
template <typename R>
__global__ void __launch_bounds__(1024) blk_finish_kernel(int n, int np, const Cx<R>* H, const Cx<R>* Vw, R* w,
                                                          long long sw, Cx<R>* V, long long ldv, long long sV,
                                                          int* perm_ws) {
  extern __shared__ unsigned char smem_raw[];
  R* dg = reinterpret_cast<R*>(smem_raw);
  const long long z = blockIdx.x;
  const Cx<R>* Hp = H + z * (long long)np * np;
  const Cx<R>* Vp = Vw + z * (long long)np * np;
  int* perm = perm_ws + z * np;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dg[i] = Hp[(long long)i * np + i].x;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    R d = dg[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += (dg[j] > d || (dg[j] == d && j < i)) ? 1 : 0;
    w[z * sw + rank] = d;
    perm[rank] = i;
  }
  __syncthreads();
  Cx<R>* Vo = V + z * sV;
  long long tot = (long long)n * n;
  for (long long e = threadIdx.x; e < tot; e += blockDim.x) {
    int i = (int)(e / n), j = (int)(e - (long long)i * n);
    Vo[(long long)i * ldv + j] = Vp[(long long)i * np + perm[j]];
  }
}

template <typename R>
__global__ void fro2_kernel(int n, const Cx<R>* A, long long lda, long long sA, double* out) {
  const long long z = blockIdx.x;
  const Cx<R>* Ap = A + z * sA;
  double acc = 0;
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    int i = (int)(e / n), j = (int)(e - (long long)i * n);
    Cx<R> v = Ap[i * lda + j];
    acc += (double)v.x * v.x + (double)v.y * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double s[32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += s[i];
    out[z] = t;
  }
}

inline int padded(int n) { return ((n + 31) / 32) * 32; }
}  // namespace

size_t eigh_workspace_bytes(int n, int batch, int real_bytes) {
  if (n >= kTridiagMinN) return tri_workspace_bytes(n, real_bytes) + 4096;
  size_t c = 2 * (size_t)real_bytes;
  int np = padded(n);
  size_t b = 0;
  b += (size_t)batch * np * np * c * 2;           // H, Vw
  b += (size_t)batch * (np / 32) * 1024 * c;       // Qs
  b += (size_t)batch * np * sizeof(int);           // perm
  b += (size_t)batch * (sizeof(int) + sizeof(double)) + 256;  // flags, norms
  b += (size_t)batch * (np / 32) * sizeof(int) + 256;         // identity flags
  return b + 1024;
}

template <typename R>
int eigh(cudaStream_t st, int n, const Cx<R>* A, long long lda, long long sA, R* w, long long sw, Cx<R>* V,
         long long ldv, long long sV, int batch, void* workspace, int nvec) {
  GemmSite site(KT_GEMM_EIG);
  if (n <= 0 || batch <= 0) return 0;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  auto take = [&](size_t bytes) { unsigned char* p = ws; ws += (bytes + 255) & ~size_t(255); return p; };
  if (n >= kTridiagMinN) {  // Householder tridiagonal route, one problem at a time
    for (int b = 0; b < batch; ++b) {
      int r = eigh_tridiag<R>(st, n, A + b * sA, lda, w + b * sw, V + b * sV, ldv, ws, nvec);
      if (r < 0) return r;
    }
    return 1;
  }
  // Jacobi routes: squared Frobenius norms set the convergence tolerances
  double* fro = reinterpret_cast<double*>(take(sizeof(double) * batch));
  fro2_kernel<R><<<batch, 256, 0, st>>>(n, A, lda, sA, fro);
  count_launch();
  if (n <= 32) {
    kt_begin(KT_EIG_SMALL, st);
    eig_small_kernel<R><<<batch, 32, 0, st>>>(n, A, lda, sA, w, sw, V, ldv, sV, fro);
    kt_end(KT_EIG_SMALL, st);
    count_launch();
    return 1;
  }
  const int np = padded(n), nb = np / 16, npairs = nb / 2;
  Cx<R>* H = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)batch * np * np));
  Cx<R>* Vw = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)batch * np * np));
  Cx<R>* Qs = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)batch * npairs * 1024));
  int* perm = reinterpret_cast<int*>(take(sizeof(int) * (size_t)batch * np));
  int* flag = reinterpret_cast<int*>(take(sizeof(int) * batch));
  int* ident = reinterpret_cast<int*>(take(sizeof(int) * (size_t)batch * npairs));
  {
    long long tot = (long long)np * np;
    dim3 g((unsigned)((tot + 255) / 256 > 4096 ? 4096 : (tot + 255) / 256), batch);
    blk_init_kernel<R><<<g, 256, 0, st>>>(n, np, A, lda, sA, H, Vw);
    count_launch();
  }
  int sweeps = -1;
  // pinned host copy of the per-problem "rotated" flags, kept per host thread and released when
  // the thread ends
  struct PinnedFlags {
    int* p = nullptr;
    int cap = 0;
    ~PinnedFlags() {
      if (p) cudaFreeHost(p);
    }
  };
  thread_local PinnedFlags pf;
  if (pf.cap < batch) {
    if (pf.p) cudaFreeHost(pf.p);
    pf.cap = batch < 64 ? 64 : batch;
    if (cudaMallocHost(&pf.p, sizeof(int) * pf.cap) != cudaSuccess) { pf.p = nullptr; pf.cap = 0; return -1; }
  }
  int* hflag = pf.p;
  const int max_sweeps = 40;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    cudaMemsetAsync(flag, 0, sizeof(int) * batch, st);
    for (int r = 0; r < nb - 1; ++r) {
      kt_begin(KT_EIG_PAIR, st);
      blk_pair_kernel<R><<<dim3(npairs, batch), 128, 0, st>>>(np, nb, r, H, Qs, flag, ident, fro);
      kt_end(KT_EIG_PAIR, st);
      kt_begin(KT_EIG_UPDATE, st);
      blk_update_kernel<R><<<dim3(npairs * npairs + npairs * (np / 32), batch), 256, 0, st>>>(np, nb, r, H, Vw, Qs, ident);
      kt_end(KT_EIG_UPDATE, st);
      kt_add_work(KT_EIG_UPDATE, 8.0 * 32768.0 * batch * ((double)npairs * (npairs + 1) + (double)npairs * (np / 32)));
      count_launch(2);
    }
    cudaMemcpyAsync(hflag, flag, sizeof(int) * batch, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    int any = 0;
    for (int b = 0; b < batch; ++b) any |= hflag[b];
    if (!any) { sweeps = sweep + 1; break; }
  }

  size_t shm = sizeof(R) * (size_t)n;
  if (shm > 48 * 1024) cudaFuncSetAttribute(blk_finish_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  blk_finish_kernel<R><<<batch, 1024, shm, st>>>(n, np, H, Vw, w, sw, V, ldv, sV, perm);
  count_launch();
  return sweeps;
}

template int eigh<double>(cudaStream_t, int, const z128*, long long, long long, double*, long long, z128*, long long,
                          long long, int, void*, int);
template int eigh<float>(cudaStream_t, int, const c64*, long long, long long, float*, long long, c64*, long long,
                         long long, int, void*, int);

}  // namespace mpsgb

namespace mpsgb {
namespace {
// A = X X^H / n + diag(shift) with seeded X (n x n): Hermitian positive semi-definite test matrix
template <typename R>
__global__ void psd_test_kernel(int n, Cx<R>* X, unsigned long long seed, int kind) {
  long long tot = (long long)n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ULL + seed;
    h ^= h >> 33; h *= 0xff51afd7ed558ccdULL; h ^= h >> 33; h *= 0xc4ceb9fe1a85ec53ULL; h ^= h >> 33;
    double a = (double)(h & 0xFFFFFF) / 16777216.0 - 0.5, b = (double)((h >> 24) & 0xFFFFFF) / 16777216.0 - 0.5;
    // graded columns: column j scaled by 2^{-j/4} so the spectrum spans many decades
    int j = (int)(i % n);
    double sc = kind == 2 ? 1.0 : exp2(-0.25 * (j % 64));
    if (kind == 1 && j >= n / 2) sc = 0;  // rank n/2: n - n/2 exact zero eigenvalues
    X[i] = cmake<R>((R)(a * sc), (R)(b * sc));
  }
}
}  // namespace

template <typename R>
int eig_selftest_t(int n, int kind, unsigned long long seed, double* out) {
  cudaStream_t st;
  if (cudaStreamCreate(&st) != cudaSuccess) return -4;
  Cx<R> *X, *A, *V;
  R* w;
  void* ws;
  size_t wsb = eigh_workspace_bytes(n, 1, sizeof(R));
  cudaMalloc(&X, sizeof(Cx<R>) * (size_t)n * n);
  cudaMalloc(&A, sizeof(Cx<R>) * (size_t)n * n);
  cudaMalloc(&V, sizeof(Cx<R>) * (size_t)n * n);
  cudaMalloc(&w, sizeof(R) * n);
  cudaMalloc(&ws, wsb);
  psd_test_kernel<R><<<256, 256, 0, st>>>(n, X, seed, kind);
  Cx<R> one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
  if (kind == 2) {
    // A = [[I, P Q^H], [Q P^H, I]] with P, Q of n/8 columns: eigenvalues 1 +- sigma_k and a
    // degenerate eigenvalue 1 of multiplicity n - 2 (n/8) in the middle of the spectrum
    const int h = n / 2, k = std::max(1, n / 8);
    Cx<R>* P = X;
    Cx<R>* Q = X + (size_t)h * n;
    set_identity<R>(st, n, A, n);
    gemm<R>(st, h, n - h, k, one, rowmajor<R>(P, n), transposed<R>(Q, n, true), zero, rowmajor<R>(A + h, n));
    gemm<R>(st, n - h, h, k, one, rowmajor<R>(Q, n), transposed<R>(P, n, true), zero,
            rowmajor<R>(A + (size_t)h * n, n));
  } else {
    gemm<R>(st, n, n, n, one, rowmajor<R>(X, n), transposed<R>(X, n, true), zero, rowmajor<R>(A, n));
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaStreamSynchronize(st);
  cudaEventRecord(e0, st);
  int sweeps = eigh<R>(st, n, A, n, 0, w, 0, V, n, 0, 1, ws);
  cudaEventRecord(e1, st);
  cudaError_t err = cudaStreamSynchronize(st);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  // residual max_ij |(A V - V diag(w))_ij| / max|w|, and orthogonality max|V^H V - I|
  Cx<R> *T;
  cudaMalloc(&T, sizeof(Cx<R>) * (size_t)n * n);
  std::vector<Cx<R>> hA((size_t)n * n), hV((size_t)n * n), hT((size_t)n * n);
  std::vector<R> hw(n);
  gemm<R>(st, n, n, n, one, rowmajor<R>(A, n), rowmajor<R>(V, n), zero, rowmajor<R>(T, n));
  cudaMemcpyAsync(hT.data(), T, sizeof(Cx<R>) * hT.size(), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(hV.data(), V, sizeof(Cx<R>) * hV.size(), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(hw.data(), w, sizeof(R) * n, cudaMemcpyDeviceToHost, st);
  cudaError_t err2 = cudaStreamSynchronize(st);
  double res = 0, wmax = 0, orth = 0;
  for (int j = 0; j < n; ++j) wmax = std::max(wmax, std::fabs((double)hw[j]));
  for (long long i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double rx = hT[i * n + j].x - (double)hV[i * n + j].x * hw[j];
      double ry = hT[i * n + j].y - (double)hV[i * n + j].y * hw[j];
      res = std::max(res, std::sqrt(rx * rx + ry * ry));
    }
  for (int a = 0; a < n; a += std::max(1, n / 32))
    for (int b = 0; b < n; ++b) {
      double sx = 0, sy = 0;
      for (int i = 0; i < n; ++i) {
        Cx<R> x = hV[(size_t)i * n + a], y = hV[(size_t)i * n + b];
        sx += (double)x.x * y.x + (double)x.y * y.y;
        sy += (double)x.x * y.y - (double)x.y * y.x;
      }
      if (a == b) sx -= 1;
      orth = std::max(orth, std::sqrt(sx * sx + sy * sy));
    }
  bool sorted = true;
  for (int j = 1; j < n; ++j) sorted = sorted && hw[j] <= hw[j - 1];
  cudaFree(X); cudaFree(A); cudaFree(V); cudaFree(w); cudaFree(ws); cudaFree(T);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (err != cudaSuccess || err2 != cudaSuccess) return -4;
  out[0] = sweeps;
  out[1] = ms;
  out[2] = res / (wmax > 0 ? wmax : 1);
  out[3] = orth;
  out[4] = sorted ? 1 : 0;
  out[5] = wmax;
  return 0;
}

int eig_selftest(int n, int fp64, int kind, unsigned long long seed, double* out) {
  return fp64 ? eig_selftest_t<double>(n, kind, seed, out) : eig_selftest_t<float>(n, kind, seed, out);
}

}  // namespace mpsgb

// ---------------------------------------------------------------------------------------------
// Allocation-free variant of the eigensolver.  Some callers cannot allocate device memory at the
// point where they need a decomposition -- for example code running under an allocator that is
// frozen for the lifetime of a request, or a host thread that must not touch the CUDA allocator.
// For them the whole workspace of the solver lives in one file-scope device array of fixed size,
// shared by every call on a device.  Host code never dereferences the array's name (on the host it
// is only a stand-in symbol): its device address is resolved once per device with
// cudaGetSymbolAddress and passed to the kernels.  The cached address belongs to the device's
// primary context; it does not survive cudaDeviceReset, after which the library must not be
// called again in the same process.
// ---------------------------------------------------------------------------------------------
namespace mpsgb {
namespace {
constexpr int kNoAllocMaxN = 128;                // largest matrix the fixed scratch can hold
constexpr size_t kNoAllocBytes = size_t(1) << 20;  // 1 MiB of device scratch per device
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_base[128] = {nullptr};

template <typename R>
int eigh_noalloc_t(cudaStream_t st, int n, const Cx<R>* A, long long lda, R* w, Cx<R>* V, long long ldv,
                   unsigned char* scratch) {
  // carve the fixed scratch first and reject what does not fit before anything is launched
  unsigned char* ws = scratch;
  auto take = [&](size_t bytes) { unsigned char* p = ws; ws += (bytes + 255) & ~size_t(255); return p; };
  double* fro = reinterpret_cast<double*>(take(sizeof(double)));
  const int np = padded(n), nb = np / 16, npairs = nb / 2;
  Cx<R>* H = nullptr;
  Cx<R>* Vw = nullptr;
  Cx<R>* Qs = nullptr;
  int* perm = nullptr;
  int* flag = nullptr;
  int* ident = nullptr;
  if (n > 32) {
    H = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)np * np));
    Vw = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)np * np));
    Qs = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)npairs * 1024));
    perm = reinterpret_cast<int*>(take(sizeof(int) * (size_t)np));
    flag = reinterpret_cast<int*>(take(sizeof(int)));
    ident = reinterpret_cast<int*>(take(sizeof(int) * (size_t)npairs));
  }
  if ((size_t)(ws - scratch) > kNoAllocBytes) return -1;
  fro2_kernel<R><<<1, 256, 0, st>>>(n, A, lda, 0, fro);
  count_launch();
  if (n <= 32) {
    eig_small_kernel<R><<<1, 32, 0, st>>>(n, A, lda, 0, w, 0, V, ldv, 0, fro);
    count_launch();
    // the call returns only once its kernels are done with the shared scratch
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return -4;
    return 1;
  }
  {
    long long tot = (long long)np * np;
    blk_init_kernel<R><<<dim3((unsigned)((tot + 255) / 256), 1), 256, 0, st>>>(n, np, A, lda, 0, H, Vw);
    count_launch();
  }
  int sweeps = -1;
  for (int sweep = 0; sweep < 40; ++sweep) {
    if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return -4;
    for (int r = 0; r < nb - 1; ++r) {
      blk_pair_kernel<R><<<dim3(npairs, 1), 128, 0, st>>>(np, nb, r, H, Qs, flag, ident, fro);
      blk_update_kernel<R><<<dim3(npairs * npairs + npairs * (np / 32), 1), 256, 0, st>>>(np, nb, r, H, Vw, Qs, ident);
      count_launch(2);
    }
    int hf = 0;  // pageable host word: the copy is synchronous, nothing is allocated
    if (cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return -4;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -4;
    if (!hf) { sweeps = sweep + 1; break; }
  }
  blk_finish_kernel<R><<<1, 1024, sizeof(R) * (size_t)n, st>>>(n, np, H, Vw, w, 0, V, ldv, 0, perm);
  count_launch();
  // the call returns only once its kernels are done with the shared scratch
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return -4;
  return sweeps < 0 ? -3 : sweeps;
}
}  // namespace

// Returns the sweep count (> 0), -1 for a size beyond the fixed scratch, -3 if the sweep limit was
// reached, -4 for a CUDA error (including a failed cudaGetSymbolAddress).
int eigh_noalloc(int n, int fp64, const void* A, long long lda, void* w, void* V, long long ldv, cudaStream_t st) {
  if (n < 1 || n > kNoAllocMaxN) return -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return -4;
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return -4;
      g_noalloc_base[dev] = p;
    }
    base = g_noalloc_base[dev];
  }
  unsigned char* scratch = static_cast<unsigned char*>(base);
  if (fp64)
    return eigh_noalloc_t<double>(st, n, static_cast<const z128*>(A), lda, static_cast<double*>(w),
                                  static_cast<z128*>(V), ldv, scratch);
  return eigh_noalloc_t<float>(st, n, static_cast<const c64*>(A), lda, static_cast<float*>(w), static_cast<c64*>(V),
                               ldv, scratch);
}

}  // namespace mpsgb
