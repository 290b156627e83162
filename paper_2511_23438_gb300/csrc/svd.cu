// Singular value decomposition by one-sided (Hestenes) Jacobi rotations on the rows of a complex
// matrix, and the helper kernels of the exact truncation route (Sec. III: the MPO of an
// inter-block gate is applied, the spanned blocks are made right-isometric, and every spanned bond
// is truncated by the SVD of the centre block).
//
// X (p x q) is overwritten by K X, where K is a product of 2 x 2 unitary rotations of row pairs
// that makes the rows mutually orthogonal.  Rows (a, b) with Gram [[al, g], [conj(g), be]] and
// g = |g| e^{i phi} are replaced by
//     x_a <- c x_a - s e^{-i phi} x_b,     x_b <- s e^{i phi} x_a + c x_b,
// with t = sign(z) / (|z| + sqrt(1 + z^2)), z = (be - al) / (2 |g|), c = 1 / sqrt(1 + t^2), s = c t
// (the symmetric Schur rotation of the real matrix [[al, |g|], [|g|, be]] after the phase of g is
// moved into row b).  The same rotations accumulate in J (J = K, starting from I).  A pair is
// rotated while |g| > tol sqrt(al be); sweeps visit every pair once in the round-robin (circle)
// order, pairs of one round are disjoint and run in parallel.  At convergence the rows are
// s_i v_i with orthonormal v_i, and X_in = K^H X_out = U diag(s) V^H with U[:, i] = conj(K[i, :]).
// Singular values are never squared: the rotations act on X itself, so small singular values
// keep an absolute error of the order of eps |X| (not sqrt(eps) |X| as through a Gram matrix).
//
// Preconditioning (single problems): rows whose singular values are spread over many decades are
// all dominated by the largest component, and plain Jacobi then needs tens of sweeps.  Before the
// sweeps X is rotated by the eigenvectors of its Gram X X^H (descending), which orthogonalises the
// rows down to about sqrt(eps) of the largest; the rows below 1e-3 of the level's largest are then
// rotated again by the eigenvectors of their own Gram, and so on (at most four levels).  These are
// unitary rotations of the rows (accumulated in J like the Jacobi rotations), so they change
// nothing but the starting point: the sweeps that follow still decide every singular value on X
// itself, now in three to five sweeps.
//
// Two launch forms: one CTA per problem (batched, __syncthreads between rounds) and one problem
// over a cooperative grid (bounded grid barriers between rounds, as in the Householder reduction).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.hpp"

namespace mpsgb {

namespace {
constexpr int kSvdThreads = 512;
constexpr int kSvdMaxSweeps = 40;

__device__ __forceinline__ void svd_grid_sync(unsigned* count, unsigned target, int* err, long long lim) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
    const long long t0 = clock64();
    unsigned v;
    for (;;) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if (v >= target) break;
      if (clock64() - t0 > lim) { atomicExch(err, 1); break; }
    }
  }
  __syncthreads();
}

// players of round r in the circle method for pp (even) players: position 0 fixed, 1 .. pp-1 rotate
__device__ __forceinline__ int rr_player(int pp, int r, int j) { return j == 0 ? 0 : ((j - 1 + r) % (pp - 1)) + 1; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One pair (a, b): Gram entries, test, rotation of the rows of X and J.  Whole warp.
// Returns true if the pair was rotated.
template <typename R>
__device__ bool jacobi_pair(int p, int q, Cx<R>* X, long long ldx, Cx<R>* J, long long ldj, int a, int b, double tol,
                            double thr) {
  const int lane = threadIdx.x & 31;
  Cx<R>* xa = X + (long long)a * ldx;
  Cx<R>* xb = X + (long long)b * ldx;
  R al = 0, be = 0, gr = 0, gi = 0;
  for (int j = lane; j < q; j += 32) {
    const Cx<R> u = xa[j], v = xb[j];
    al = fma(u.x, u.x, fma(u.y, u.y, al));
    be = fma(v.x, v.x, fma(v.y, v.y, be));
    gr = fma(u.x, v.x, fma(u.y, v.y, gr));   // conj(u) v
    gi = fma(u.x, v.y, fma(-u.y, v.x, gi));
  }
  const double A = warp_sum((double)al), B = warp_sum((double)be), GR = warp_sum((double)gr), GI = warp_sum((double)gi);
  const double g = sqrt(GR * GR + GI * GI);
  // a row far below the numerical-rank cut is noise: it is not rotated (it would only chase its own
  // rounding errors), and it stays that small whatever is rotated into the other rows
  if (!(fmin(A, B) >= thr)) return false;
  if (!(g > tol * sqrt(A) * sqrt(B)) || !(g > 0)) return false;
  const double z = (B - A) / (2.0 * g);
  const double t = (z >= 0 ? 1.0 : -1.0) / (fabs(z) + hypot(1.0, z));
  if (!(t != 0)) return false;
  const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
  const double er = GR / g, ei = GI / g;  // e^{i phi}
  // x_a' = c x_a - s conj(e) x_b ; x_b' = s e x_a + c x_b
  const Cx<R> m_ab = cmake<R>((R)(-s * er), (R)(s * ei));   // -s e^{-i phi}
  const Cx<R> m_ba = cmake<R>((R)(s * er), (R)(s * ei));    // s e^{i phi}
  const R cr = (R)c;
  for (int j = lane; j < q; j += 32) {
    const Cx<R> u = xa[j], v = xb[j];
    xa[j] = cr * u + m_ab * v;
    xb[j] = m_ba * u + cr * v;
  }
  Cx<R>* ja = J + (long long)a * ldj;
  Cx<R>* jb = J + (long long)b * ldj;
  for (int j = lane; j < p; j += 32) {
    const Cx<R> u = ja[j], v = jb[j];
    ja[j] = cr * u + m_ab * v;
    jb[j] = m_ba * u + cr * v;
  }
  return true;
}

// Sweeps until no pair is rotated.  GRID = false: CTA blockIdx.x solves problem blockIdx.x of a
// batch (pointers advanced by the batch strides); GRID = true: the whole cooperative grid solves one
// problem.  flags: kSvdMaxSweeps words per problem (zeroed by the host); out_sweeps[problem] gets
// the number of sweeps, or -1 if the limit was reached.
template <typename R, bool GRID>
__global__ void __launch_bounds__(kSvdThreads) jacobi_rows_kernel(int p, int q, Cx<R>* X, long long ldx, long long sX,
                                                                 Cx<R>* J, long long ldj, long long sJ, int* flags,
                                                                 int* out_sweeps, double tol, const double* thr_sq,
                                                                 unsigned* bar, int* err, long long lim) {
  const int prob = GRID ? 0 : blockIdx.x;
  const double thr = thr_sq[prob];
  X += prob * sX;
  J += prob * sJ;
  flags += prob * kSvdMaxSweeps;
  const int warps_cta = blockDim.x >> 5;
  const int gw = GRID ? blockIdx.x * warps_cta + (threadIdx.x >> 5) : (threadIdx.x >> 5);
  const int nw = GRID ? gridDim.x * warps_cta : warps_cta;
  const int pp = p + (p & 1);
  const int npairs = pp / 2;
  __shared__ int rotated;
  unsigned nbar = 0;
  int sweeps = -1;
  for (int sweep = 0; sweep < kSvdMaxSweeps; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < pp - 1; ++r) {
      for (int k = gw; k < npairs; k += nw) {
        int a = rr_player(pp, r, k), b = rr_player(pp, r, pp - 1 - k);
        if (a > b) { const int tmp = a; a = b; b = tmp; }
        if (b >= p) continue;  // the padding player
        if (jacobi_pair<R>(p, q, X, ldx, J, ldj, a, b, tol, thr) && (threadIdx.x & 31) == 0) rotated = 1;
      }
      if (GRID) svd_grid_sync(bar, (++nbar) * gridDim.x, err, lim);
      else __syncthreads();
    }
    if (GRID) {
      if (threadIdx.x == 0 && rotated) atomicOr(&flags[sweep], 1);
      svd_grid_sync(bar, (++nbar) * gridDim.x, err, lim);
      if (threadIdx.x == 0) rotated = atomicAdd(&flags[sweep], 0);
      __syncthreads();
    }
    if (!rotated) { sweeps = sweep + 1; break; }
    __syncthreads();
  }
  if (threadIdx.x == 0 && (!GRID || blockIdx.x == 0)) out_sweeps[prob] = sweeps;
}

// Row norms (FP64) and the descending order: perm[rank] = row, ties in row order.
template <typename R>
__global__ void row_norms_kernel(int p, int q, const Cx<R>* X, long long ldx, long long sX, double* nrm) {
  const int prob = blockIdx.y;
  X += prob * sX;
  nrm += (long long)prob * p;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (w >= p) return;
  const Cx<R>* x = X + (long long)w * ldx;
  double acc = 0;
  for (int j = lane; j < q; j += 32) acc += (double)x[j].x * x[j].x + (double)x[j].y * x[j].y;
  acc = warp_sum(acc);
  if (lane == 0) nrm[w] = sqrt(acc);
}

// noise threshold on squared row norms: (0.1 eps max(p, q))^2 |X|_F^2 / min(p, q), a tenth of the
// numerical-rank cut s_0 max(p, q) eps at the least s_0 can be
__global__ void noise_threshold_kernel(int p, int q, const double* nrm, double eps, double* thr) {
  const int prob = blockIdx.x;
  nrm += (long long)prob * p;
  double acc = 0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) acc += nrm[i] * nrm[i];
  acc = warp_sum(acc);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    const double f = 0.1 * eps * (double)(p > q ? p : q);
    thr[prob] = f * f * t / (double)(p < q ? p : q);
  }
}

__global__ void rank_sort_kernel(int p, const double* nrm, int* perm, double* s_sorted) {
  const int prob = blockIdx.y;
  nrm += (long long)prob * p;
  perm += (long long)prob * p;
  s_sorted += (long long)prob * p;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p) return;
  // a total order (a non-finite norm counts as -1, below every norm, ties by row) so that the
  // ranks are always a permutation of 0 .. p-1; the host rejects non-finite norms afterwards
  auto key = [](double x) { return isfinite(x) ? x : -1.0; };
  const double v = key(nrm[i]);
  int rank = 0;
  for (int j = 0; j < p; ++j) {
    const double u = key(nrm[j]);
    rank += (u > v) || (u == v && j < i);
  }
  perm[rank] = i;
  s_sorted[rank] = nrm[i];
}

// Vh[i, :] = X[perm[i], :] / s_i (zero row where s_i == 0); U[r, i] = conj(J[perm[i], r])
template <typename R>
__global__ void svd_finish_kernel(int p, int q, const Cx<R>* X, long long ldx, long long sX, const Cx<R>* J,
                                  long long ldj, long long sJ, const int* perm, const double* s, Cx<R>* Vh,
                                  long long ldvh, long long sVh, Cx<R>* U, long long ldu, long long sU, int* err) {
  const int prob = blockIdx.y;
  X += prob * sX; J += prob * sJ; Vh += prob * sVh; U += prob * sU;
  perm += (long long)prob * p;
  s += (long long)prob * p;
  const long long totv = (long long)p * q, totu = (long long)p * p;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < totv + totu;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < totv) {
      if (!Vh) continue;
      const long long i = e / q, j = e - i * q;
      const int pi = perm[i];
      if (pi < 0 || pi >= p) { atomicExch(err, 2); continue; }  // never taken: perm is a permutation
      const double si = s[i];
      const Cx<R> x = X[(long long)pi * ldx + j];
      const R f = si > 0 ? (R)(1.0 / si) : R(0);
      Vh[i * ldvh + j] = f * x;
    } else {
      if (!U) continue;
      const long long f2 = e - totv;
      const long long r = f2 / p, i = f2 - r * p;
      const int pi = perm[i];
      if (pi < 0 || pi >= p) { atomicExch(err, 2); continue; }
      U[r * ldu + i] = conj(J[(long long)pi * ldj + r]);
    }
  }
}

template <typename R>
__global__ void identity_batch_kernel(int p, Cx<R>* J, long long ldj, long long sJ) {
  const int prob = blockIdx.y;
  J += prob * sJ;
  const long long tot = (long long)p * p;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / p, j = e - i * p;
    J[i * ldj + j] = cmake<R>(i == j ? R(1) : R(0), R(0));
  }
}

// Expansion of one block by the rank-2 MPO of exp(-i phi Z_i Z_j) = cos(phi) I I - i sin(phi) Z_i Z_j
// (the operator Schmidt form; MPO index v is the slow part of a doubled bond index):
//   mode 0, block p:          out[a, s, v r + b]       = c_v(s) in[a, s, b], c_0 = cos phi, c_1 = -i sin phi z_i(s)
//   mode 1, blocks between:   out[v l + a, s, w r + b] = delta_vw in[a, s, b]
//   mode 2, block q:          out[v l + a, s, b]       = c_v(s) in[a, s, b], c_0 = 1, c_1 = z_j(s)
// z(s) = 1 - 2 bit(s), bit `shift` counted from the least significant end.
template <typename R>
__global__ void mpo_expand_kernel(int mode, int l, int d, int r, const Cx<R>* in, Cx<R>* out, double cphi, double sphi,
                                  int shift) {
  const int lo = mode == 0 ? l : 2 * l, ro = mode == 2 ? r : 2 * r;
  const long long tot = (long long)lo * d * ro;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long A = e / ((long long)d * ro);
    const long long rem = e - A * (long long)d * ro;
    const int s = (int)(rem / ro);
    const long long B = rem - (long long)s * ro;
    const int v = (int)(A / l), w = (int)(B / r);
    const long long a = A - (long long)v * l, b = B - (long long)w * r;
    const Cx<R> x = in[(a * d + s) * (long long)r + b];
    const double z = ((s >> shift) & 1) ? -1.0 : 1.0;
    Cx<R> y;
    if (mode == 0) y = w == 0 ? (R)cphi * x : cmake<R>(0, (R)(-sphi * z)) * x;
    else if (mode == 1) y = v == w ? x : cmake<R>(0, 0);
    else y = v == 0 ? x : (R)z * x;
    out[e] = y;
  }
}

// theta[(a, s), (t, b)] *= exp(-i phi z(s, shift_a) z(t, shift_b)), z(x, k) = 1 - 2 bit_k(x)
template <typename R>
__global__ void two_site_phase_kernel(int l, int da, int db, int r, Cx<R>* th, double phi, int shift_a, int shift_b) {
  const long long tot = (long long)l * da * db * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long ab = e / r;
    const int t = (int)(ab % db);
    const int s = (int)((ab / db) % da);
    const double z = (((s >> shift_a) & 1) ? -1.0 : 1.0) * (((t >> shift_b) & 1) ? -1.0 : 1.0);
    double sn, cs;
    sincos(phi * z, &sn, &cs);
    th[e] = cmake<R>((R)cs, (R)(-sn)) * th[e];
  }
}

// insert a zero bit at position pos of v
__device__ __forceinline__ int insert_zero_bit(int v, int pos) {
  return ((v >> pos) << (pos + 1)) | (v & ((1 << pos) - 1));
}

// th (l, da, db, r): a general two-qubit gate u on bit shift_a of the first physical index and bit
// shift_b of the second (u's row / column index 2 x + y, x the first qubit's bit); one thread per
// group of the four amplitudes that differ only in those two bits
template <typename R>
__global__ void two_site_gate_kernel(int l, int da, int db, int r, Cx<R>* th, Gate4 u, int shift_a, int shift_b) {
  const int ha = da >> 1, hb = db >> 1;
  const long long tot = (long long)l * ha * hb * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long b = e % r;
    const long long q = e / r;
    const int tr = (int)(q % hb);
    const int sr = (int)((q / hb) % ha);
    const long long a = q / ((long long)hb * ha);
    const int s0 = insert_zero_bit(sr, shift_a), t0 = insert_zero_bit(tr, shift_b);
    long long idx[4];
    Cx<R> x[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int s = s0 | ((v >> 1) << shift_a), t = t0 | ((v & 1) << shift_b);
      idx[v] = ((a * da + s) * db + t) * r + b;
      x[v] = th[idx[v]];
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      Cx<R> acc = cmake<R>(0, 0);
#pragma unroll
      for (int v = 0; v < 4; ++v) cfma(acc, cmake<R>((R)u.re[4 * w + v], (R)u.im[4 * w + v]), x[v]);
      th[idx[w]] = acc;
    }
  }
}

// X[i, j] *= c * s[i] for i < rows, j < cols
template <typename R>
__global__ void scale_rows_kernel(int rows, int cols, Cx<R>* X, long long ld, const double* s, double c) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / cols, j = e - i * cols;
    X[i * ld + j] = (R)(c * s[i]) * X[i * ld + j];
  }
}

// X[i, j] *= c * s[j] for i < rows, j < cols
template <typename R>
__global__ void scale_cols_kernel(int rows, int cols, Cx<R>* X, long long ld, const double* s, double c) {
  const long long tot = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / cols, j = e - i * cols;
    X[i * ld + j] = (R)(c * s[j]) * X[i * ld + j];
  }
}

inline int grid_of(long long n, int t) {
  long long b = (n + t - 1) / t;
  return (int)std::min<long long>(std::max<long long>(b, 1), 65535LL * 8);
}
}  // namespace

size_t svd_rows_workspace_bytes(int p, int q, int batch, int real_bytes) {
  const size_t c = 2 * (size_t)real_bytes;
  size_t b = 0;
  auto add = [&](size_t x) { b += (x + 255) & ~size_t(255); };
  add(c * (size_t)p * q * batch);               // working copy of X
  add(c * (size_t)p * p * batch);               // J
  add(sizeof(double) * (size_t)p * batch * 2);  // norms, sorted s
  add(sizeof(double) * (size_t)batch);          // noise thresholds
  add(sizeof(int) * (size_t)p * batch);         // perm
  add(sizeof(int) * (size_t)kSvdMaxSweeps * batch + sizeof(int) * batch + 64);
  if (batch == 1) {  // preconditioner: Gram, its eigenvectors and eigenvalues, a rotated copy
    add(c * (size_t)p * p * 2);
    add((size_t)real_bytes * p);
    add(c * (size_t)p * (size_t)std::max(p, q));
    add(eigh_workspace_bytes(p, 1, real_bytes));
  }
  return b + 1024;
}

template <typename R>
int svd_rows(cudaStream_t st, int p, int q, const Cx<R>* X, long long ldx, double* s, double* s_host, Cx<R>* Vh,
             long long ldvh, Cx<R>* U, long long ldu, void* workspace, int batch, long long sX, long long sVh,
             long long sU) {
  if (p < 1 || q < 1 || batch < 1) return -4;
  char* ws = static_cast<char*>(workspace);
  auto take = [&](size_t bytes) { char* r = ws; ws += (bytes + 255) & ~size_t(255); return r; };
  Cx<R>* Xw = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)p * q * batch));
  Cx<R>* Jw = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)p * p * batch));
  double* nrm = reinterpret_cast<double*>(take(sizeof(double) * (size_t)p * batch * 2));
  double* thr = reinterpret_cast<double*>(take(sizeof(double) * (size_t)batch));
  int* perm = reinterpret_cast<int*>(take(sizeof(int) * (size_t)p * batch));
  int* flags = reinterpret_cast<int*>(take(sizeof(int) * (size_t)kSvdMaxSweeps * batch + sizeof(int) * batch + 64));
  int* sweeps = flags + kSvdMaxSweeps * batch;
  unsigned* bar = reinterpret_cast<unsigned*>(sweeps + batch);
  int* err = reinterpret_cast<int*>(bar + 4);
  cudaMemsetAsync(flags, 0, sizeof(int) * (size_t)kSvdMaxSweeps * batch + sizeof(int) * batch + 64, st);
  for (int b = 0; b < batch; ++b)
    copy_view<R, R>(st, p, q, rowmajor<R>(const_cast<Cx<R>*>(X) + b * sX, ldx), rowmajor<R>(Xw + (size_t)b * p * q, q));
  identity_batch_kernel<R><<<dim3(grid_of((long long)p * p, 256), batch), 256, 0, st>>>(p, Jw, p, (long long)p * p);
  count_launch();
  const double eps = sizeof(R) == 8 ? 2.220446049250313e-16 : 1.1920929e-7;
  if (batch == 1 && p >= 2) {
    double top0 = 0;
    Cx<R>* G = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)p * p * 2));
    Cx<R>* V = G + (size_t)p * p;
    R* w = reinterpret_cast<R*>(take(sizeof(R) * (size_t)p));
    Cx<R>* T = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)p * std::max(p, q)));
    void* eigws = take(eigh_workspace_bytes(p, 1, sizeof(R)));
    const Cx<R> one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    std::vector<R> hw(p);
    int start = 0;
    for (int level = 0; level < 4 && start < p - 1; ++level) {
      const int m = p - start;
      Cx<R>* Xs = Xw + (size_t)start * q;
      Cx<R>* Js = Jw + (size_t)start * p;
      gemm<R>(st, m, m, q, one, rowmajor<R>(Xs, q), transposed<R>(Xs, q, true), zero, rowmajor<R>(G, m));
      const int es = eigh<R>(st, m, G, m, 0, w, 0, V, m, 0, 1, eigws);
      if (es == -2) return -2;
      if (es == -4) return -4;
      if (es < 0) break;  // no usable eigenvectors for this level: the sweeps start from here
      cudaMemcpyAsync(hw.data(), w, sizeof(R) * m, cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) return -4;
      // rows at the rounding floor of the first level (or a Gram that is not finite) carry no
      // direction worth rotating to: the sweeps start from here
      if (level == 0) top0 = (double)hw[0];
      if (!std::isfinite((double)hw[0]) || !((double)hw[0] > 64.0 * eps * eps * top0)) break;
      gemm<R>(st, m, q, m, one, transposed<R>(V, m, true), rowmajor<R>(Xs, q), zero, rowmajor<R>(T, q));
      cudaMemcpyAsync(Xs, T, sizeof(Cx<R>) * (size_t)m * q, cudaMemcpyDeviceToDevice, st);
      gemm<R>(st, m, p, m, one, transposed<R>(V, m, true), rowmajor<R>(Js, p), zero, rowmajor<R>(T, p));
      cudaMemcpyAsync(Js, T, sizeof(Cx<R>) * (size_t)m * p, cudaMemcpyDeviceToDevice, st);
      int t = 0;
      while (t < m && (double)hw[t] > 1e-6 * (double)hw[0]) ++t;
      if (t == 0 || t >= m - 1) break;
      start += t;
    }
  }
  const double tol = eps * std::sqrt((double)std::max(q, 16));
  const long long lim = wait_limit_cycles();
  // one CTA per problem unless a single large problem can use the whole GPU
  const bool grid_mode = batch == 1 && (long long)p * q >= (1LL << 18) && p >= 64;
  row_norms_kernel<R><<<dim3((p + 7) / 8, batch), 256, 0, st>>>(p, q, Xw, q, (long long)p * q, nrm);
  noise_threshold_kernel<<<batch, 256, 0, st>>>(p, q, nrm, eps, thr);
  count_launch(2);
  kt_begin(KT_SVD, st);
  if (!grid_mode) {
    jacobi_rows_kernel<R, false><<<batch, kSvdThreads, 0, st>>>(p, q, Xw, q, (long long)p * q, Jw, p, (long long)p * p,
                                                                flags, sweeps, tol, thr, bar, err, lim);
  } else {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_rows_kernel<R, true>, kSvdThreads, 0);
    if (per_sm < 1) return -4;
    const int need = (p / 2 + (kSvdThreads / 32) - 1) / (kSvdThreads / 32);  // one warp per pair of a round
    int grid = std::max(1, std::min(sms, need));
    int p_ = p, q_ = q;
    long long ldx_ = q, sX_ = (long long)p * q, ldj_ = p, sJ_ = (long long)p * p;
    double tol_ = tol;
    long long lim_ = lim;
    void* args[] = {&p_, &q_, &Xw, &ldx_, &sX_, &Jw, &ldj_, &sJ_, &flags, &sweeps, &tol_, &thr, &bar, &err, &lim_};
    if (cudaLaunchCooperativeKernel((void*)jacobi_rows_kernel<R, true>, dim3(grid), dim3(kSvdThreads), args, 0, st) !=
        cudaSuccess)
      return -4;
  }
  kt_end(KT_SVD, st);
  count_launch();
  row_norms_kernel<R><<<dim3((p + 7) / 8, batch), 256, 0, st>>>(p, q, Xw, q, (long long)p * q, nrm);
  rank_sort_kernel<<<dim3((p + 127) / 128, batch), 128, 0, st>>>(p, nrm, perm, nrm + (size_t)p * batch);
  svd_finish_kernel<R><<<dim3(grid_of((long long)p * (p + q), 256), batch), 256, 0, st>>>(
      p, q, Xw, q, (long long)p * q, Jw, p, (long long)p * p, perm, nrm + (size_t)p * batch, Vh, ldvh, sVh, U, ldu, sU,
      err);
  count_launch(3);
  if (s) cudaMemcpyAsync(s, nrm + (size_t)p * batch, sizeof(double) * (size_t)p * batch, cudaMemcpyDeviceToDevice, st);
  if (s_host)
    cudaMemcpyAsync(s_host, nrm + (size_t)p * batch, sizeof(double) * (size_t)p * batch, cudaMemcpyDeviceToHost, st);
  std::vector<int> hs(batch);
  int herr = 0;
  cudaMemcpyAsync(hs.data(), sweeps, sizeof(int) * batch, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return -4;
  if (herr == 2) return -4;  // a bad permutation was caught (see svd_finish_kernel)
  if (herr) return -2;
  if (s_host)
    for (int i = 0; i < p * batch; ++i)
      if (!std::isfinite(s_host[i])) return -5;  // the input was not finite
  int mx = 0;
  for (int v : hs) {
    if (v < 0) return -1;
    mx = std::max(mx, v);
  }
  return mx;
}

template <typename R>
void mpo_expand(cudaStream_t st, int mode, int l, int d, int r, const Cx<R>* in, Cx<R>* out, double phi, int shift) {
  const long long tot = (long long)(mode == 0 ? l : 2 * l) * d * (mode == 2 ? r : 2 * r);
  mpo_expand_kernel<R><<<grid_of(tot, 256), 256, 0, st>>>(mode, l, d, r, in, out, std::cos(phi), std::sin(phi), shift);
  count_launch();
}

template <typename R>
void scale_rows(cudaStream_t st, int rows, int cols, Cx<R>* X, long long ld, const double* s, double c) {
  scale_rows_kernel<R><<<grid_of((long long)rows * cols, 256), 256, 0, st>>>(rows, cols, X, ld, s, c);
  count_launch();
}

template <typename R>
void two_site_phase(cudaStream_t st, int l, int da, int db, int r, Cx<R>* th, double phi, int shift_a, int shift_b) {
  two_site_phase_kernel<R><<<grid_of((long long)l * da * db * r, 256), 256, 0, st>>>(l, da, db, r, th, phi, shift_a,
                                                                                    shift_b);
  count_launch();
}

template <typename R>
void two_site_gate(cudaStream_t st, int l, int da, int db, int r, Cx<R>* th, const Gate4& u, int shift_a, int shift_b) {
  two_site_gate_kernel<R><<<grid_of((long long)l * (da >> 1) * (db >> 1) * r, 256), 256, 0, st>>>(l, da, db, r, th, u,
                                                                                                 shift_a, shift_b);
  count_launch();
}

template <typename R>
void scale_cols(cudaStream_t st, int rows, int cols, Cx<R>* X, long long ld, const double* s, double c) {
  scale_cols_kernel<R><<<grid_of((long long)rows * cols, 256), 256, 0, st>>>(rows, cols, X, ld, s, c);
  count_launch();
}

#define MPSGB_SVD_INST(R)                                                                                           \
  template int svd_rows<R>(cudaStream_t, int, int, const Cx<R>*, long long, double*, double*, Cx<R>*, long long,   \
                           Cx<R>*, long long, void*, int, long long, long long, long long);                         \
  template void mpo_expand<R>(cudaStream_t, int, int, int, int, const Cx<R>*, Cx<R>*, double, int);                 \
  template void scale_rows<R>(cudaStream_t, int, int, Cx<R>*, long long, const double*, double);              \
  template void scale_cols<R>(cudaStream_t, int, int, Cx<R>*, long long, const double*, double);             \
  template void two_site_phase<R>(cudaStream_t, int, int, int, int, Cx<R>*, double, int, int);                    \
  template void two_site_gate<R>(cudaStream_t, int, int, int, int, Cx<R>*, const Gate4&, int, int);
MPSGB_SVD_INST(double)
MPSGB_SVD_INST(float)

}  // namespace mpsgb

// ---------------------------------------------------------------------------------------------
// Kernel check of svd_rows on a caller-supplied host matrix (allocates its own device memory).
// ---------------------------------------------------------------------------------------------
namespace mpsgb {
namespace {
template <typename R>
int svd_selftest_t(int p, int q, const double* Xh, double* s_out, double* out) {
  cudaStream_t st;
  if (cudaStreamCreate(&st) != cudaSuccess) return -4;
  const size_t nx = (size_t)p * q;
  std::vector<Cx<R>> hx(nx), hv(nx), hu((size_t)p * p);
  for (size_t i = 0; i < nx; ++i) hx[i] = cmake<R>((R)Xh[2 * i], (R)Xh[2 * i + 1]);
  Cx<R> *X = nullptr, *Vh = nullptr, *U = nullptr;
  double* s = nullptr;
  void* ws = nullptr;
  const size_t wsb = svd_rows_workspace_bytes(p, q, 1, sizeof(R));
  cudaError_t e = cudaSuccess;
  e = cudaMalloc(&X, sizeof(Cx<R>) * nx);
  if (e == cudaSuccess) e = cudaMalloc(&Vh, sizeof(Cx<R>) * nx);
  if (e == cudaSuccess) e = cudaMalloc(&U, sizeof(Cx<R>) * (size_t)p * p);
  if (e == cudaSuccess) e = cudaMalloc(&s, sizeof(double) * p);
  if (e == cudaSuccess) e = cudaMalloc(&ws, wsb);
  int sweeps = -4;
  float ms = 0;
  std::vector<double> hs(p);
  if (e == cudaSuccess) {
    cudaMemcpyAsync(X, hx.data(), sizeof(Cx<R>) * nx, cudaMemcpyHostToDevice, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    sweeps = svd_rows<R>(st, p, q, X, q, s, hs.data(), Vh, q, U, p, ws);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemcpyAsync(hv.data(), Vh, sizeof(Cx<R>) * nx, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(hu.data(), U, sizeof(Cx<R>) * (size_t)p * p, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) sweeps = -4;
  }
  cudaFree(X); cudaFree(Vh); cudaFree(U); cudaFree(s); cudaFree(ws);
  cudaStreamDestroy(st);
  if (e != cudaSuccess) return -4;
  // residual max |U diag(s) Vh - X| / max |X|, unitarity of U, orthonormality of the rows of Vh
  // whose s is above the numerical-rank cut
  double xmax = 0, res = 0, ou = 0, ov = 0;
  for (size_t i = 0; i < nx; ++i) xmax = std::max(xmax, std::hypot(Xh[2 * i], Xh[2 * i + 1]));
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < q; ++j) {
      double ar = 0, ai = 0;
      for (int k = 0; k < p; ++k) {
        const Cx<R> u = hu[(size_t)i * p + k], v = hv[(size_t)k * q + j];
        ar += hs[k] * ((double)u.x * v.x - (double)u.y * v.y);
        ai += hs[k] * ((double)u.x * v.y + (double)u.y * v.x);
      }
      res = std::max(res, std::hypot(ar - Xh[2 * ((size_t)i * q + j)], ai - Xh[2 * ((size_t)i * q + j) + 1]));
    }
  const double eps = sizeof(R) == 8 ? 2.220446049250313e-16 : 1.1920929e-7;
  int kr = 0;
  while (kr < p && hs[kr] > hs[0] * std::max(p, q) * eps) ++kr;
  for (int a = 0; a < p; ++a)
    for (int b = 0; b < p; ++b) {
      double ur = 0, ui = 0, vr = 0, vi = 0;
      for (int k = 0; k < p; ++k) {
        const Cx<R> x = hu[(size_t)k * p + a], y = hu[(size_t)k * p + b];
        ur += (double)x.x * y.x + (double)x.y * y.y;
        ui += (double)x.x * y.y - (double)x.y * y.x;
      }
      if (a == b) ur -= 1;
      ou = std::max(ou, std::hypot(ur, ui));
      if (a < kr && b < kr) {
        for (int j = 0; j < q; ++j) {
          const Cx<R> x = hv[(size_t)a * q + j], y = hv[(size_t)b * q + j];
          vr += (double)x.x * y.x + (double)x.y * y.y;
          vi += (double)x.x * y.y - (double)x.y * y.x;
        }
        if (a == b) vr -= 1;
        ov = std::max(ov, std::hypot(vr, vi));
      }
    }
  for (int i = 0; i < p; ++i) s_out[i] = hs[i];
  out[0] = sweeps;
  out[1] = ms;
  out[2] = res / (xmax > 0 ? xmax : 1);
  out[3] = ou;
  out[4] = ov;
  out[5] = kr;
  return 0;
}
}  // namespace

int svd_selftest(int p, int q, int fp64, const double* X, double* s, double* out) {
  return fp64 ? svd_selftest_t<double>(p, q, X, s, out) : svd_selftest_t<float>(p, q, X, s, out);
}

}  // namespace mpsgb
