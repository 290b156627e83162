// Hermitian eigensolver for larger matrices: Householder reduction to a real symmetric
// tridiagonal T, eigenvalues of T by multisection, eigenvectors of T by inverse iteration on
// its unreduced blocks, orthonormalisation, and back-transformation with the reflectors.
//
// 1. hetrd_kernel (cooperative, one CTA per SM): for column i the reflector
//    H_i = I - tau_i v_i v_i^H (v_i[i+1] = 1) maps W[i+1:, i] to (beta, 0, ...), beta real;
//    p = tau W22 v, w = p - (tau/2)(p^H v) v, W22 -= v w^H + w v^H.  Rows are owned
//    cyclically by the CTAs; two bounded grid barriers per column (p ready, update done).
//    T = Q^H A Q with Q = H_0 H_1 ... H_{n-2}; d = diag, e = sub-diagonal.
// 2. T is split where |e_i| <= 32 eps ||T||; bisect_kernel finds eigenvalue k of each
//    unreduced block by 33-section of its Sturm count (one warp per eigenvalue).
// 3. inverse_iter_kernel: one thread per eigenvector; LU with partial pivoting of
//    (T_b - lambda I) on the eigenvalue's block, three solves from a seeded start vector.
// 4. cluster_mgs_kernel: one CTA per cluster of close eigenvalues of one block;
//    Gram-Schmidt (twice) of its vectors in order.
// 5. All eigenvectors of T are made orthonormal (block Gram-Schmidt twice, Cholesky-QR
//    twice, on real GEMMs), then X = Q Z is formed with compact-WY panels of 32 reflectors.
// Every grid barrier waits a bounded time; on timeout it records an error word.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.hpp"

namespace mpsgb {

namespace {
// Grid-wide barrier on a monotonic arrival counter: CTA thread 0 adds 1 with release semantics
// and polls with acquire loads until `target` (= barrier index x gridDim.x) is reached.  The
// wait is bounded by clock64() (lim cycles, wait_limit_cycles() on the host); on timeout it records
// err and continues, so the kernel always finishes and the host reports the error.
__device__ __forceinline__ void grid_sync(unsigned* count, unsigned target, int* err, long long lim) {
  __syncthreads();
  if (threadIdx.x == 0) {
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

// Split form of grid_sync: grid_arrive publishes this CTA's writes and counts it in; grid_wait
// (after independent work) waits until `target` arrivals, bounded like grid_sync.
__device__ __forceinline__ void grid_arrive(unsigned* count) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
}
__device__ __forceinline__ void grid_wait(unsigned* count, unsigned target, int* err, long long lim) {
  if (threadIdx.x == 0) {
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

// Householder reduction of the Hermitian n x n matrix A to real symmetric tridiagonal form.
// Rows of the working matrix are owned cyclically by the CTAs (CTA c: rows c, c + G, ...; slot t
// holds row c + t G).  A CTA keeps its rows in shared memory except the first T0 slots when not
// all fit; those rows stay in the global copy W, and as the lowest-numbered rows they drop out of
// the active trailing matrix first (after column c + (T0 - 1) G).  Per column i:
//   A. every CTA forms the reflector (beta, tau, v) of column i itself from the contiguous copy of
//      column i in colbuf (parity i & 1), v kept in shared memory; owned rows: p_r = tau (W22 v)_r
//      (one warp per row) and a partial p^H v; arrive at barrier 1, apply the part -p_r conj(v_j)
//      of the update that needs only the CTA's own p_r, wait at barrier 1;
//   B. every CTA loads p into shared memory; owned rows: W22 -= v w^H + w v^H with
//      w = p - (tau/2)(p^H v) v, column i+1 first: it goes to colbuf (other parity), its squared
//      norm below the sub-diagonal is accumulated, the owner of row i+1 writes d[i+1], and the
//      CTA arrives at barrier 2; then the rest of its rows (columns i+2 ..), the Householder
//      vector into column i of W (global) for the back-transformation, and the wait on
//      barrier 2, whose latency the update hides (the next column only needs colbuf).
// acc[0..1]: squared norm of column i (parity i & 1); acc[2..5]: p^H v (re, im) by parity.
template <typename R>
__global__ void __launch_bounds__(512) hetrd_kernel(int n, const Cx<R>* A, long long lda, Cx<R>* W, R* d, R* e,
                                                    Cx<R>* tau, Cx<R>* pb, Cx<R>* colbuf, double* acc, unsigned* bar,
                                                    int* err, long long lim, int s_fit) {
  extern __shared__ __align__(16) unsigned char hetrd_smem[];
  __shared__ double hsc[6];  // tau (re, im), 1 / (alpha - beta) (re, im), a2 (re, im)
  Cx<R>* vs = reinterpret_cast<Cx<R>*>(hetrd_smem);
  Cx<R>* ps = vs + n;
  Cx<R>* rs = ps + n;  // s_fit cached rows
  const int G = gridDim.x, c = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
  const int warp = t >> 5, lane = t & 31, nw = nt >> 5;
  const int nslots = c < n ? (n - c + G - 1) / G : 0;
  const int T0 = nslots > s_fit ? nslots - s_fit : 0;
  auto rowp = [&](int slot) -> Cx<R>* {
    return slot >= T0 ? rs + (long long)(slot - T0) * n : W + (long long)(c + slot * G) * n;
  };
  unsigned nbar = 0;
  double nrm = 0;
  for (int slot = 0; slot < nslots; ++slot) {
    const int r = c + slot * G;
    Cx<R>* dst = rowp(slot);
    for (int j = t; j < n; j += nt) dst[j] = A[(long long)r * lda + j];
    if (t == 0) {
      const Cx<R> a0 = A[(long long)r * lda];
      colbuf[r] = a0;
      if (r >= 2) nrm += (double)abs2(a0);
      if (r == 0) d[0] = a0.x;
    }
  }
  if (t == 0 && nrm != 0) atomicAdd(&acc[0], nrm);
  grid_sync(bar, (++nbar) * G, err, lim);
  for (int i = 0; i < n - 1; ++i) {
    const int par = i & 1;
    const Cx<R>* col = colbuf + (size_t)par * n;   // column i, rows >= i + 1
    Cx<R>* coln = colbuf + (size_t)(par ^ 1) * n;  // column i + 1, written in phase B
    // ---- A: reflector of column i (thread 0 of every CTA forms the same scalars in FP64 and
    // shares them: FP64 divisions and square roots are slow on this part, so they are not
    // repeated by every thread), v into shared memory
    if (t == 0) {
      const Cx<R> alpha = col[i + 1];
      const double xn2 = acc[par];
      const double ar = alpha.x, ai = alpha.y;
      double beta, tr, ti, sr = 0, si = 0;
      if (xn2 == 0.0 && ai == 0.0) {
        beta = ar; tr = 0; ti = 0;
      } else {
        const double nrm_all = sqrt(ar * ar + ai * ai + xn2);
        beta = ar >= 0 ? -nrm_all : nrm_all;
        tr = (beta - ar) / beta;
        ti = -ai / beta;
        const double dr = ar - beta, di = ai, den = dr * dr + di * di;  // scale = 1 / (alpha - beta)
        sr = dr / den;
        si = -di / den;
      }
      hsc[0] = tr; hsc[1] = ti; hsc[2] = sr; hsc[3] = si;
      if (c == 0) {
        e[i] = (R)beta;
        tau[i] = cmake<R>((R)tr, (R)ti);
      }
    }
    __syncthreads();
    const Cx<R> tv = cmake<R>((R)hsc[0], (R)hsc[1]);
    const Cx<R> scale = cmake<R>((R)hsc[2], (R)hsc[3]);
    for (int j = i + 1 + t; j < n; j += nt) vs[j] = j == i + 1 ? cmake<R>(1, 0) : scale * col[j];
    __syncthreads();
    const int s0 = i + 1 <= c ? 0 : (i + 1 - c + G - 1) / G;  // first slot with a row >= i + 1
    {
      double dre = 0, dim = 0;
      for (int slot = s0 + warp; slot < nslots; slot += nw) {
        const int r = c + slot * G;
        const Cx<R>* row = rowp(slot);
        Cx<R> sacc = cmake<R>(0, 0);
#pragma unroll 16
        for (int j = i + 1 + lane; j < n; j += 32) cfma(sacc, row[j], vs[j]);
        R sr = sacc.x, si = sacc.y;
        for (int o = 16; o > 0; o >>= 1) {
          sr += __shfl_xor_sync(0xffffffffu, sr, o);
          si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) {
          const Cx<R> pv = tv * cmake<R>(sr, si);
          pb[r] = pv;
          ps[r] = pv;
          const Cx<R> v = vs[r];
          dre += (double)pv.x * v.x + (double)pv.y * v.y;  // conj(p) v
          dim += (double)pv.x * v.y - (double)pv.y * v.x;
        }
      }
      if (lane == 0 && (dre != 0 || dim != 0)) {
        atomicAdd(&acc[2 + 2 * par], dre);
        atomicAdd(&acc[3 + 2 * par], dim);
      }
    }
    // The update W22 -= v w^H + w v^H, w = p + a2 v, splits into the local part -p_r conj(v_j) of
    // an owned row r and the part -v_r conj(p_j + 2 Re(a2) v_j) that needs every p_j and the
    // reduced p^H v.  The local part is applied while the other CTAs reach barrier 1.
    grid_arrive(bar);
    ++nbar;
    for (int sb = s0; sb < nslots; sb += 4) {
      Cx<R>* rp[4];
      Cx<R> pr[4];
      bool ok[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int slot = sb + q;
        ok[q] = slot < nslots;
        rp[q] = rowp(ok[q] ? slot : sb);
        pr[q] = ok[q] ? ps[c + slot * G] : cmake<R>(0, 0);
      }
      for (int j0 = i + 1 + t; j0 < n; j0 += 4 * nt) {
        Cx<R> x[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = j0 + u * nt;
            if (ok[q] && j < n) x[q][u] = rp[q][j];
          }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u * nt;
          if (j >= n) break;
          const Cx<R> cvj = conj(vs[j]);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (ok[q]) rp[q][j] = x[q][u] - pr[q] * cvj;
        }
      }
    }
    grid_wait(bar, nbar * G, err, lim);
    // ---- B: rank-2 update of the owned rows
    for (int j = i + 1 + t; j < n; j += nt) ps[j] = pb[j];
    if (t == 0) {  // a2 = -tau (p^H v) / 2
      const double pr = acc[2 + 2 * par], pi = acc[3 + 2 * par], tr = hsc[0], ti = hsc[1];
      hsc[4] = -0.5 * (tr * pr - ti * pi);
      hsc[5] = -0.5 * (tr * pi + ti * pr);
      if (c == 0) {  // buffers of the other parity are free again
        acc[par] = 0;
        acc[2 + 2 * (par ^ 1)] = 0;
        acc[3 + 2 * (par ^ 1)] = 0;
      }
    }
    __syncthreads();
    const R ra2 = (R)(2.0 * hsc[4]);  // 2 Re(a2)
    {  // column i + 1 of the owned rows (one thread per row), then arrive
      double nn = 0;
      const Cx<R> uj = conj(ps[i + 1] + ra2 * vs[i + 1]);
      for (int slot = s0 + t; slot < nslots; slot += nt) {
        const int r = c + slot * G;
        Cx<R>* row = rowp(slot);
        const Cx<R> y = row[i + 1] - vs[r] * uj;
        row[i + 1] = y;
        coln[r] = y;
        if (r >= i + 3) nn += (double)abs2(y);
        if (r == i + 1) d[i + 1] = y.x;
      }
      if (nn != 0) atomicAdd(&acc[par ^ 1], nn);
    }
    grid_arrive(bar);
    ++nbar;
    // columns i + 2 .. of the owned rows, four rows at a time, four column strides per pass
    for (int sb = s0; sb < nslots; sb += 4) {
      Cx<R>* rp[4];
      Cx<R> vr[4];
      bool ok[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int slot = sb + q;
        ok[q] = slot < nslots;
        const int r = c + (ok[q] ? slot : sb) * G;
        rp[q] = rowp(ok[q] ? slot : sb);
        vr[q] = ok[q] ? vs[r] : cmake<R>(0, 0);
        // Householder vector for the back-transformation (global copy)
        if (t == 0 && ok[q] && r > i + 1) W[(long long)r * n + i] = vr[q];
      }
      for (int j0 = i + 2 + t; j0 < n; j0 += 4 * nt) {
        Cx<R> x[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = j0 + u * nt;
            if (ok[q] && j < n) x[q][u] = rp[q][j];
          }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = j0 + u * nt;
          if (j >= n) break;
          const Cx<R> uj = conj(ps[j] + ra2 * vs[j]);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (!ok[q]) continue;
            rp[q][j] = x[q][u] - vr[q] * uj;
          }
        }
      }
    }
    grid_wait(bar, nbar * G, err, lim);
  }
}

// number of eigenvalues of T smaller than x (Sturm sequence with a pivot floor)
template <typename R>
__device__ int sturm_count(int n, const R* d, const R* e, R x, R pivmin) {
  int cnt = 0;
  R q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0;
  for (int k = 1; k < n; ++k) {
    q = d[k] - x - e[k - 1] * e[k - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0;
  }
  return cnt;
}

// Eigenvalue k (ascending) of the unreduced block [blo[f], bhi[f]) that contains row f, with
// k = f - blo[f], by multisection on the block's Sturm count: one warp per row f, the 32 lanes
// evaluate 32 interior points, so every step shrinks the bracket 33-fold.
template <typename R>
__global__ void bisect_kernel(int n, const R* d, const R* e, const int* blo, const int* bhi, R* wf, R lo0, R hi0,
                              R pivmin) {
  const int f = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (f >= n) return;
  const int s = blo[f], m = bhi[f] - s, idx = f - s;
  R lo = lo0, hi = hi0;
  const R eps = sizeof(R) == 8 ? R(2.2e-16) : R(1.2e-7);
  for (int it = 0; it < 40; ++it) {
    if (hi - lo <= R(2) * eps * fmax(fabs(lo), fabs(hi)) + pivmin) break;
    const R x = lo + (hi - lo) * (R)(lane + 1) / R(33);
    const bool above = sturm_count<R>(m, d + s, e + s, x, pivmin) > idx;  // eigenvalue idx lies below x
    const unsigned ball = __ballot_sync(0xffffffffu, above);
    const int first = ball ? __ffs(ball) - 1 : 32;
    const R nlo = first == 0 ? lo : lo + (hi - lo) * (R)first / R(33);
    const R nhi = first == 32 ? hi : lo + (hi - lo) * (R)(first + 1) / R(33);
    if (!(nlo > lo || nhi < hi)) break;  // no representable progress
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) wf[f] = R(0.5) * (lo + hi);
}

// Inverse iteration for output column j: eigenvalue wf[f] of block [blo[f], bhi[f]), f = perm[j].
// (T_b - lambda I) z = b is solved by Gaussian elimination with partial pivoting on the block's
// rows only, so the vector is supported on its block and vectors of different blocks are
// exactly orthogonal.  The factors live in per-column scratch laid out [row][column] so that the
// threads of a warp access consecutive words.
template <typename R>
__global__ void inverse_iter_kernel(int n, const R* d, const R* e, const int* perm, const R* wf, const int* blo,
                                    const int* bhi, R* Z, R* U0, R* U1, R* U2, R* Lm, unsigned char* piv, R pfloor,
                                    int nv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nv) return;
  const int f = perm[j];
  const R lam = wf[f];
  const int s = blo[f], t = bhi[f];
  const long long K = n;
  for (int i = 0; i < s; ++i) Z[i * K + j] = R(0);
  for (int i = t; i < n; ++i) Z[i * K + j] = R(0);
  // factor: rows of (T_b - lam I); U has diagonal U0 and two super-diagonals U1, U2
  R a = d[s] - lam, b = t - s > 1 ? e[s] : R(0), cc = 0;  // current row: a (diag), b (super), cc (2nd super)
  for (int i = s; i < t - 1; ++i) {
    R below_sub = e[i], below_diag = d[i + 1] - lam, below_sup = (i + 2 < t) ? e[i + 1] : R(0);
    if (fabs(a) >= fabs(below_sub)) {  // no row swap
      R l = a == R(0) ? R(0) : below_sub / a;
      if (fabs(a) < pfloor) a = a < R(0) ? -pfloor : pfloor;  // perturbed pivot (|l| <= 1 either way)
      U0[i * K + j] = a; U1[i * K + j] = b; U2[i * K + j] = cc; Lm[i * K + j] = l; piv[i * K + j] = 0;
      a = below_diag - l * b;
      b = below_sup - l * cc;
      cc = 0;
    } else {  // swap rows i and i+1
      R l = a / below_sub;
      U0[i * K + j] = below_sub; U1[i * K + j] = below_diag; U2[i * K + j] = below_sup; Lm[i * K + j] = l;
      piv[i * K + j] = 1;
      R na = b - l * below_diag;
      R nb = cc - l * below_sup;
      a = na; b = nb; cc = 0;
    }
  }
  if (fabs(a) < pfloor) a = a < R(0) ? -pfloor : pfloor;
  U0[(long long)(t - 1) * K + j] = a;
  U1[(long long)(t - 1) * K + j] = 0;
  U2[(long long)(t - 1) * K + j] = 0;
  // seeded start vector (distinct per j so that equal shifts give independent vectors)
  for (int i = s; i < t; ++i) {
    unsigned long long h = (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ULL + (unsigned long long)(j + 7) * 0xD1B54A32D192ED03ULL;
    h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ULL; h ^= h >> 29;
    Z[i * K + j] = (R)((double)(h & 0xFFFFFF) / 16777216.0 + 0.5);
  }
  for (int iter = 0; iter < 3; ++iter) {
    // forward: apply L (with the recorded swaps) to z; the running entry stays in a register
    R cur = Z[s * K + j];
    for (int i = s; i < t - 1; ++i) {
      R zi = cur, zn = Z[(i + 1) * K + j];
      if (piv[i * K + j]) { R tmp = zi; zi = zn; zn = tmp; }
      Z[i * K + j] = zi;
      cur = zn - Lm[i * K + j] * zi;
    }
    Z[(t - 1) * K + j] = cur;
    // backward: U z = y
    R z2 = 0, z1 = 0;
    for (int i = t - 1; i >= s; --i) {
      R v = (Z[i * K + j] - U1[i * K + j] * z1 - U2[i * K + j] * z2) / U0[i * K + j];
      Z[i * K + j] = v;
      z2 = z1; z1 = v;
    }
    // normalise (scaled by the largest entry first, so that squares cannot overflow)
    R mx = 0, sq = 0;
    for (int i = s; i < t; ++i) mx = fmax(mx, fabs(Z[i * K + j]));
    if (!(mx > R(0)) || isinf(mx)) mx = 1;
    const R rmx = R(1) / mx;
    for (int i = s; i < t; ++i) { const R z = Z[i * K + j] * rmx; sq += z * z; }
    const R inv = rmx / sqrt(sq);
    for (int i = s; i < t; ++i) Z[i * K + j] *= inv;
  }
}

// Gram-Schmidt, in order, of the columns cidx[coff[c] .. coff[c+1]) (at most 64) of Z: one cluster
// of close eigenvalues of one unreduced block per CTA; the vectors live on rows [rlo[c], rhi[c]).
// The cluster's vectors are first gathered into ZT (transposed scratch, one contiguous row per
// vector) so that every later pass reads consecutive words; each vector is projected twice
// against all earlier members (classical Gram-Schmidt with one re-orthogonalisation, the dot
// products of a pass taken side by side by the warps), normalised, and scattered back.
template <typename R>
__global__ void __launch_bounds__(256) cluster_mgs_kernel(int n, R* Z, R* ZT, const int* cidx, const int* coff,
                                                          const int* rlo, const int* rhi) {
  __shared__ R coef[64];
  __shared__ R red[8];
  __shared__ int col[64];
  const int c0 = coff[blockIdx.x], m = coff[blockIdx.x + 1] - c0;
  const int r0 = rlo[blockIdx.x], r1 = rhi[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const long long K = n;
  if (threadIdx.x < m) col[threadIdx.x] = cidx[c0 + threadIdx.x];
  __syncthreads();
  // gather: ZT[col][r] = Z[r][col] (a warp reads the members' entries of one row together)
  for (int r = r0 + warp; r < r1; r += nw) {
    if (lane < m) ZT[col[lane] * K + r] = Z[r * K + col[lane]];
    if (lane + 32 < m) ZT[col[lane + 32] * K + r] = Z[r * K + col[lane + 32]];
  }
  __syncthreads();
  for (int a = 0; a < m; ++a) {
    R* x = ZT + col[a] * K;
    for (int pass = 0; pass < 2 && a > 0; ++pass) {
      for (int b = warp; b < a; b += nw) {
        const R* y = ZT + col[b] * K;
        R sdot = 0;
        for (int r = r0 + lane; r < r1; r += 32) sdot += y[r] * x[r];
        for (int o = 16; o > 0; o >>= 1) sdot += __shfl_xor_sync(0xffffffffu, sdot, o);
        if (lane == 0) coef[b] = sdot;
      }
      __syncthreads();
      for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        R v = x[r];
        for (int b = 0; b < a; ++b) v -= coef[b] * ZT[col[b] * K + r];
        x[r] = v;
      }
      __syncthreads();
    }
    R sq = 0;
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) sq += x[r] * x[r];
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0) red[warp] = sq;
    __syncthreads();
    R tot = 0;
    for (int q = 0; q < nw; ++q) tot += red[q];
    const R inv = tot > R(0) ? R(1) / sqrt(tot) : R(0);
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) x[r] = x[r] * inv;
    __syncthreads();
  }
  // scatter back
  for (int r = r0 + warp; r < r1; r += nw) {
    if (lane < m) Z[r * K + col[lane]] = ZT[col[lane] * K + r];
    if (lane + 32 < m) Z[r * K + col[lane + 32]] = ZT[col[lane + 32] * K + r];
  }
}

// Panel of nb Householder vectors (columns i0 .. i0+nb-1 of W) as an explicit (n - i0 - 1) x nb
// matrix: v_j has a unit entry at row i0 + j + 1, W[r][i0 + j] below it and zeros above.
template <typename R>
__global__ void panel_kernel(int n, int i0, int nb, const Cx<R>* W, Cx<R>* P) {
  const int m = n - i0 - 1;
  const long long tot = (long long)m * nb;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int rr = (int)(e / nb), j = (int)(e - (long long)rr * nb);
    int r = i0 + 1 + rr;  // global row
    Cx<R> v = cmake<R>(0, 0);
    if (r == i0 + j + 1) v = cmake<R>(1, 0);
    else if (r > i0 + j + 1) v = W[(long long)r * n + i0 + j];
    P[e] = v;
  }
}

// Compact-WY factor T (nb x nb, upper triangular) of H_{i0} ... H_{i0+nb-1} = I - V T V^H from
// S = V^H V: T[j][j] = tau_j, T[0:j, j] = -tau_j T[0:j, 0:j] S[0:j, j].
template <typename R>
__global__ void __launch_bounds__(32) wy_t_kernel(int nb, const Cx<R>* S, const Cx<R>* tau, Cx<R>* T) {
  // thread a owns row a of T; column j needs the columns before it, so j runs in order
  __shared__ Cx<R> Ts[32][33];
  __shared__ Cx<R> Ss[32][33];
  const int a = threadIdx.x;
  for (int j = 0; j < nb; ++j)
    if (a < nb) { Ss[a][j] = S[a * nb + j]; Ts[a][j] = cmake<R>(0, 0); }
  __syncwarp();
  for (int j = 0; j < nb; ++j) {
    const Cx<R> tj = tau[j];
    Cx<R> acc = cmake<R>(0, 0);
    if (a < j)
      for (int b = a; b < j; ++b) cfma(acc, Ts[a][b], Ss[b][j]);
    __syncwarp();
    if (a < j) Ts[a][j] = cmake<R>(R(0), R(0)) - tj * acc;
    if (a == j) Ts[j][j] = tj;
    __syncwarp();
  }
  for (int j = 0; j < nb; ++j)
    if (a < nb) T[a * nb + j] = Ts[a][j];
}

// Real G (nb x nb symmetric positive definite, nb <= 64) = R^T R with R upper triangular
// (right-looking Cholesky, the trailing update spread over all threads), then R^{-1} by a
// column sweep from the last row (R X = I: row k of X is fixed, then removed from the rows
// above), writes R^{-1} (nb x nb, row-major).  A non-positive pivot sets err and is clamped.
// Dynamic shared memory: two 64 x 65 arrays of R.
template <typename R>
__global__ void __launch_bounds__(256) chol_inv_kernel(int nb, const R* G, R* Rinv, int* err) {
  extern __shared__ __align__(16) unsigned char ci_smem[];
  R(*A)[65] = reinterpret_cast<R(*)[65]>(ci_smem);
  R(*X)[65] = reinterpret_cast<R(*)[65]>(ci_smem + sizeof(R) * 64 * 65);
  const int t = threadIdx.x, nt = blockDim.x;
  for (int e = t; e < nb * nb; e += nt) {
    const int r = e / nb, c = e % nb;
    A[r][c] = G[e];
    X[r][c] = r == c ? R(1) : R(0);
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    R piv = A[j][j];
    if (!(piv > R(0))) {
      if (t == 0) atomicExch(err, 2);
      piv = sizeof(R) == 8 ? R(1e-300) : R(1e-30);
    }
    const R rjj = sqrt(piv);
    __syncthreads();
    for (int c = j + 1 + t; c < nb; c += nt) A[j][c] /= rjj;
    if (t == 0) A[j][j] = rjj;
    __syncthreads();
    const int m = nb - j - 1;
    for (int e = t; e < m * m; e += nt) {
      const int r = j + 1 + e / m, c = j + 1 + e % m;
      if (c >= r) A[r][c] -= A[j][r] * A[j][c];
    }
    __syncthreads();
  }
  for (int k = nb - 1; k >= 0; --k) {
    const R inv = R(1) / A[k][k];
    for (int c = k + t; c < nb; c += nt) X[k][c] *= inv;
    __syncthreads();
    for (int e = t; e < k * (nb - k); e += nt) {
      const int r = e / (nb - k), c = k + e % (nb - k);
      X[r][c] -= A[r][k] * X[k][c];
    }
    __syncthreads();
  }
  for (int e = t; e < nb * nb; e += nt) {
    const int r = e / nb, c = e % nb;
    Rinv[e] = r <= c ? X[r][c] : R(0);
  }
}

// Z[r, 0:nb] <- Z[r, 0:nb] Ti for the rows of one tile of RT rows per CTA (Ti: nb x nb upper
// triangular, nb <= 64), in place: each CTA reads its rows into shared memory before writing back.
template <typename R>
__global__ void __launch_bounds__(256) right_mul_inplace_kernel(int m, int nb, R* Z, long long ldz, const R* Ti) {
  constexpr int RT = sizeof(R) == 8 ? 16 : 64;
  __shared__ R Zs[RT][65];
  __shared__ R Ts[64][65];
  const int r0 = blockIdx.x * RT;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) Ts[e / nb][e % nb] = Ti[e];
  for (int e = threadIdx.x; e < RT * nb; e += blockDim.x) {
    const int rr = e / nb, c = e % nb;
    Zs[rr][c] = r0 + rr < m ? Z[(long long)(r0 + rr) * ldz + c] : R(0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RT * nb; e += blockDim.x) {
    const int rr = e / nb, c = e % nb;
    if (r0 + rr >= m) continue;
    R acc = 0;
    for (int k = 0; k <= c; ++k) acc += Zs[rr][k] * Ts[k][c];
    Z[(long long)(r0 + rr) * ldz + c] = acc;
  }
}

template <typename R>
__global__ void real_to_complex_kernel(long long cnt, const R* Z, Cx<R>* X) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt; e += (long long)gridDim.x * blockDim.x)
    X[e] = cmake<R>(Z[e], R(0));
}
}  // namespace

size_t tri_workspace_bytes(int n, int real_bytes) {
  size_t c = 2 * (size_t)real_bytes, nn = (size_t)n * n;
  size_t b = 0;
  b += nn * c;                   // W
  b += nn * c;                   // X (back-transform)
  b += 5 * nn * real_bytes;      // Z, U0, U1, U2, L
  b += nn;                       // pivots
  b += 8 * (size_t)n * c;        // d, e, tau, v, p, w, cluster bounds
  b += 2 * (size_t)n * c + 256;  // column buffer of the reduction (two parities)
  b += 6 * (size_t)n * 8 + 8 * 256;  // block eigenvalues, block bounds, permutation, cluster lists
  b += 3 * 32 * (size_t)n * c + 2 * 32 * 32 * c + 7 * 256;  // WY panel, Y1, Y2, S, T
  b += (size_t)(8 + 1) * n * 64 * (c / 2) + 2 * 64 * 64 * (c / 2) + 5 * 256;  // real orthonormalisation
  b += (size_t)16 * n * 32 * c + 256;                                          // split-K partials
  return b + 64 * 1024;
}

// Returns 1, -2 if a grid barrier of the reduction timed out, -3 if the eigenvectors could not be
// orthonormalised, -4 on a CUDA error.  nvec > 0: only the first nvec eigenvectors are formed.
template <typename R>
int eigh_tridiag(cudaStream_t st, int n, const Cx<R>* A, long long lda, R* w, Cx<R>* V, long long ldv, void* workspace,
                 int nvec) {
  nvec = (nvec <= 0 || nvec > n) ? n : nvec;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  auto take = [&](size_t bytes) { unsigned char* p = ws; ws += (bytes + 255) & ~size_t(255); return p; };
  const size_t nn = (size_t)n * n;
  Cx<R>* Wm = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * nn));
  Cx<R>* X = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * nn));
  R* Z = reinterpret_cast<R*>(take(sizeof(R) * nn));
  R* U0 = reinterpret_cast<R*>(take(sizeof(R) * nn));
  R* U1 = reinterpret_cast<R*>(take(sizeof(R) * nn));
  R* U2 = reinterpret_cast<R*>(take(sizeof(R) * nn));
  R* Lm = reinterpret_cast<R*>(take(sizeof(R) * nn));
  unsigned char* piv = take(nn);
  R* dv = reinterpret_cast<R*>(take(sizeof(R) * n));
  R* ev = reinterpret_cast<R*>(take(sizeof(R) * n));
  Cx<R>* tau = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * n));
  Cx<R>* pb = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * n));
  Cx<R>* colbuf = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * 2 * (size_t)n));
  Cx<R>* Pn = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)n * 32));
  Cx<R>* Sm = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * 32 * 32));
  Cx<R>* Tm = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * 32 * 32));
  Cx<R>* Y1 = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)n * 32));
  Cx<R>* Y2 = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * (size_t)n * 32));
  const size_t wc_elems = (size_t)16 * n * 32;  // split-K partial products of the WY panels
  Cx<R>* Wc = reinterpret_cast<Cx<R>*>(take(sizeof(Cx<R>) * wc_elems));
  const size_t wr_elems = (size_t)8 * n * 64;
  R* Wr = reinterpret_cast<R*>(take(sizeof(R) * wr_elems));
  R* Cr = reinterpret_cast<R*>(take(sizeof(R) * (size_t)n * 64));
  R* Sr = reinterpret_cast<R*>(take(sizeof(R) * 64 * 64));
  R* Tr = reinterpret_cast<R*>(take(sizeof(R) * 64 * 64));
  R* wf = reinterpret_cast<R*>(take(sizeof(R) * n));
  int* blo = reinterpret_cast<int*>(take(sizeof(int) * n));
  int* bhi = reinterpret_cast<int*>(take(sizeof(int) * n));
  int* perm = reinterpret_cast<int*>(take(sizeof(int) * n));
  int* cl_idx = reinterpret_cast<int*>(take(sizeof(int) * n));
  int* cl_off = reinterpret_cast<int*>(take(sizeof(int) * (n + 1)));
  int* cl_rlo = reinterpret_cast<int*>(take(sizeof(int) * n));
  int* cl_rhi = reinterpret_cast<int*>(take(sizeof(int) * n));
  double* acc = reinterpret_cast<double*>(take(sizeof(double) * 8));
  unsigned* bar = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * 4));
  int* d_err = reinterpret_cast<int*>(take(sizeof(int) * 4));
  cudaMemsetAsync(acc, 0, sizeof(double) * 8, st);
  cudaMemsetAsync(bar, 0, sizeof(unsigned) * 4, st);
  cudaMemsetAsync(d_err, 0, sizeof(int) * 4, st);
  // ---- 1. tridiagonalisation (cooperative persistent kernel, one CTA per SM)
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // shared memory: v and p of the current column plus as many owned rows as fit
  const size_t row_bytes = sizeof(Cx<R>) * (size_t)n;
  const size_t smem_cap = 220 * 1024;
  if (2 * row_bytes > smem_cap) return -4;
  // about a dozen rows per CTA, at most one CTA per SM: below n ~ 1800 fewer CTAs take part in each
  // grid barrier, all their rows fit in shared memory, and the SMs left over can run the
  // reductions of other handles (other streams) at the same time
  int grid = std::min(sms, std::max(16, (n + 11) / 12));
  const int slots = (n + grid - 1) / grid;
  int s_fit = (int)std::min<size_t>((size_t)slots, (smem_cap - 2 * row_bytes) / row_bytes);
  const size_t hsm = (2 + (size_t)s_fit) * row_bytes;
  // the attribute is a property of the kernel, shared by every host thread: it is raised once to
  // the largest size any launch uses (setting it per launch would race between handles)
  static std::once_flag attr_once;
  static bool attr_ok = false;
  std::call_once(attr_once, [smem_cap] {
    attr_ok = cudaFuncSetAttribute(hetrd_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cap) ==
              cudaSuccess;
  });
  if (!attr_ok || hsm > smem_cap) return -4;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hetrd_kernel<R>, 512, hsm);
  if (per_sm < 1) return -4;
  int n_ = n;
  long long lda_ = lda;
  long long lim = wait_limit_cycles();
  void* args[] = {&n_, (void*)&A, &lda_, &Wm, &dv, &ev, &tau, &pb, &colbuf, &acc, &bar, &d_err, &lim, &s_fit};
  kt_begin(KT_HETRD, st);
  if (cudaLaunchCooperativeKernel((void*)hetrd_kernel<R>, dim3(grid), dim3(512), args, hsm, st) != cudaSuccess) return -4;
  kt_end(KT_HETRD, st);
  // algorithmic work: the real flops of a complex Hermitian tridiagonal reduction, 16 n^3 / 3
  kt_add_work(KT_HETRD, 16.0 / 3.0 * (double)n * n * n);
  count_launch();
  // ---- 2. split T at negligible off-diagonal entries (|e_i| <= 32 eps ||T||, an absolute
  // perturbation of the order of the reduction's own backward error); eigenvalues of each
  // unreduced block by bisection (Gershgorin interval from the host copy of T)
  std::vector<R> hd(n), he(n);
  int herr = 0;
  cudaMemcpyAsync(hd.data(), dv, sizeof(R) * n, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(he.data(), ev, sizeof(R) * n, cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return -4;
  if (herr != 0) return -2;
  double lo = 1e300, hi = -1e300, emax2 = 0, tnorm = 0;
  for (int i = 0; i < n; ++i) {
    double off = (i > 0 ? std::fabs((double)he[i - 1]) : 0) + (i < n - 1 ? std::fabs((double)he[i]) : 0);
    lo = std::min(lo, (double)hd[i] - off);
    hi = std::max(hi, (double)hd[i] + off);
    if (i < n - 1) emax2 = std::max(emax2, (double)he[i] * he[i]);
    tnorm = std::max(tnorm, std::fabs((double)hd[i]) + off);
  }
  const double eps = sizeof(R) == 8 ? 2.2e-16 : 1.2e-7;
  const double safmin = sizeof(R) == 8 ? 2.3e-308 : 1.2e-38;
  const R pivmin = (R)(safmin * std::max(1.0, emax2) * 4);
  lo -= 4 * eps * tnorm + 2 * pivmin;
  hi += 4 * eps * tnorm + 2 * pivmin;
  const double tol_split = 32 * eps * tnorm;
  std::vector<int> hblo(n), hbhi(n);
  for (int i = 0, s0 = 0; i < n; ++i) {
    const bool last = i == n - 1 || std::fabs((double)he[i]) <= tol_split;
    if (i < n - 1 && last) he[i] = R(0);
    if (last) {
      for (int r = s0; r <= i; ++r) { hblo[r] = s0; hbhi[r] = i + 1; }
      s0 = i + 1;
    }
  }
  cudaMemcpyAsync(ev, he.data(), sizeof(R) * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(blo, hblo.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(bhi, hbhi.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
  kt_begin(KT_TRIVEC, st);
  bisect_kernel<R><<<(n + 3) / 4, 128, 0, st>>>(n, dv, ev, blo, bhi, wf, (R)lo, (R)hi, pivmin);
  kt_end(KT_TRIVEC, st);
  count_launch();
  // all eigenvalues in descending order (ties in row order), w and the column permutation
  std::vector<R> hwf(n);
  cudaMemcpyAsync(hwf.data(), wf, sizeof(R) * n, cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return -4;
  std::vector<int> hperm(n);
  for (int i = 0; i < n; ++i) hperm[i] = i;
  std::stable_sort(hperm.begin(), hperm.end(), [&](int x, int y) { return hwf[x] > hwf[y]; });
  std::vector<R> hw(n);
  for (int j = 0; j < n; ++j) hw[j] = hwf[hperm[j]];
  cudaMemcpyAsync(perm, hperm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(w, hw.data(), sizeof(R) * n, cudaMemcpyHostToDevice, st);
  // ---- 3. eigenvectors of the blocks by inverse iteration
  // pivots of (T_b - lambda I) are kept at least eps ||T|| in magnitude: a perturbation of the size
  // of the eigenvalue error that also bounds the growth of the solution
  const R pfloor = (R)std::max(eps * tnorm, (double)pivmin);
  kt_begin(KT_TRIVEC, st);
  inverse_iter_kernel<R><<<(nvec + 127) / 128, 128, 0, st>>>(n, dv, ev, perm, wf, blo, bhi, Z, U0, U1, U2, Lm, piv,
                                                              pfloor, nvec);
  kt_end(KT_TRIVEC, st);
  count_launch();
  // ---- 4. clusters of close eigenvalues: re-orthogonalise
  // clusters: within one unreduced block, runs of eigenvalues closer than ortol (vectors of
  // different blocks are orthogonal by construction), re-orthogonalised in chunks of at most 64
  const double ortol = (sizeof(R) == 8 ? 1e-10 : 1e-6) * std::max(tnorm, 1e-300);
  std::vector<int> cidx, coff(1, 0), crlo, crhi;
  {
    std::vector<int> order(nvec);  // computed positions grouped by block, descending within a block
    for (int j = 0; j < nvec; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hblo[hperm[x]] < hblo[hperm[y]]; });
    for (int q = 0; q < nvec;) {
      const int blk = hblo[hperm[order[q]]];
      int q1 = q + 1;
      while (q1 < nvec && hblo[hperm[order[q1]]] == blk && (double)hw[order[q1 - 1]] - (double)hw[order[q1]] < ortol) ++q1;
      for (int a0 = q; q1 - q > 1 && a0 < q1; a0 += 64) {
        for (int a = a0; a < std::min(q1, a0 + 64); ++a) cidx.push_back(order[a]);
        coff.push_back((int)cidx.size());
        crlo.push_back(blk);
        crhi.push_back(hbhi[hperm[order[q]]]);
      }
      q = q1;
    }
  }
  const size_t ncl = crlo.size();
  if (ncl > 0) {
    cudaMemcpyAsync(cl_idx, cidx.data(), sizeof(int) * cidx.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(cl_off, coff.data(), sizeof(int) * coff.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(cl_rlo, crlo.data(), sizeof(int) * ncl, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(cl_rhi, crhi.data(), sizeof(int) * ncl, cudaMemcpyHostToDevice, st);
    kt_begin(KT_TRIVEC, st);
    cluster_mgs_kernel<R><<<(unsigned)ncl, 256, 0, st>>>(n, Z, U0, cl_idx, cl_off, cl_rlo, cl_rhi);  // U0: free LU scratch
    kt_end(KT_TRIVEC, st);
    count_launch();
  }
  // ---- 5. back-transformation
  {
    // X = Q Z with Q = H_0 ... H_{n-2}, applied block by block from the last one:
    // X[i0+1:, :] <- (I - V T V^H) X[i0+1:, :]
    const int NB = 32;
    const long long nn_ = (long long)n * n;
    // Orthonormalise the eigenvectors of T (real, columns of Z) in descending-eigenvalue order:
    // each block of 64 columns is projected twice against all earlier columns (block classical
    // Gram-Schmidt) and then made orthonormal by Cholesky-QR, also twice.  Inverse iteration
    // leaves the vectors of well-separated eigenvalues orthogonal to working precision, so they
    // are unchanged; the vectors of close eigenvalues are made orthogonal.
    const int ci_smem = 2 * 64 * 65 * (int)sizeof(R);
    static std::once_flag ci_once;
    static bool ci_ok = false;
    std::call_once(ci_once, [ci_smem] {
      ci_ok = cudaFuncSetAttribute(chol_inv_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, ci_smem) ==
              cudaSuccess;
    });
    if (!ci_ok) return -4;
    // a fixed launch sequence for given sizes and buffers (all inside the workspace): replayed as a
    // CUDA graph where possible
    GraphKey key{{2, n, nvec, (long long)sizeof(R), (long long)(uintptr_t)workspace, (long long)(uintptr_t)V, ldv,
                  (long long)(uintptr_t)st, 0, 0, 0, 0}};
    const int bt = replay_or_issue(st, key, [&](cudaStream_t cs) -> int {
    for (int b0 = 0; b0 < nvec; b0 += 64) {
      const int nb = std::min(64, nvec - b0);
      R* Zb = Z + b0;
      for (int pass = 0; pass < 2 && b0 > 0; ++pass) {
        rgemm<R>(cs, b0, nb, n, R(1), Z, n, true, Zb, n, false, R(0), Cr, nb, Wr, wr_elems);
        rgemm<R>(cs, n, nb, b0, R(-1), Z, n, false, Cr, nb, false, R(1), Zb, n, Wr, wr_elems);
      }
      for (int pass = 0; pass < 2; ++pass) {
        rgemm<R>(cs, nb, nb, n, R(1), Zb, n, true, Zb, n, false, R(0), Sr, nb, Wr, wr_elems);
        chol_inv_kernel<R><<<1, 256, ci_smem, cs>>>(nb, Sr, Tr, d_err + 1);
        right_mul_inplace_kernel<R><<<(n + (sizeof(R) == 8 ? 15 : 63)) / (sizeof(R) == 8 ? 16 : 64), 256, 0, cs>>>(
            n, nb, Zb, n, Tr);
        count_launch(2);
      }
    }
      real_to_complex_kernel<R><<<1024, 256, 0, cs>>>(nn_, Z, X);
    count_launch();
    const Cx<R> one = cmake<R>(1, 0), zero = cmake<R>(0, 0), mone = cmake<R>(-1, 0);
    const int nref = n - 1;
    for (int i0 = ((nref - 1) / NB) * NB; i0 >= 0; i0 -= NB) {
      const int nb = std::min(NB, nref - i0);
      const int m = n - i0 - 1;
      panel_kernel<R><<<256, 256, 0, cs>>>(n, i0, nb, Wm, Pn);
      count_launch();
      // S = V^H V, T from S, Y = V^H X, Y2 = T Y, X -= V Y2
      gemm_splitk<R>(cs, nb, nb, m, one, transposed<R>(Pn, nb, true), rowmajor<R>(Pn, nb), zero, rowmajor<R>(Sm, nb),
                     Wc, wc_elems);
      wy_t_kernel<R><<<1, 32, 0, cs>>>(nb, Sm, tau + i0, Tm);
      count_launch();
      Cx<R>* Xs = X + (long long)(i0 + 1) * n;
      gemm_splitk<R>(cs, nb, nvec, m, one, transposed<R>(Pn, nb, true), rowmajor<R>(Xs, n), zero, rowmajor<R>(Y1, n),
                     Wc, wc_elems);
      gemm<R>(cs, nb, nvec, nb, one, rowmajor<R>(Tm, nb), rowmajor<R>(Y1, n), zero, rowmajor<R>(Y2, n));
      gemm<R>(cs, m, nvec, nb, mone, rowmajor<R>(Pn, nb), rowmajor<R>(Y2, n), one, rowmajor<R>(Xs, n));
    }
    copy_view<R, R>(cs, n, nvec, rowmajor<R>(X, n), rowmajor<R>(V, ldv));
    return 0;
    });
    if (bt != 0) return -4;
  }
  int cherr = 0;
  cudaMemcpyAsync(&cherr, d_err + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return -4;
  return cherr != 0 ? -3 : 1;
}

template int eigh_tridiag<double>(cudaStream_t, int, const z128*, long long, double*, z128*, long long, void*, int);
template int eigh_tridiag<float>(cudaStream_t, int, const c64*, long long, float*, c64*, long long, void*, int);

}  // namespace mpsgb
