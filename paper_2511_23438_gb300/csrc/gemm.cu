// CUDA-core complex GEMM over two-level strided views, batched.
//   C(i, j) = alpha * sum_k A(i, k) B(k, j) + beta * C(i, j)
// Used for every contraction of the FP64 form and for the small (bond x bond)
// products of the truncation core in all forms.  64x64 output tile per CTA,
// 256 threads each owning a 4x4 sub-tile, K staged through shared memory.
#include <algorithm>

#include "common.cuh"
#include "kernels.hpp"

namespace mpsgb {

thread_local int g_gemm_site = KT_GEMM;

namespace {
constexpr int BM = 64, BN = 64, BK = 16;  // tile of the real split-K GEMM below

// Complex GEMM tile kernel: a (16 TM) x (16 TM) output tile per CTA of 256 threads, each thread a
// TM x TM register tile (rows g*64 + 4*ty + q, columns g*64 + 4*tx + q for g < TM/4, q < 4), K
// staged through shared memory in slices of CK with the next slice prefetched into registers
// while the current one is multiplied.  Any two-level strided view is accepted; loads are
// coalesced along whichever of the operand's indices is contiguous.
constexpr int CK = 8;
template <typename R, int TM>
struct CTile {
  static constexpr int T = 16 * TM;          // tile edge
  static constexpr int LD = T + 16 / (int)sizeof(R);  // padded row (16-byte multiple)
  static constexpr int PER = T * CK / 256;   // operand elements loaded per thread per slice
};

template <typename R>
__device__ __forceinline__ void ld4(const Cx<R>* p, Cx<R>* out) {  // 4 consecutive complex, 16-byte aligned
  if constexpr (sizeof(R) == 4) {
    const float4 u = reinterpret_cast<const float4*>(p)[0], v = reinterpret_cast<const float4*>(p)[1];
    out[0] = cmake<R>(u.x, u.y); out[1] = cmake<R>(u.z, u.w); out[2] = cmake<R>(v.x, v.y); out[3] = cmake<R>(v.z, v.w);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double2 u = reinterpret_cast<const double2*>(p)[q];
      out[q] = cmake<R>(u.x, u.y);
    }
  }
}

template <typename R, int TM>
__global__ void __launch_bounds__(256, 1) cgemm_kernel(int M, int N, int K, Cx<R> alpha, View<R> A, View<R> B,
                                                       Cx<R> beta, View<R> C, long long sA, long long sB,
                                                       long long sC, int kchunk) {
  using Tl = CTile<R, TM>;
  constexpr int T = Tl::T, LD = Tl::LD, PER = Tl::PER, G = TM / 4;
  __shared__ __align__(16) Cx<R> As[2][CK][LD];
  __shared__ __align__(16) Cx<R> Bs[2][CK][LD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * T, j0 = blockIdx.x * T;
  const long long z = blockIdx.z;
  const Cx<R>* Ap = A.ptr + z * sA;
  const Cx<R>* Bp = B.ptr + z * sB;
  Cx<R>* Cp = C.ptr + z * sC;
  // split K (kchunk > 0): slice z covers k in [z kchunk, (z+1) kchunk); A and B are shared
  const int kbeg = kchunk > 0 ? (int)z * kchunk : 0;
  const int kend = kchunk > 0 ? min(K, kbeg + kchunk) : K;
  // A: contiguous along k (row-major) -> k fastest in the thread mapping, else i fastest
  const bool a_kfast = A.col.inner == 0 && A.col.stride == 1;
  const bool b_kfast = B.row.inner == 0 && B.row.stride == 1;
  int ai[PER], ak[PER], bk[PER], bj[PER];
  long long aro[PER], bco[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int e = tid + 256 * u;
    if (a_kfast) { ak[u] = e % CK; ai[u] = e / CK; } else { ai[u] = e % T; ak[u] = e / T; }
    if (b_kfast) { bk[u] = e % CK; bj[u] = e / CK; } else { bj[u] = e % T; bk[u] = e / T; }
    aro[u] = (i0 + ai[u] < M) ? A.row(i0 + ai[u]) : -1;
    bco[u] = (j0 + bj[u] < N) ? B.col(j0 + bj[u]) : -1;
  }
  Cx<R> pa[PER], pb[PER];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int k = k0 + ak[u];
      Cx<R> v = cmake<R>(0, 0);
      if (aro[u] >= 0 && k < kend) { v = Ap[aro[u] + A.col(k)]; if (A.conj) v.y = -v.y; }
      pa[u] = v;
      const int kb = k0 + bk[u];
      Cx<R> w = cmake<R>(0, 0);
      if (bco[u] >= 0 && kb < kend) { w = Bp[B.row(kb) + bco[u]]; if (B.conj) w.y = -w.y; }
      pb[u] = w;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      As[buf][ak[u]][ai[u]] = pa[u];
      Bs[buf][bk[u]][bj[u]] = pb[u];
    }
  };
  Cx<R> acc[TM][TM];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) acc[a][b] = cmake<R>(0, 0);
  fetch(kbeg);
  stash(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = kbeg; k0 < kend; k0 += CK) {
    const bool more = k0 + CK < kend;
    if (more) fetch(k0 + CK);
#pragma unroll
    for (int kk = 0; kk < CK; ++kk) {
      Cx<R> a[TM], b[TM];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        ld4<R>(&As[buf][kk][g * 64 + 4 * ty], a + 4 * g);
        ld4<R>(&Bs[buf][kk][g * 64 + 4 * tx], b + 4 * g);
      }
#pragma unroll
      for (int s = 0; s < TM; ++s)
#pragma unroll
        for (int t = 0; t < TM; ++t) cfma(acc[s][t], a[s], b[t]);
    }
    if (more) {
      stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
  const bool use_beta = (beta.x != R(0) || beta.y != R(0));
#pragma unroll
  for (int s = 0; s < TM; ++s) {
    const int i = i0 + (s / 4) * 64 + 4 * ty + (s % 4);
    if (i >= M) continue;
    const long long ro = C.row(i);
#pragma unroll
    for (int t = 0; t < TM; ++t) {
      const int j = j0 + (t / 4) * 64 + 4 * tx + (t % 4);
      if (j >= N) continue;
      const long long o = ro + C.col(j);
      Cx<R> v = alpha * acc[s][t];
      if (use_beta) v = v + beta * Cp[o];
      Cp[o] = v;
    }
  }
}
// C = alpha * sum_z W[z] + beta * C (the split-K partial products, summed in a fixed order)
template <typename R>
__global__ void csplit_reduce_kernel(int M, int N, int splits, Cx<R> alpha, const Cx<R>* W, Cx<R> beta, View<R> C) {
  const long long tot = (long long)M * N;
  const bool use_beta = (beta.x != R(0) || beta.y != R(0));
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    Cx<R> s = cmake<R>(0, 0);
    for (int zz = 0; zz < splits; ++zz) s = s + W[zz * tot + e];
    const int i = (int)(e / N), j = (int)(e % N);
    const long long o = C.row(i) + C.col(j);
    Cx<R> v = alpha * s;
    if (use_beta) v = v + beta * C.ptr[o];
    C.ptr[o] = v;
  }
}
}  // namespace

template <typename R>
void gemm_splitk(cudaStream_t st, int M, int N, int K, Cx<R> alpha, View<R> A, View<R> B, Cx<R> beta, View<R> C,
                 Cx<R>* ws, size_t ws_elems) {
  if (M <= 0 || N <= 0) return;
  const long long tiles = (long long)((M + 63) / 64) * ((N + 63) / 64);
  int splits = (int)std::min<long long>((2 * 152 + tiles - 1) / tiles, K / 64);
  while (splits > 1 && (size_t)splits * M * N > ws_elems) --splits;
  if (splits <= 1 || ws == nullptr) {
    gemm<R>(st, M, N, K, alpha, A, B, beta, C);
    return;
  }
  const int kchunk = ((K + splits - 1) / splits + CK - 1) / CK * CK;
  splits = (K + kchunk - 1) / kchunk;
  View<R> W = rowmajor<R>(ws, N);
  kt_begin(g_gemm_site, st);
  dim3 grid((N + 63) / 64, (M + 63) / 64, splits);
  cgemm_kernel<R, 4><<<grid, 256, 0, st>>>(M, N, K, cmake<R>(1, 0), A, B, cmake<R>(0, 0), W, 0, 0, (long long)M * N,
                                           kchunk);
  const long long tot = (long long)M * N;
  csplit_reduce_kernel<R><<<(unsigned)std::min<long long>((tot + 255) / 256, 1216), 256, 0, st>>>(M, N, splits, alpha,
                                                                                                  ws, beta, C);
  kt_end(g_gemm_site, st);
  kt_add_work(g_gemm_site, 8.0 * M * N * (double)K);
  count_launch(2);
}

template void gemm_splitk<double>(cudaStream_t, int, int, int, z128, View<double>, View<double>, z128, View<double>,
                                  z128*, size_t);
template void gemm_splitk<float>(cudaStream_t, int, int, int, c64, View<float>, View<float>, c64, View<float>, c64*,
                                 size_t);

template <typename R>
void gemm(cudaStream_t st, int M, int N, int K, Cx<R> alpha, View<R> A, View<R> B, Cx<R> beta, View<R> C, int batch,
          long long sA, long long sB, long long sC) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {  // C = beta * C
    scale_view(st, M, N, beta, C, batch, sC);
    return;
  }
  kt_begin(g_gemm_site, st);
  // 128 x 128 tiles (FP32) when they alone fill the GPU, else 64 x 64 tiles
  const long long t128 = (long long)((M + 127) / 128) * ((N + 127) / 128) * batch;
  bool big = false;
  if constexpr (sizeof(R) == 4) {
    if (t128 >= 148) {
      big = true;
      dim3 grid((N + 127) / 128, (M + 127) / 128, batch);
      cgemm_kernel<R, 8><<<grid, 256, 0, st>>>(M, N, K, alpha, A, B, beta, C, sA, sB, sC, 0);
    }
  }
  if (!big) {
    dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
    cgemm_kernel<R, 4><<<grid, 256, 0, st>>>(M, N, K, alpha, A, B, beta, C, sA, sB, sC, 0);
  }
  kt_end(g_gemm_site, st);
  kt_add_work(g_gemm_site, 8.0 * M * N * (double)K * batch);
  count_launch();
}

// ---------------------------------------------------------------- real GEMM with split-K
// C = alpha op(A) op(B) + beta C on plain row-major real matrices (op = transpose if ta / tb).
// Same 64 x 64 tile as the complex kernel.  For tall-skinny products with long K the K range is
// split over grid.z into a workspace and reduced in a fixed order (deterministic).
namespace {
template <typename R>
__global__ void __launch_bounds__(256) rgemm_kernel(int M, int N, int K, int kchunk, R alpha, const R* A, long long lda,
                                                    int ta, const R* B, long long ldb, int tb, R beta, R* C,
                                                    long long ldc, long long sCz) {
  __shared__ R As[BK][BM + 1];
  __shared__ R Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  R* Cz = C + (long long)blockIdx.z * sCz;
  R acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = R(0);
  for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u;
      // coalesced along the contiguous index of each operand
      int ii, kk;
      if (ta) { kk = e / BM; ii = e % BM; } else { ii = e / BK; kk = e % BK; }
      int i = i0 + ii, k = k0 + kk;
      R v = R(0);
      if (i < M && k < ke) v = ta ? A[(long long)k * lda + i] : A[(long long)i * lda + k];
      As[kk][ii] = v;
      int jj;
      if (tb) { jj = e / BK; kk = e % BK; } else { kk = e / BN; jj = e % BN; }
      int j = j0 + jj;
      k = k0 + kk;
      R w = R(0);
      if (k < ke && j < N) w = tb ? B[(long long)j * ldb + k] : B[(long long)k * ldb + j];
      Bs[kk][jj] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R a[4], b[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) { a[t] = As[kk][ty + 16 * t]; b[t] = Bs[kk][tx + 16 * t]; }
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[s][t] = fma(a[s], b[t], acc[s][t]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int i = i0 + ty + 16 * s;
    if (i >= M) continue;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = j0 + tx + 16 * t;
      if (j >= N) continue;
      R* o = Cz + (long long)i * ldc + j;
      *o = beta != R(0) ? alpha * acc[s][t] + beta * *o : alpha * acc[s][t];
    }
  }
}

template <typename R>
__global__ void rgemm_reduce_kernel(int M, int N, int splits, R alpha, const R* W, R beta, R* C, long long ldc) {
  const long long tot = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    R s = R(0);
    for (int z = 0; z < splits; ++z) s += W[z * tot + e];
    R* o = C + (e / N) * ldc + e % N;
    *o = beta != R(0) ? alpha * s + beta * *o : alpha * s;
  }
}
}  // namespace

template <typename R>
void rgemm(cudaStream_t st, int M, int N, int K, R alpha, const R* A, long long lda, bool ta, const R* B, long long ldb,
           bool tb, R beta, R* C, long long ldc, R* ws, size_t ws_elems) {
  if (M <= 0 || N <= 0) return;
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  int splits = 1;
  if (K > 2 * BK * 8 && ws != nullptr) {
    splits = std::max(1, std::min((304 + tiles - 1) / tiles, K / 128));
    while (splits > 1 && (size_t)splits * M * N > ws_elems) --splits;
  }
  const int kchunk = splits > 1 ? ((K + splits - 1) / splits + BK - 1) / BK * BK : std::max(K, 1);
  splits = splits > 1 ? (K + kchunk - 1) / kchunk : 1;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
  kt_begin(g_gemm_site, st);
  if (splits == 1) {
    rgemm_kernel<R><<<grid, 256, 0, st>>>(M, N, K, kchunk, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc, 0);
    count_launch();
  } else {
    rgemm_kernel<R><<<grid, 256, 0, st>>>(M, N, K, kchunk, R(1), A, lda, ta, B, ldb, tb, R(0), ws, N,
                                         (long long)M * N);
    const long long tot = (long long)M * N;
    rgemm_reduce_kernel<R><<<(unsigned)std::min<long long>((tot + 255) / 256, 1216), 256, 0, st>>>(M, N, splits, alpha,
                                                                                                    ws, beta, C, ldc);
    count_launch();
    count_launch();
  }
  kt_end(g_gemm_site, st);
  kt_add_work(g_gemm_site, 2.0 * M * N * (double)K);
}

template void rgemm<double>(cudaStream_t, int, int, int, double, const double*, long long, bool, const double*,
                            long long, bool, double, double*, long long, double*, size_t);
template void rgemm<float>(cudaStream_t, int, int, int, float, const float*, long long, bool, const float*, long long,
                           bool, float, float*, long long, float*, size_t);

template void gemm<double>(cudaStream_t, int, int, int, z128, View<double>, View<double>, z128, View<double>, int,
                           long long, long long, long long);
template void gemm<float>(cudaStream_t, int, int, int, c64, View<float>, View<float>, c64, View<float>, int, long long,
                          long long, long long);

}  // namespace mpsgb
