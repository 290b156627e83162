// CUDA-core complex GEMM over two-level strided views, batched.
//   C(i, j) = alpha * sum_k A(i, k) B(k, j) + beta * C(i, j)
// Used for every contraction of the FP64 form and for the small (bond x bond)
// products of the truncation core in all forms.  64x64 output tile per CTA,
// 256 threads each owning a 4x4 sub-tile, K staged through shared memory.
#include "common.cuh"
#include "kernels.hpp"

namespace mpsgb {

namespace {
constexpr int BM = 64, BN = 64, BK = 16;

template <typename R>
__global__ void __launch_bounds__(256) cgemm_kernel(int M, int N, int K, Cx<R> alpha, View<R> A, View<R> B, Cx<R> beta,
                                                    View<R> C, long long sA, long long sB, long long sC) {
  __shared__ Cx<R> As[BK][BM + 1];
  __shared__ Cx<R> Bs[BK][BN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
  const long long z = blockIdx.z;
  const Cx<R>* Ap = A.ptr + z * sA;
  const Cx<R>* Bp = B.ptr + z * sB;
  Cx<R>* Cp = C.ptr + z * sC;
  Cx<R> acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = cmake<R>(0, 0);
  // row offsets of A and column offsets of B are fixed per thread
  long long arow[4];
  int ai[4], ak[4], bk[4], bj[4];
  long long bcol[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    int e = tid + 256 * u;
    ai[u] = e / BK; ak[u] = e % BK;
    arow[u] = (i0 + ai[u] < M) ? A.row(i0 + ai[u]) : 0;
    bk[u] = e / BN; bj[u] = e % BN;
    bcol[u] = (j0 + bj[u] < N) ? B.col(j0 + bj[u]) : 0;
  }
  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      int i = i0 + ai[u], k = k0 + ak[u];
      Cx<R> v = cmake<R>(0, 0);
      if (i < M && k < K) { v = Ap[arow[u] + A.col(k)]; if (A.conj) v.y = -v.y; }
      As[ak[u]][ai[u]] = v;
      int kb = k0 + bk[u], j = j0 + bj[u];
      Cx<R> w = cmake<R>(0, 0);
      if (kb < K && j < N) { w = Bp[B.row(kb) + bcol[u]]; if (B.conj) w.y = -w.y; }
      Bs[bk[u]][bj[u]] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Cx<R> a[4], b[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) { a[t] = As[kk][ty + 16 * t]; b[t] = Bs[kk][tx + 16 * t]; }
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int t = 0; t < 4; ++t) cfma(acc[s][t], a[s], b[t]);
    }
    __syncthreads();
  }
  const bool use_beta = (beta.x != R(0) || beta.y != R(0));
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    int i = i0 + ty + 16 * s;
    if (i >= M) continue;
    long long ro = C.row(i);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      int j = j0 + tx + 16 * t;
      if (j >= N) continue;
      long long o = ro + C.col(j);
      Cx<R> v = alpha * acc[s][t];
      if (use_beta) v = v + beta * Cp[o];
      Cp[o] = v;
    }
  }
}
}  // namespace

template <typename R>
void gemm(cudaStream_t st, int M, int N, int K, Cx<R> alpha, View<R> A, View<R> B, Cx<R> beta, View<R> C, int batch,
          long long sA, long long sB, long long sC) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {  // C = beta * C
    scale_view(st, M, N, beta, C, batch, sC);
    return;
  }
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  kt_begin(KT_GEMM, st);
  cgemm_kernel<R><<<grid, 256, 0, st>>>(M, N, K, alpha, A, B, beta, C, sA, sB, sC);
  kt_end(KT_GEMM, st);
  kt_add_work(KT_GEMM, 8.0 * M * N * (double)K * batch);
  count_launch();
}

template void gemm<double>(cudaStream_t, int, int, int, z128, View<double>, View<double>, z128, View<double>, int,
                           long long, long long, long long);
template void gemm<float>(cudaStream_t, int, int, int, c64, View<float>, View<float>, c64, View<float>, int, long long,
                          long long, long long);

}  // namespace mpsgb
