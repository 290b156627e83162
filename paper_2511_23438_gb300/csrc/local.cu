// Bandwidth-bound and small helper kernels: in-block (physical-leg) gates, the
// product initial state, element-wise combinations and FP64 reductions.
#include "common.cuh"
#include "kernels.hpp"

namespace mpsgb {

unsigned long long g_launch_count = 0;
thread_local unsigned long long* t_launch_sink = nullptr;

namespace {
long long g_wait_limit = 4000000000LL;
}
long long wait_limit_cycles() { return __atomic_load_n(&g_wait_limit, __ATOMIC_RELAXED); }
void set_wait_limit_cycles(long long c) { __atomic_store_n(&g_wait_limit, c, __ATOMIC_RELAXED); }

namespace {
inline int nblocks(long long n, int t) { long long b = (n + t - 1) / t; return (int)(b > 65535LL * 16 ? 65535LL * 16 : b); }

// One thread per (a, b) fibre of the (l, d, r) block: the d values along the
// physical axis are read (stride r), multiplied by U and written back in place.
// Consecutive threads take consecutive b, so every access of a warp is coalesced.
template <typename R, int DMAX>
__global__ void apply_phys_kernel(Cx<R>* blk, int l, int d, int r, const Cx<R>* U) {
  __shared__ Cx<R> Us[DMAX * DMAX];
  for (int i = threadIdx.x; i < d * d; i += blockDim.x) Us[i] = U[i];
  __syncthreads();
  long long nf = (long long)l * r;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nf; f += (long long)gridDim.x * blockDim.x) {
    long long a = f / r, b = f - a * r;
    Cx<R>* base = blk + a * (long long)d * r + b;
    Cx<R> v[DMAX];
#pragma unroll
    for (int t = 0; t < DMAX; ++t) if (t < d) v[t] = base[(long long)t * r];
#pragma unroll
    for (int s = 0; s < DMAX; ++s) {
      if (s >= d) break;
      Cx<R> acc = cmake<R>(0, 0);
#pragma unroll
      for (int t = 0; t < DMAX; ++t) if (t < d) cfma(acc, Us[s * d + t], v[t]);
      base[(long long)s * r] = acc;
    }
  }
}

template <typename R>
__global__ void init_product_kernel(Cx<R>* blk, int k, double c, double s) {
  int d = 1 << k;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    double v = 1.0;
    for (int t = 0; t < k; ++t) v *= ((i >> (k - 1 - t)) & 1) ? s : c;  // first qubit = most significant bit
    blk[i] = cmake<R>((R)v, (R)0);
  }
}

template <typename R>
__global__ void scale_view_kernel(int M, int N, Cx<R> alpha, View<R> C, long long sC) {
  long long tot = (long long)M * N;
  Cx<R>* p = C.ptr + blockIdx.y * sC;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / N, j = e - i * N;
    long long o = C.row(i) + C.col(j);
    p[o] = alpha * p[o];
  }
}

template <typename R>
__global__ void axpby_kernel(int M, int N, Cx<R> a, View<R> X, Cx<R> b, View<R> Y, View<R> C) {
  long long tot = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / N, j = e - i * N;
    Cx<R> x = X.ptr[X.row(i) + X.col(j)];
    if (X.conj) x.y = -x.y;
    Cx<R> v = a * x;
    if (Y.ptr) {
      Cx<R> y = Y.ptr[Y.row(i) + Y.col(j)];
      if (Y.conj) y.y = -y.y;
      v = v + b * y;
    }
    C.ptr[C.row(i) + C.col(j)] = v;
  }
}

template <typename Rd, typename Rs>
__global__ void copy_view_kernel(int M, int N, View<Rs> src, View<Rd> dst) {
  long long tot = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / N, j = e - i * N;
    Cx<Rs> x = src.ptr[src.row(i) + src.col(j)];
    if (src.conj) x.y = -x.y;
    dst.ptr[dst.row(i) + dst.col(j)] = cmake<Rd>((Rd)x.x, (Rd)x.y);
  }
}

template <typename R>
__global__ void scale_cols_pow_kernel(int nrow, int ncol, Cx<R>* M, long long ld, const R* s, int p2) {
  long long tot = (long long)nrow * ncol;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / ncol, j = e - i * ncol;
    R v = s[j];
    R f = p2 > 0 ? sqrt(v) : R(1) / sqrt(v);
    M[i * ld + j] = f * M[i * ld + j];
  }
}

__device__ __forceinline__ int popc(int x) { return __popc(x); }

template <typename R>
__global__ void weighted_phys_kernel(int mode, int l, int d, int r, const Cx<R>* Y1, const Cx<R>* Y0, Cx<R>* Z,
                                     double coef) {
  long long tot = (long long)l * d * r;
  int k = 31 - __clz(d);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long a = e / ((long long)d * r);
    long long rem = e - a * (long long)d * r;
    int s = (int)(rem / r);
    long long b = rem - (long long)s * r;
    Cx<R> v = Y1 ? Y1[e] : cmake<R>(0, 0);
    if (mode == 3) {
      Cx<R> acc = cmake<R>(0, 0);
      for (int t = 0; t < k; ++t) acc = acc + Y0[(a * d + (s ^ (1 << t))) * (long long)r + b];
      v = v + (R)coef * acc;
    } else {
      R m = (R)(k - 2 * popc(s));  // sum of z over the block's qubits
      R w = mode == 1 ? m : m * m;
      v = v + (R)(coef * w) * Y0[e];
    }
    Z[e] = v;
  }
}

// Z = Y1 + coef * O(Y0) over a block-shaped tensor (l, d, r): mode 0, O = identity; mode 1,
// O = sum_t s_t X_t (bit flips of the physical index, s_t = -1 where bit t of negmask is set)
template <typename R>
__global__ void stag_x_kernel(int mode, int l, int d, int r, const Cx<R>* Y1, const Cx<R>* Y0, Cx<R>* Z, double coef,
                              int negmask) {
  long long tot = (long long)l * d * r;
  int k = 31 - __clz(d);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long a = e / ((long long)d * r);
    long long rem = e - a * (long long)d * r;
    int s = (int)(rem / r);
    long long b = rem - (long long)s * r;
    Cx<R> v = Y1 ? Y1[e] : cmake<R>(0, 0);
    Cx<R> acc = cmake<R>(0, 0);
    if (mode == 0) {
      acc = Y0[e];
    } else {
      for (int t = 0; t < k; ++t) {
        const Cx<R> y = Y0[(a * d + (s ^ (1 << t))) * (long long)r + b];
        acc = ((negmask >> t) & 1) ? acc - y : acc + y;
      }
    }
    Z[e] = v + (R)coef * acc;
  }
}

template <typename R>
__global__ void dot_fp64_kernel(long long n, const Cx<R>* X, const Cx<R>* Y, double* out) {
  double re = 0, im = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    Cx<R> x = X[e], y = Y[e];
    re += (double)x.x * y.x + (double)x.y * y.y;
    im += (double)x.x * y.y - (double)x.y * y.x;
  }
  for (int o = 16; o > 0; o >>= 1) { re += __shfl_xor_sync(0xffffffffu, re, o); im += __shfl_xor_sync(0xffffffffu, im, o); }
  __shared__ double sr[32], si[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sr[w] = re; si[w] = im; }
  __syncthreads();
  if (w == 0) {
    re = lane < (int)(blockDim.x >> 5) ? sr[lane] : 0; im = lane < (int)(blockDim.x >> 5) ? si[lane] : 0;
    for (int o = 16; o > 0; o >>= 1) { re += __shfl_xor_sync(0xffffffffu, re, o); im += __shfl_xor_sync(0xffffffffu, im, o); }
    if (lane == 0) { atomicAdd(out, re); atomicAdd(out + 1, im); }
  }
}

template <typename R>
__global__ void trace_fp64_kernel(int n, const Cx<R>* A, long long lda, double* out) {
  double re = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) re += (double)A[i * lda + i].x;
  for (int o = 16; o > 0; o >>= 1) re += __shfl_xor_sync(0xffffffffu, re, o);
  __shared__ double sr[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sr[w] = re;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sr[i];
    out[0] = t;
  }
}

template <typename R>
__global__ void set_identity_kernel(int n, Cx<R>* A, long long lda) {
  long long tot = (long long)n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / n, j = e - i * n;
    A[i * lda + j] = cmake<R>(i == j ? R(1) : R(0), R(0));
  }
}

template <typename R>
__global__ void set_zero_kernel(long long count, Cx<R>* A) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x)
    A[e] = cmake<R>(0, 0);
}

template <typename R>
__global__ void env_split_kernel(int r, const Cx<R>* Yp, const Cx<R>* Ym, double phi, Cx<R>* E) {
  long long tot = (long long)r * r;
  Cx<R> ep = cmake<R>((R)cos(2 * phi), (R)(-sin(2 * phi)));  // e^{-2 i phi}
  Cx<R> em = cmake<R>((R)cos(2 * phi), (R)(sin(2 * phi)));   // e^{+2 i phi}
  long long n2 = 2LL * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / r, j = e - i * r;
    Cx<R> yp = Yp[e], ym = Ym[e];
    Cx<R> d = yp + ym;
    Cx<R> o = ep * yp + em * ym;
    E[i * n2 + j] = d;
    E[(i + r) * n2 + j + r] = d;
    E[i * n2 + j + r] = o;
    // lower-left block is the Hermitian conjugate of the upper-right one
    E[(j + r) * n2 + i] = conj(o);
  }
}

template <typename R>
__global__ void env_assemble_kernel(int r, const Cx<R>* E00, const Cx<R>* E01, Cx<R>* E) {
  long long tot = (long long)r * r;
  long long n2 = 2LL * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / r, j = e - i * r;
    E[i * n2 + j] = E00[e];
    E[(i + r) * n2 + j + r] = E00[e];
    E[i * n2 + j + r] = E01[e];
    E[(j + r) * n2 + i] = conj(E01[e]);
  }
}

template <typename R>
__global__ void block_diag2_kernel(int r, const Cx<R>* P, const Cx<R>* Q, Cx<R>* G) {
  long long tot = (long long)r * r;
  long long n2 = 2LL * r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    long long i = e / r, j = e - i * r;
    G[i * n2 + j] = P[e];
    G[(i + r) * n2 + j + r] = Q[e];
    G[i * n2 + j + r] = cmake<R>(0, 0);
    G[(i + r) * n2 + j] = cmake<R>(0, 0);
  }
}
}  // namespace

template <typename R>
void apply_phys(cudaStream_t st, Cx<R>* blk, int l, int d, int r, const Cx<R>* U) {
  long long nf = (long long)l * r;
  int g = nblocks(nf, 256);
  kt_begin(KT_PHYS, st);
  if (d <= 4) apply_phys_kernel<R, 4><<<g, 256, 0, st>>>(blk, l, d, r, U);
  else if (d <= 8) apply_phys_kernel<R, 8><<<g, 256, 0, st>>>(blk, l, d, r, U);
  else if (d <= 16) apply_phys_kernel<R, 16><<<g, 256, 0, st>>>(blk, l, d, r, U);
  else apply_phys_kernel<R, 32><<<g, 256, 0, st>>>(blk, l, d, r, U);
  kt_end(KT_PHYS, st);
  kt_add_work(KT_PHYS, 2.0 * (double)l * d * r * sizeof(Cx<R>));
  count_launch();
}

template <typename R>
void init_product(cudaStream_t st, Cx<R>* blk, int k, double c, double s) {
  init_product_kernel<R><<<1, 64, 0, st>>>(blk, k, c, s);
  count_launch();
}

template <typename R>
void scale_view(cudaStream_t st, int M, int N, Cx<R> alpha, View<R> C, int batch, long long sC) {
  dim3 g(nblocks((long long)M * N, 256), batch);
  scale_view_kernel<R><<<g, 256, 0, st>>>(M, N, alpha, C, sC);
  count_launch();
}

template <typename R>
void axpby(cudaStream_t st, int M, int N, Cx<R> a, View<R> X, Cx<R> b, View<R> Y, View<R> C) {
  if (M <= 0 || N <= 0) return;
  axpby_kernel<R><<<nblocks((long long)M * N, 256), 256, 0, st>>>(M, N, a, X, b, Y, C);
  count_launch();
}

template <typename Rd, typename Rs>
void copy_view(cudaStream_t st, int M, int N, View<Rs> src, View<Rd> dst) {
  if (M <= 0 || N <= 0) return;
  copy_view_kernel<Rd, Rs><<<nblocks((long long)M * N, 256), 256, 0, st>>>(M, N, src, dst);
  count_launch();
}

template <typename R>
void scale_cols_pow(cudaStream_t st, int nrow, int ncol, Cx<R>* M, long long ld, const R* s, int p2) {
  if (nrow <= 0 || ncol <= 0) return;
  scale_cols_pow_kernel<R><<<nblocks((long long)nrow * ncol, 256), 256, 0, st>>>(nrow, ncol, M, ld, s, p2);
  count_launch();
}

template <typename R>
void stag_x(cudaStream_t st, int mode, int l, int d, int r, const Cx<R>* Y1, const Cx<R>* Y0, Cx<R>* Z, double coef,
            int negmask) {
  long long tot = (long long)l * d * r;
  stag_x_kernel<R><<<nblocks(tot, 256), 256, 0, st>>>(mode, l, d, r, Y1, Y0, Z, coef, negmask);
  count_launch();
}

template <typename R>
void weighted_phys(cudaStream_t st, int mode, int l, int d, int r, const Cx<R>* Y1, const Cx<R>* Y0, Cx<R>* Z,
                   double coef) {
  long long tot = (long long)l * d * r;
  weighted_phys_kernel<R><<<nblocks(tot, 256), 256, 0, st>>>(mode, l, d, r, Y1, Y0, Z, coef);
  count_launch();
}

template <typename R>
void dot_fp64(cudaStream_t st, long long n, const Cx<R>* X, const Cx<R>* Y, double* out) {
  cudaMemsetAsync(out, 0, 2 * sizeof(double), st);
  int g = nblocks(n, 256);
  if (g > 1024) g = 1024;
  dot_fp64_kernel<R><<<g, 256, 0, st>>>(n, X, Y, out);
  count_launch();
}

template <typename R>
void trace_fp64(cudaStream_t st, int n, const Cx<R>* A, long long lda, double* out) {
  trace_fp64_kernel<R><<<1, 256, 0, st>>>(n, A, lda, out);
  count_launch();
}

template <typename R>
void set_identity(cudaStream_t st, int n, Cx<R>* A, long long lda) {
  set_identity_kernel<R><<<nblocks((long long)n * n, 256), 256, 0, st>>>(n, A, lda);
  count_launch();
}

template <typename R>
void set_zero(cudaStream_t st, long long count, Cx<R>* A) {
  if (count <= 0) return;
  set_zero_kernel<R><<<nblocks(count, 256), 256, 0, st>>>(count, A);
  count_launch();
}

template <typename R>
void env_from_split_grams(cudaStream_t st, int r, const Cx<R>* Yp, const Cx<R>* Ym, double phi, Cx<R>* E) {
  env_split_kernel<R><<<nblocks((long long)r * r, 256), 256, 0, st>>>(r, Yp, Ym, phi, E);
  count_launch();
}

template <typename R>
void env_assemble(cudaStream_t st, int r, const Cx<R>* E00, const Cx<R>* E01, Cx<R>* E) {
  env_assemble_kernel<R><<<nblocks((long long)r * r, 256), 256, 0, st>>>(r, E00, E01, E);
  count_launch();
}

template <typename R>
void block_diag2(cudaStream_t st, int r, const Cx<R>* P, const Cx<R>* Q, Cx<R>* G) {
  block_diag2_kernel<R><<<nblocks((long long)r * r, 256), 256, 0, st>>>(r, P, Q, G);
  count_launch();
}

#define INST(R)                                                                                              \
  template void apply_phys<R>(cudaStream_t, Cx<R>*, int, int, int, const Cx<R>*);                            \
  template void init_product<R>(cudaStream_t, Cx<R>*, int, double, double);                                  \
  template void scale_view<R>(cudaStream_t, int, int, Cx<R>, View<R>, int, long long);                      \
  template void axpby<R>(cudaStream_t, int, int, Cx<R>, View<R>, Cx<R>, View<R>, View<R>);                   \
  template void scale_cols_pow<R>(cudaStream_t, int, int, Cx<R>*, long long, const R*, int);                 \
  template void weighted_phys<R>(cudaStream_t, int, int, int, int, const Cx<R>*, const Cx<R>*, Cx<R>*, double); \
  template void stag_x<R>(cudaStream_t, int, int, int, int, const Cx<R>*, const Cx<R>*, Cx<R>*, double, int);    \
  template void dot_fp64<R>(cudaStream_t, long long, const Cx<R>*, const Cx<R>*, double*);                   \
  template void trace_fp64<R>(cudaStream_t, int, const Cx<R>*, long long, double*);                          \
  template void set_identity<R>(cudaStream_t, int, Cx<R>*, long long);                                       \
  template void set_zero<R>(cudaStream_t, long long, Cx<R>*);                                                \
  template void env_from_split_grams<R>(cudaStream_t, int, const Cx<R>*, const Cx<R>*, double, Cx<R>*);      \
  template void env_assemble<R>(cudaStream_t, int, const Cx<R>*, const Cx<R>*, Cx<R>*);                      \
  template void block_diag2<R>(cudaStream_t, int, const Cx<R>*, const Cx<R>*, Cx<R>*);
INST(double)
INST(float)
template void copy_view<double, double>(cudaStream_t, int, int, View<double>, View<double>);
template void copy_view<float, float>(cudaStream_t, int, int, View<float>, View<float>);
template void copy_view<double, float>(cudaStream_t, int, int, View<float>, View<double>);
template void copy_view<float, double>(cudaStream_t, int, int, View<double>, View<float>);

}  // namespace mpsgb
