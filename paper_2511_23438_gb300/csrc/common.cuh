// Shared device/host definitions for the mpsgb CUDA library.
// Complex numbers are plain {re, im} structs so that the same templates serve
// complex128 (FP64 form) and complex64 (split / FP32 forms).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

namespace mpsgb {

template <typename R> struct alignas(2 * sizeof(R)) Cx { R x, y; };
using z128 = Cx<double>;
using c64 = Cx<float>;

template <typename R> __host__ __device__ __forceinline__ Cx<R> cmake(R a, R b) { Cx<R> c; c.x = a; c.y = b; return c; }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return cmake(a.x + b.x, a.y + b.y); }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return cmake(a.x - b.x, a.y - b.y); }
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return cmake(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R> __host__ __device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return cmake(s * a.x, s * a.y); }
template <typename R> __host__ __device__ __forceinline__ Cx<R> conj(Cx<R> a) { return cmake(a.x, -a.y); }
template <typename R> __host__ __device__ __forceinline__ R abs2(Cx<R> a) { return a.x * a.x + a.y * a.y; }
// acc += a * b
template <typename R> __host__ __device__ __forceinline__ void cfma(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}

// Offset of index x along one matrix dimension of a two-level strided view:
// off(x) = (x / inner) * outer + (x % inner) * stride.  inner == 0 means a plain
// stride (no split).  This single form covers row-major matrices, their
// transposes, and the "qubit-split" sub-matrices (rows or columns whose physical
// index has one bit fixed) and interleaved MPO column blocks used by the engine.
struct Off {
  long long inner, stride, outer;
  __host__ __device__ __forceinline__ long long operator()(long long x) const {
    if (inner == 0) return x * stride;
    long long q = x / inner;
    return q * outer + (x - q * inner) * stride;
  }
};
inline Off plain(long long stride) { Off o; o.inner = 0; o.stride = stride; o.outer = 0; return o; }
inline Off split(long long inner, long long stride, long long outer) { Off o; o.inner = inner; o.stride = stride; o.outer = outer; return o; }

// A matrix operand: element (i, j) lives at ptr + row(i) + col(j); conj applies on load.
template <typename R> struct View {
  Cx<R>* ptr;
  Off row, col;
  bool conj;
};
template <typename R> inline View<R> rowmajor(Cx<R>* p, long long ld) { View<R> v; v.ptr = p; v.row = plain(ld); v.col = plain(1); v.conj = false; return v; }
// (i, j) -> element (j, i) of a row-major matrix, optionally conjugated (op = T or H)
template <typename R> inline View<R> transposed(Cx<R>* p, long long ld, bool cj) { View<R> v; v.ptr = p; v.row = plain(1); v.col = plain(ld); v.conj = cj; return v; }

// Launch accounting: every kernel launch made by the library bumps this counter
// so callers can report how many of our kernels ran in a timed region.
extern unsigned long long g_launch_count;
// while this thread captures a CUDA graph, launches are counted here instead (they run, and are
// counted, each time the graph is launched)
extern thread_local unsigned long long* t_launch_sink;
inline void count_launch(unsigned long long n = 1) {
  if (t_launch_sink) *t_launch_sink += n;
  else __atomic_add_fetch(&g_launch_count, n, __ATOMIC_RELAXED);
}

// Cycle limit of the library's bounded device waits on other CTAs (grid barriers).  The default
// (4e9 cycles, about 2 s at 2 GHz) is far above any legitimate wait; a test can lower it through
// mpsgb_set_wait_limit to make a wait run out and exercise the MPSGB_ETIMEDOUT path.
long long wait_limit_cycles();
void set_wait_limit_cycles(long long cycles);

// Optional per-launch-site timing with CUDA events (off by default): when enabled,
// kt_begin / kt_end bracket the launches of one site on their stream and the
// accumulated device time is read back by mpsgb_kernel_times().
enum KtSite { KT_GEMM = 0, KT_EIG_PAIR, KT_EIG_UPDATE, KT_EIG_SMALL, KT_PHYS, KT_TC_GEMM, KT_HETRD, KT_TRIVEC,
              KT_SVD, KT_GEMM_EIG, KT_GEMM_CHOL, KT_NSITES };
// timing site that CUDA-core GEMMs issued on this thread are charged to (KT_GEMM unless a caller
// sets another for its scope with GemmSite)
extern thread_local int g_gemm_site;
struct GemmSite {
  int prev;
  explicit GemmSite(int site) : prev(g_gemm_site) { g_gemm_site = site; }
  ~GemmSite() { g_gemm_site = prev; }
};
extern bool g_kt_enabled;
void kt_begin_impl(int site, cudaStream_t st);
void kt_end_impl(int site, cudaStream_t st);
inline void kt_begin(int site, cudaStream_t st) { if (g_kt_enabled) kt_begin_impl(site, st); }
inline void kt_end(int site, cudaStream_t st) { if (g_kt_enabled) kt_end_impl(site, st); }
// useful work of a bracketed launch: real flops for arithmetic sites, bytes for data movement
// (the in-block gate and the Householder reduction, whose trailing-matrix passes are its cost)
void kt_add_work(int site, double work);

}  // namespace mpsgb
