// Complex GEMM on the 5th-generation tensor cores (tcgen05, sm_103a), fed by TMA.
//
//   C(i, j) = alpha * sum_k A(i, k) B(k, j) + beta * C(i, j)      (complex64 in and out)
//
// Split precision: every real component x is written as x_hi + x_lo with
// x_hi = bf16(x), x_lo = bf16(x - x_hi) (16 significant bits; kind::f16), or with
// x_hi = tf32(x), x_lo = tf32(x - x_hi) (22 significant bits; kind::tf32, half the
// BF16 tensor rate), and a real product x * y is formed from the three products
// hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory.  The complex product uses four real accumulators
// P = Ar Br, T = Ai Bi, U = Ar Bi, W = Ai Br, so Re = P - T and Im = U + W.
//
// Data path: a conversion kernel writes the operands as planes (BF16 or TF32-in-FP32)
// [re_hi, im_hi, re_lo, im_lo] x rows x Kp (K contiguous, Kp a multiple of the K tile,
// zero padded); per K tile of 128 bytes a row (64 BF16 / 32 TF32 elements) the TMA unit
// loads a 4-plane box of A (128 rows) and of B (BN rows) into 128-byte-swizzled shared
// memory; one thread issues the 48 tcgen05.mma (M = 128, N = BN, 32 bytes of K each:
// K = 16 BF16 / 8 TF32) of the tile; tcgen05.commit frees the stage;
// four epilogue warps read the accumulators with tcgen05.ld and write C.
// Warp roles: warp 0 TMA producer, warp 1 TMEM owner + MMA issuer, warps 2-5 epilogue.
// Every mbarrier wait is bounded: on timeout the kernel records an error word and
// stops issuing work (it never spins without a limit).
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "kernels.hpp"

namespace mpsgb {

namespace {
constexpr int TBM = 128, TSTAGES = 2, TBN = 64;
constexpr int ROWB = 128;                          // bytes of one tile row (the swizzle span)
constexpr int A_STAGE_BYTES = 4 * TBM * ROWB;      // 64 KB
constexpr int B_STAGE_BYTES = 4 * TBN * ROWB;      // 32 KB
template <bool TF>
struct Split {                                     // plane element: BF16 (kind::f16) or TF32 in FP32 (kind::tf32)
  static constexpr int ES = TF ? 4 : 2;            // bytes per element
  static constexpr int BK = ROWB / ES;             // K elements per tile
};
constexpr int STAGE_BYTES = A_STAGE_BYTES + B_STAGE_BYTES;
constexpr int TMEM_COLS = 4 * TBN;                 // P, T, U, W accumulators
constexpr long long WAIT_LIMIT = 1LL << 26;        // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; returns false (and records the error) if the phase never completed
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code) {
  for (long long i = 0; i < WAIT_LIMIT; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 128) __nanosleep(32);
  }
  atomicExch(err, code);
  return false;
}

__device__ __forceinline__ void tma_load_3d(const CUtensorMap* tm, uint64_t* bar, void* dst, int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(tm), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

// Instruction descriptor: FP32 accumulate (D format 1), A and B format BF16 (1, kind::f16) or
// TF32 (2, kind::tf32), both K-major, N / 8 and M / 16.
__host__ __device__ constexpr uint32_t idesc_split(int M, int N, bool tf32) {
  return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <bool TF>
__device__ __forceinline__ void mma_split(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (TF) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
  }
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

#define TMEM_LD16(taddr, r)                                                                                        \
  asm volatile(                                                                                                    \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"     \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), \
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])                  \
      : "r"(taddr))

template <bool TF>
__global__ void __launch_bounds__(192, 1)
    tc_cgemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                    int nkb, c64 alpha, c64 beta, View<float> C, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[TSTAGES];
  __shared__ __align__(8) uint64_t empty_bar[TSTAGES];
  __shared__ __align__(8) uint64_t accum_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    mbar_init(&accum_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % TSTAGES;
        if (kb >= TSTAGES && !mbar_wait(&empty_bar[s], ((kb / TSTAGES) - 1) & 1, err, 1)) { abort_flag = 1; break; }
        if (abort_flag) break;
        unsigned char* a_dst = smem + s * STAGE_BYTES;
        unsigned char* b_dst = a_dst + A_STAGE_BYTES;
        mbar_expect_tx(&full_bar[s], STAGE_BYTES);
        tma_load_3d(&tmA, &full_bar[s], a_dst, kb * Split<TF>::BK, m0, 0);
        tma_load_3d(&tmB, &full_bar[s], b_dst, kb * Split<TF>::BK, n0, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = idesc_split(TBM, TBN, TF);
      // (accumulator, A plane, B plane): P = Ar Br, T = Ai Bi, U = Ar Bi, W = Ai Br, 3 split terms each
      const int acc_of[12] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3};
      const int ap[12] = {0, 0, 2, 1, 1, 3, 0, 0, 2, 1, 1, 3};
      const int bp[12] = {0, 2, 0, 1, 3, 1, 1, 3, 1, 0, 2, 0};
      bool ok = true;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb % TSTAGES;
        if (!mbar_wait(&full_bar[s], (kb / TSTAGES) & 1, err, 2)) { abort_flag = 1; ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_base = smem_u32(smem + s * STAGE_BYTES);
        const uint32_t b_base = a_base + A_STAGE_BYTES;
        for (int kk = 0; kk < ROWB / 32; ++kk) {  // 32 bytes of K per MMA
          for (int t = 0; t < 12; ++t) {
            uint64_t ad = sdesc(a_base + ap[t] * (TBM * ROWB) + kk * 32);
            uint64_t bd = sdesc(b_base + bp[t] * (TBN * ROWB) + kk * 32);
            uint32_t accumulate = (kb > 0 || kk > 0 || (t % 3) != 0) ? 1u : 0u;
            mma_split<TF>(tmem + acc_of[t] * TBN, ad, bd, idesc, accumulate);
          }
        }
        mma_commit(&empty_bar[s]);
      }
      mma_commit(&accum_bar);
    }
  } else {  // epilogue warps 2..5: TMEM lane quarter = warp % 4
    const int q = warp & 3;
    const int row = m0 + q * 32 + lane;
    bool ok = mbar_wait(&accum_bar, 0, err, 3);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && !abort_flag) {
      const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
      const bool use_beta = (beta.x != 0.f || beta.y != 0.f);
      long long ro = row < M ? C.row(row) : 0;
      for (int c0 = 0; c0 < TBN; c0 += 16) {
        uint32_t P[16], T[16], U[16], W[16];
        TMEM_LD16(tq + 0 * TBN + c0, P);
        TMEM_LD16(tq + 1 * TBN + c0, T);
        TMEM_LD16(tq + 2 * TBN + c0, U);
        TMEM_LD16(tq + 3 * TBN + c0, W);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            int col = n0 + c0 + j;
            if (col >= N) break;
            c64 v = cmake<float>(__uint_as_float(P[j]) - __uint_as_float(T[j]), __uint_as_float(U[j]) + __uint_as_float(W[j]));
            v = alpha * v;
            long long o = ro + C.col(col);
            if (use_beta) v = v + beta * C.ptr[o];
            C.ptr[o] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

__device__ __forceinline__ float to_tf32(float x) {  // round to nearest, ties away: 10 explicit mantissa bits
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// op(X) (rows x K) -> planes [re_hi, im_hi, re_lo, im_lo][rows][Kp], zero padded in k: BF16
// (hi = bf16(x), lo = bf16(x - hi)) or TF32 stored as FP32 (hi = tf32(x), lo = tf32(x - hi))
template <bool TF>
__global__ void __launch_bounds__(256) split_planes_kernel(int rows, int K, int Kp, View<float> src, bool kfast,
                                                           void* out) {
  __shared__ c64 tile[32][65];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 64;
  for (int e = threadIdx.x; e < 32 * 64; e += 256) {
    int r, k;
    if (kfast) { r = e / 64; k = e % 64; } else { r = e % 32; k = e / 32; }
    c64 v = cmake<float>(0.f, 0.f);
    if (r0 + r < rows && k0 + k < K) {
      v = src.ptr[src.row(r0 + r) + src.col(k0 + k)];
      if (src.conj) v.y = -v.y;
    }
    tile[r][k] = v;
  }
  __syncthreads();
  const size_t plane = (size_t)rows * Kp;
  for (int e = threadIdx.x; e < 32 * 64; e += 256) {
    int r = e / 64, k = e % 64;
    if (r0 + r >= rows || k0 + k >= Kp) continue;
    c64 v = tile[r][k];
    size_t o = (size_t)(r0 + r) * Kp + (k0 + k);
    if constexpr (TF) {
      float* planes = static_cast<float*>(out);
      const float rh = to_tf32(v.x), ih = to_tf32(v.y);
      planes[o] = rh;
      planes[plane + o] = ih;
      planes[2 * plane + o] = to_tf32(v.x - rh);
      planes[3 * plane + o] = to_tf32(v.y - ih);
    } else {
      __nv_bfloat16* planes = static_cast<__nv_bfloat16*>(out);
      __nv_bfloat16 rh = __float2bfloat16_rn(v.x), ih = __float2bfloat16_rn(v.y);
      __nv_bfloat16 rl = __float2bfloat16_rn(v.x - __bfloat162float(rh));
      __nv_bfloat16 il = __float2bfloat16_rn(v.y - __bfloat162float(ih));
      planes[o] = rh;
      planes[plane + o] = ih;
      planes[2 * plane + o] = rl;
      planes[3 * plane + o] = il;
    }
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
std::once_flag g_encode_once;

EncodeTiledFn encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  });
  return g_encode;
}

bool make_map(CUtensorMap* tm, void* base, int rows, int Kp, int box_rows, bool tf32) {
  EncodeTiledFn enc = encoder();
  if (!enc) return false;
  const cuuint64_t esz = tf32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, 4};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * esz, (cuuint64_t)rows * Kp * esz};
  cuuint32_t box[3] = {(cuuint32_t)(ROWB / esz), (cuuint32_t)box_rows, 4};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(tm, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box,
             es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

bool is_kfast(const View<float>& v) { return v.col.inner == 0 && v.col.stride == 1; }
}  // namespace

size_t tc_gemm_workspace_bytes(long long M, long long N, long long K, bool tf32) {
  const long long bk = tf32 ? Split<true>::BK : Split<false>::BK;
  const long long Kp = (K + 63) / 64 * 64;  // a multiple of both K tiles (the split kernel's 64-wide k blocks)
  (void)bk;
  return (size_t)(4 * (tf32 ? 4 : 2)) * (size_t)(M + N) * Kp + 2048;
}

int tc_gemm(cudaStream_t st, int M, int N, int K, c64 alpha, View<float> A, View<float> B, c64 beta, View<float> C,
            void* ws, size_t ws_bytes, int* d_err, bool tf32) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  const int Kp = (K + 63) / 64 * 64;
  if (tc_gemm_workspace_bytes(M, N, K, tf32) > ws_bytes) return -1;
  const size_t esz = tf32 ? 4 : 2;
  char* pa = reinterpret_cast<char*>(((uintptr_t)ws + 255) & ~uintptr_t(255));
  char* pb = reinterpret_cast<char*>((((uintptr_t)(pa + esz * 4 * (size_t)M * Kp)) + 255) & ~uintptr_t(255));
  // op(A) is M x K; op(B)^T is N x K with element (j, k) = op(B)(k, j)
  View<float> Bt;
  Bt.ptr = B.ptr; Bt.row = B.col; Bt.col = B.row; Bt.conj = B.conj;
  if (tf32) {
    split_planes_kernel<true><<<dim3(Kp / 64, (M + 31) / 32), 256, 0, st>>>(M, K, Kp, A, is_kfast(A), pa);
    split_planes_kernel<true><<<dim3(Kp / 64, (N + 31) / 32), 256, 0, st>>>(N, K, Kp, Bt, is_kfast(Bt), pb);
  } else {
    split_planes_kernel<false><<<dim3(Kp / 64, (M + 31) / 32), 256, 0, st>>>(M, K, Kp, A, is_kfast(A), pa);
    split_planes_kernel<false><<<dim3(Kp / 64, (N + 31) / 32), 256, 0, st>>>(N, K, Kp, Bt, is_kfast(Bt), pb);
  }
  count_launch(2);
  CUtensorMap ta, tb;
  if (!make_map(&ta, pa, M, Kp, TBM, tf32) || !make_map(&tb, pb, N, Kp, TBN, tf32)) return -2;
  const int smem = TSTAGES * STAGE_BYTES + 1024;
  static std::once_flag attr_once;  // several host threads (one per handle) may reach this at once
  std::call_once(attr_once, [smem] {
    cudaFuncSetAttribute(tc_cgemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(tc_cgemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  });
  dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM);
  kt_begin(KT_TC_GEMM, st);
  if (tf32)
    tc_cgemm_kernel<true><<<grid, 192, smem, st>>>(ta, tb, M, N, Kp / Split<true>::BK, alpha, beta, C, d_err);
  else
    tc_cgemm_kernel<false><<<grid, 192, smem, st>>>(ta, tb, M, N, Kp / Split<false>::BK, alpha, beta, C, d_err);
  kt_end(KT_TC_GEMM, st);
  kt_add_work(KT_TC_GEMM, 8.0 * M * N * (double)K);
  count_launch();
  return 0;
}

}  // namespace mpsgb

namespace mpsgb {
namespace {
__global__ void fill_random_kernel(long long n, c64* x, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long h = (unsigned long long)i * 0x9E3779B97F4A7C15ULL + seed;
    h ^= h >> 33; h *= 0xff51afd7ed558ccdULL; h ^= h >> 33; h *= 0xc4ceb9fe1a85ec53ULL; h ^= h >> 33;
    float a = (float)((h & 0xFFFFFF) / 16777216.0) - 0.5f, b = (float)(((h >> 24) & 0xFFFFFF) / 16777216.0) - 0.5f;
    x[i] = cmake<float>(a, b);
  }
}
__global__ void max_abs_diff_kernel(long long n, const c64* x, const c64* y, float* out) {
  float md = 0.f, mr = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    c64 d = x[i] - y[i];
    md = fmaxf(md, sqrtf(abs2(d)));
    mr = fmaxf(mr, sqrtf(abs2(y[i])));
  }
  atomicMax(reinterpret_cast<int*>(out), __float_as_int(md));
  atomicMax(reinterpret_cast<int*>(out + 1), __float_as_int(mr));
}
}  // namespace

// Tensor-core GEMM against the CUDA-core FP32 GEMM on seeded device data.
// mode bit 0: op(A) = A^H (A stored K x M); bit 1: op(B) = B^T (B stored N x K).
int tc_selftest(int M, int N, int K, int mode, unsigned long long seed, double* rel_err) {
  cudaStream_t st;
  if (cudaStreamCreate(&st) != cudaSuccess) return -4;
  c64 *A, *B, *C1, *C2;
  float* red;
  int* derr;
  size_t wsb = tc_gemm_workspace_bytes(M, N, K, (mode & 4) != 0);
  void* ws;
  cudaMalloc(&A, sizeof(c64) * (size_t)M * K);
  cudaMalloc(&B, sizeof(c64) * (size_t)K * N);
  cudaMalloc(&C1, sizeof(c64) * (size_t)M * N);
  cudaMalloc(&C2, sizeof(c64) * (size_t)M * N);
  cudaMalloc(&red, 2 * sizeof(float));
  cudaMalloc(&derr, sizeof(int));
  cudaMalloc(&ws, wsb);
  cudaMemsetAsync(red, 0, 2 * sizeof(float), st);
  cudaMemsetAsync(derr, 0, sizeof(int), st);
  fill_random_kernel<<<512, 256, 0, st>>>((long long)M * K, A, seed);
  fill_random_kernel<<<512, 256, 0, st>>>((long long)K * N, B, seed * 7 + 1);
  View<float> va = (mode & 1) ? transposed<float>(A, M, true) : rowmajor<float>(A, K);
  View<float> vb = (mode & 2) ? transposed<float>(B, K, false) : rowmajor<float>(B, N);
  c64 one = cmake<float>(1, 0), zero = cmake<float>(0, 0);
  int s = tc_gemm(st, M, N, K, one, va, vb, zero, rowmajor<float>(C1, N), ws, wsb, derr, (mode & 4) != 0);
  gemm<float>(st, M, N, K, one, va, vb, zero, rowmajor<float>(C2, N));
  max_abs_diff_kernel<<<256, 256, 0, st>>>((long long)M * N, C1, C2, red);
  float h[2] = {0, 0};
  int he = 0;
  cudaMemcpyAsync(h, red, 2 * sizeof(float), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&he, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(A); cudaFree(B); cudaFree(C1); cudaFree(C2); cudaFree(red); cudaFree(derr); cudaFree(ws);
  cudaStreamDestroy(st);
  if (e != cudaSuccess) return -4;
  if (s != 0) return -1;
  if (he != 0) return -3;
  *rel_err = h[1] > 0 ? (double)h[0] / h[1] : (double)h[0];
  return 0;
}

}  // namespace mpsgb
