// Per-launch-site device timing with CUDA events (measurement support for the
// benchmark's roofline figures).  Disabled by default; when enabled every
// bracketed launch records an event pair on its own stream; pairs are resolved
// (event-synchronised) only when the totals are read or the pool grows large.
#include <mutex>
#include <vector>

#include "../../include/mpsgb.h"
#include "common.cuh"

namespace mpsgb {

bool g_kt_enabled = false;

namespace {
struct Pair { cudaEvent_t a, b; int site; };
std::mutex g_mu;
std::vector<cudaEvent_t> g_free;
std::vector<Pair> g_pending;
double g_ms[KT_NSITES] = {0};
long long g_n[KT_NSITES] = {0};
double g_work[KT_NSITES] = {0};
thread_local cudaEvent_t t_open[KT_NSITES] = {nullptr};

cudaEvent_t take_event() {
  if (!g_free.empty()) { cudaEvent_t e = g_free.back(); g_free.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void resolve_locked() {
  for (auto& p : g_pending) {
    float ms = 0;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_ms[p.site] += ms;
      g_n[p.site] += 1;
    }
    g_free.push_back(p.a);
    g_free.push_back(p.b);
  }
  g_pending.clear();
}
}  // namespace

void kt_begin_impl(int site, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t e = take_event();
  cudaEventRecord(e, st);
  t_open[site] = e;
}

void kt_end_impl(int site, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!t_open[site]) return;
  cudaEvent_t e = take_event();
  cudaEventRecord(e, st);
  g_pending.push_back({t_open[site], e, site});
  t_open[site] = nullptr;
  if (g_pending.size() > 8192) resolve_locked();
}

void kt_add_work(int site, double work) {
  if (!g_kt_enabled) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_work[site] += work;
}

}  // namespace mpsgb

extern "C" {

int mpsgb_kernel_timing(int enable) {
  std::lock_guard<std::mutex> lk(mpsgb::g_mu);
  mpsgb::resolve_locked();
  for (int i = 0; i < mpsgb::KT_NSITES; ++i) { mpsgb::g_ms[i] = 0; mpsgb::g_n[i] = 0; mpsgb::g_work[i] = 0; }
  mpsgb::g_kt_enabled = enable != 0;
  return MPSGB_OK;
}

int mpsgb_kernel_times(int site, double* ms, long long* launches, double* work) {
  if (site < 0 || site >= mpsgb::KT_NSITES || !ms || !launches || !work) return MPSGB_EINVAL;
  std::lock_guard<std::mutex> lk(mpsgb::g_mu);
  mpsgb::resolve_locked();
  *ms = mpsgb::g_ms[site];
  *launches = mpsgb::g_n[site];
  *work = mpsgb::g_work[site];
  return MPSGB_OK;
}

const char* mpsgb_kernel_site_name(int site) {
  static const char* names[] = {"cgemm (CUDA-core complex GEMM: truncation core, contractions)", "jacobi pair solve", "jacobi rotation update",
                                "jacobi small (n<=32)", "in-block gate (apply_phys)", "tcgen05 split GEMM",
                                "Householder tridiagonal reduction (hetrd)",
                                "tridiagonal eigenvectors (bisection, inverse iteration, cluster GS)",
                                "one-sided Jacobi SVD (exact truncation route)",
                                "cgemm inside the eigensolver (orthonormalisation, back-transformation)",
                                "cgemm of the Cholesky factorisation and solves"};
  if (site < 0 || site >= mpsgb::KT_NSITES) return "";
  return names[site];
}

}  // extern "C"
