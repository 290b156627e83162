// C ABI of libmpsgb (declared in include/mpsgb.h): argument checks, handle
// ownership, exception-to-status conversion and the host-only helpers.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/mpsgb.h"
#include "engine.hpp"
#include "kernels.hpp"

using mpsgb::Engine;
using mpsgb::Fail;

struct mpsgb_mps {
  Engine* e = nullptr;
};

namespace {
thread_local std::string g_err;

int fail(int status, const std::string& msg) {
  g_err = msg;
  return status;
}

template <typename F>
int guarded(F&& f) {
  try {
    g_err.clear();
    return f();
  } catch (const Fail& x) {
    return fail(x.status, x.msg);
  } catch (const std::bad_alloc&) {
    return fail(MPSGB_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(MPSGB_EDEVICE, "unexpected internal error");
  }
}

int check_config(const mpsgb_config* c) {
  if (!c) return fail(MPSGB_EINVAL, "null config");
  if (c->prec < MPSGB_FP64 || c->prec > MPSGB_FP32) return fail(MPSGB_EINVAL, "unknown precision");
  if (c->route != MPSGB_ROUTE_MPO && c->route != MPSGB_ROUTE_SWAP) return fail(MPSGB_EINVAL, "unknown route");
  if (!std::isfinite(c->theta)) return fail(MPSGB_EINVAL, "theta is not finite");
  if (c->chi_max < 1 || c->chi_max > 8192) return fail(MPSGB_EINVAL, "chi_max must be in 1..8192");
  mpsgb::Layout L;
  std::string err;
  if (!mpsgb::make_layout(*c, L, err)) return fail(MPSGB_EINVAL, err);
  if (c->model != MPSGB_MODEL_TFIM && c->model != MPSGB_MODEL_XY) return fail(MPSGB_EINVAL, "unknown model");
  if (c->model == MPSGB_MODEL_XY) {
    if (c->lattice != MPSGB_LATTICE_2D_SITES) return fail(MPSGB_EINVAL, "the XY model runs on LATTICE_2D_SITES");
    if (c->route != MPSGB_ROUTE_SWAP) return fail(MPSGB_EINVAL, "the XY model's gates are routed by SWAP");
    if (c->trotter_order != 2) return fail(MPSGB_EINVAL, "the XY model's Trotter step is second order");
  }
  return MPSGB_OK;
}

int create_impl(const mpsgb_config* cfg, const mpsgb_allocator* alloc, void* stream, mpsgb_handle* out) {
  if (!out) return fail(MPSGB_EINVAL, "null output handle");
  *out = nullptr;
  int s = check_config(cfg);
  if (s) return s;
  std::string err;
  int status = 0;
  Engine* e = mpsgb::make_engine(*cfg, alloc, (cudaStream_t)stream, err, status);
  if (!e) return fail(status ? status : MPSGB_EDEVICE, err);
  auto* h = new mpsgb_mps();
  h->e = e;
  *out = h;
  return MPSGB_OK;
}
int schedule_info_of(const mpsgb::Layout& L, long long out[6]) {
  long long nintra = 0, ntr = 0;
  int dmax = 1;
  for (auto& v : L.intra) nintra += (long long)v.size();
  for (auto& g : L.inter) ntr += g.q - g.p;
  for (int k : L.k) dmax = std::max(dmax, 1 << k);
  out[0] = L.N; out[1] = nintra + (long long)L.inter.size(); out[2] = nintra;
  out[3] = (long long)L.inter.size(); out[4] = ntr; out[5] = dmax;
  return MPSGB_OK;
}

int schedule_gates_of(const mpsgb::Layout& L, int* out, int cap, int* n) {
  *n = (int)L.inter.size();
  for (int i = 0; i < cap && i < (int)L.inter.size(); ++i) {
    const auto& g = L.inter[i];
    int v[6] = {g.p, g.q, g.qi, g.qj, g.ti, g.tj};
    for (int j = 0; j < 6; ++j) out[6 * i + j] = v[j];
  }
  return MPSGB_OK;
}
}  // namespace

extern "C" {

int mpsgb_create(const mpsgb_config* cfg, const mpsgb_allocator* alloc, void* cuda_stream, mpsgb_handle* out) {
  return guarded([&]() -> int { return create_impl(cfg, alloc, cuda_stream, out); });
}

int mpsgb_apply_layer(mpsgb_handle h, mpsgb_layer layer, double angle) {
  if (!h || !h->e) return fail(MPSGB_EINVAL, "null handle");
  if (!std::isfinite(angle)) return fail(MPSGB_EINVAL, "angle is not finite");
  if (layer != MPSGB_LAYER_X && layer != MPSGB_LAYER_ZZ && layer != MPSGB_LAYER_ZSTAG)
    return fail(MPSGB_EINVAL, "unknown layer");
  return guarded([&]() -> int {
    if (layer == MPSGB_LAYER_ZSTAG) return h->e->apply_zstag(angle);
    return layer == MPSGB_LAYER_X ? h->e->apply_x(angle) : h->e->apply_zz(angle);
  });
}

int mpsgb_apply_gates(mpsgb_handle h, int first, int count, double phi) {
  if (!h || !h->e) return fail(MPSGB_EINVAL, "null handle");
  if (!std::isfinite(phi)) return fail(MPSGB_EINVAL, "angle is not finite");
  return guarded([&]() -> int { return h->e->apply_gates(first, count, phi); });
}

int mpsgb_step(mpsgb_handle h, double J, double hx, double dt, int trotter_order, int nsteps) {
  if (!h || !h->e) return fail(MPSGB_EINVAL, "null handle");
  if (!std::isfinite(J) || !std::isfinite(hx) || !std::isfinite(dt)) return fail(MPSGB_EINVAL, "parameter is not finite");
  if (trotter_order != 1 && trotter_order != 2) return fail(MPSGB_EINVAL, "trotter_order must be 1 or 2");
  if (nsteps < 0) return fail(MPSGB_EINVAL, "nsteps must be >= 0");
  return guarded([&]() -> int { return h->e->step(J, hx, dt, trotter_order, nsteps); });
}

int mpsgb_truncate(mpsgb_handle h, int chi) {
  if (!h || !h->e) return fail(MPSGB_EINVAL, "null handle");
  return guarded([&]() -> int { return h->e->truncate(chi); });
}

int mpsgb_observables(mpsgb_handle h, double out[4]) {
  if (!h || !h->e || !out) return fail(MPSGB_EINVAL, "null argument");
  return guarded([&]() -> int { return h->e->observables(out); });
}

int mpsgb_expect(mpsgb_handle h, mpsgb_obs obs, double* out) {
  if (!h || !h->e || !out) return fail(MPSGB_EINVAL, "null argument");
  if (obs < MPSGB_Z_TOT || obs > MPSGB_X_STAG2) return fail(MPSGB_EINVAL, "unknown observable");
  if (obs == MPSGB_X_STAG2) return guarded([&]() -> int { return h->e->x_stag2(out); });
  double v[4];
  int s = mpsgb_observables(h, v);
  if (s) return s;
  *out = v[(int)obs];
  return MPSGB_OK;
}

int mpsgb_fidelity(mpsgb_handle h, double* F) {
  if (!h || !h->e || !F) return fail(MPSGB_EINVAL, "null argument");
  *F = h->e->F;
  return MPSGB_OK;
}

int mpsgb_singular_values(mpsgb_handle h, int bond, double* out, int cap, int* n) {
  if (!h || !h->e || !n || (cap > 0 && !out)) return fail(MPSGB_EINVAL, "null argument");
  return guarded([&]() -> int {
    std::vector<double> s;
    int st = h->e->singular_values(bond, s);
    if (st) return st;
    *n = (int)s.size();
    for (int i = 0; i < cap && i < (int)s.size(); ++i) out[i] = s[i];
    return MPSGB_OK;
  });
}

int mpsgb_bond_dims(mpsgb_handle h, int* out, int cap, int* n) {
  if (!h || !h->e || !n || (cap > 0 && !out)) return fail(MPSGB_EINVAL, "null argument");
  const auto& d = h->e->dims;
  *n = (int)d.size();
  for (int i = 0; i < cap && i < (int)d.size(); ++i) out[i] = d[i];
  return MPSGB_OK;
}

int mpsgb_footprint_bytes(const mpsgb_config* cfg, size_t* bytes) {
  if (!bytes) return fail(MPSGB_EINVAL, "null argument");
  int s = check_config(cfg);
  if (s) return s;
  mpsgb::Layout L;
  std::string err;
  if (!mpsgb::make_layout(*cfg, L, err)) return fail(MPSGB_EINVAL, err);
  double mb = 1;
  for (double b : L.bound) mb = std::max(mb, b);
  double chi = std::min<double>(cfg->chi_max, mb);
  int dmax = 1;
  for (int k : L.k) dmax = std::max(dmax, 1 << k);
  size_t elem = cfg->prec == MPSGB_FP64 ? 16 : 8;
  *bytes = (size_t)(chi * chi) * dmax * L.N * elem;
  return MPSGB_OK;
}

int mpsgb_batch_step(mpsgb_handle* hs, int count, int nlayers, int use_graph) {
  if (!hs || count < 0 || nlayers < 0) return fail(MPSGB_EINVAL, "bad batch arguments");
  if (use_graph != 0 && use_graph != 1) return fail(MPSGB_EINVAL, "use_graph must be 0 or 1");
  const int nsteps = nlayers;
  for (int i = 0; i < count; ++i) {
    if (!hs[i] || !hs[i]->e) return fail(MPSGB_EINVAL, "null handle in batch");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(MPSGB_EINVAL, "the same handle twice in a batch");
  }
  std::vector<int> st(count, 0);
  std::vector<std::string> msg(count);
  std::vector<std::thread> th;
  th.reserve(count);
  for (int i = 0; i < count; ++i)
    th.emplace_back([&, i] {
      mpsgb::set_graphs_enabled(use_graph != 0);
      const mpsgb_config& c = hs[i]->e->cfg;
      st[i] = mpsgb_step(hs[i], c.J, c.h, c.dt, c.trotter_order, nsteps);
      if (st[i]) msg[i] = mpsgb_last_error();
    });
  for (auto& t : th) t.join();
  for (int i = 0; i < count; ++i)
    if (st[i]) return fail(st[i], "handle " + std::to_string(i) + ": " + msg[i]);
  g_err.clear();
  return MPSGB_OK;
}

int mpsgb_save(mpsgb_handle h, const char* path) {
  if (!h || !h->e || !path) return fail(MPSGB_EINVAL, "null argument");
  return guarded([&]() -> int { return h->e->save(path); });
}

int mpsgb_load(const char* path, const mpsgb_allocator* alloc, void* cuda_stream, mpsgb_handle* out) {
  if (!path || !out) return fail(MPSGB_EINVAL, "null argument");
  *out = nullptr;
  return guarded([&]() -> int {
    FILE* fh = std::fopen(path, "rb");
    if (!fh) return fail(MPSGB_EINVAL, std::string("cannot open ") + path);
    char magic[8];
    mpsgb_config cfg;
    if (std::fread(magic, 1, 8, fh) != 8 || std::memcmp(magic, "MPSGBv2", 8) != 0 ||
        std::fread(&cfg, sizeof(cfg), 1, fh) != 1) {
      std::fclose(fh);
      return fail(MPSGB_EINVAL, "not an mpsgb checkpoint");
    }
    mpsgb_handle h = nullptr;
    int s = create_impl(&cfg, alloc, cuda_stream, &h);
    if (s) { std::fclose(fh); return s; }
    try {
      h->e->load_blocks(fh);
    } catch (...) {
      std::fclose(fh);
      mpsgb_destroy(h);
      throw;
    }
    std::fclose(fh);
    *out = h;
    return MPSGB_OK;
  });
}

void mpsgb_destroy(mpsgb_handle h) {
  if (!h) return;
  delete h->e;
  delete h;
}

const char* mpsgb_last_error(void) { return g_err.c_str(); }

int mpsgb_stats(mpsgb_handle h, long long out[5]) {
  if (!h || !h->e || !out) return fail(MPSGB_EINVAL, "null argument");
  const auto& s = h->e->stats;
  out[0] = s.truncations; out[1] = s.gates; out[2] = s.centre_moves; out[3] = s.eig_calls; out[4] = s.eig_sweeps;
  return MPSGB_OK;
}

long long mpsgb_set_wait_limit(long long cycles) {
  long long prev = mpsgb::wait_limit_cycles();
  mpsgb::set_wait_limit_cycles(cycles > 0 ? cycles : 4000000000LL);
  return prev;
}

int mpsgb_counters(mpsgb_handle h, long long* out, int cap, int* n) {
  if (!h || !h->e || !n || (cap > 0 && !out)) return fail(MPSGB_EINVAL, "null argument");
  const auto& s = h->e->stats;
  const long long v[7] = {s.truncations, s.gates, s.centre_moves, s.eig_calls, s.eig_sweeps, s.chol_ok, s.chol_fallbacks};
  *n = 7;
  for (int i = 0; i < cap && i < 7; ++i) out[i] = v[i];
  return MPSGB_OK;
}

unsigned long long mpsgb_launch_count(void) { return __atomic_load_n(&mpsgb::g_launch_count, __ATOMIC_RELAXED); }

int mpsgb_schedule_info(int Lx, int Ly, long long out[6]) {
  if (!out) return fail(MPSGB_EINVAL, "null argument");
  mpsgb::Layout L;
  std::string err;
  if (!mpsgb::make_layout(Lx, Ly, L, err)) return fail(MPSGB_EINVAL, err);
  return schedule_info_of(L, out);
}

int mpsgb_schedule_gates(int Lx, int Ly, int* out, int cap, int* n) {
  if (!n || (cap > 0 && !out)) return fail(MPSGB_EINVAL, "null argument");
  mpsgb::Layout L;
  std::string err;
  if (!mpsgb::make_layout(Lx, Ly, L, err)) return fail(MPSGB_EINVAL, err);
  return schedule_gates_of(L, out, cap, n);
}

int mpsgb_config_schedule_info(const mpsgb_config* cfg, long long out[6]) {
  if (!cfg || !out) return fail(MPSGB_EINVAL, "null argument");
  mpsgb::Layout L;
  std::string err;
  if (!mpsgb::make_layout(*cfg, L, err)) return fail(MPSGB_EINVAL, err);
  return schedule_info_of(L, out);
}

int mpsgb_config_schedule_gates(const mpsgb_config* cfg, int* out, int cap, int* n) {
  if (!cfg || !n || (cap > 0 && !out)) return fail(MPSGB_EINVAL, "null argument");
  mpsgb::Layout L;
  std::string err;
  if (!mpsgb::make_layout(*cfg, L, err)) return fail(MPSGB_EINVAL, err);
  return schedule_gates_of(L, out, cap, n);
}

int mpsgb_tc_gemm_selftest(int M, int N, int K, int mode, unsigned long long seed, double* rel_err) {
  if (!rel_err || M < 1 || N < 1 || K < 1 || (long long)M * N > (1LL << 26) || (long long)K * (M + N) > (1LL << 28))
    return fail(MPSGB_EINVAL, "bad self-test arguments");
  int s = mpsgb::tc_selftest(M, N, K, mode, seed, rel_err);
  if (s == -3) return fail(MPSGB_ETIMEDOUT, "tensor-core GEMM: a bounded wait ran out");
  if (s == -4) return fail(MPSGB_EDEVICE, "CUDA error in the tensor-core GEMM self-test");
  if (s != 0) return fail(MPSGB_EDEVICE, "tensor-core GEMM could not be set up (tensor maps)");
  return MPSGB_OK;
}

int mpsgb_eig_selftest(int n, int fp64, int kind, unsigned long long seed, double out[6]) {
  if (!out || n < 1 || n > 4096 || kind < 0 || kind > 2) return fail(MPSGB_EINVAL, "bad self-test arguments");
  int s = mpsgb::eig_selftest(n, fp64, kind, seed, out);
  if (s != 0) return fail(MPSGB_EDEVICE, "CUDA error in the eigensolver self-test");
  return MPSGB_OK;
}

int mpsgb_svd_selftest(int p, int q, int fp64, const double* X, double* s, double out[6]) {
  if (!X || !s || !out || p < 1 || q < 1 || p > 4096 || (long long)p * q > (1LL << 24))
    return fail(MPSGB_EINVAL, "bad self-test arguments");
  const int st = mpsgb::svd_selftest(p, q, fp64, X, s, out);
  if (st != 0) return fail(MPSGB_EDEVICE, "CUDA error in the SVD self-test");
  return MPSGB_OK;
}

int mpsgb_eigh_noalloc(int n, int fp64, const void* A, long long lda, void* w, void* V, long long ldv,
                       void* cuda_stream) {
  if (!A || !w || !V) return fail(MPSGB_EINVAL, "null pointer");
  if (n < 1 || n > 128) return fail(MPSGB_EINVAL, "mpsgb_eigh_noalloc: n must be in 1..128 (fixed 1 MiB device scratch)");
  if (lda < n || ldv < n) return fail(MPSGB_EINVAL, "leading dimension smaller than n");
  int s = mpsgb::eigh_noalloc(n, fp64, A, lda, w, V, ldv, (cudaStream_t)cuda_stream);
  if (s == -1) return fail(MPSGB_EINVAL, "mpsgb_eigh_noalloc: matrix does not fit the fixed scratch");
  if (s == -3) return fail(MPSGB_ETIMEDOUT, "mpsgb_eigh_noalloc: Jacobi sweep limit reached");
  if (s < 0) return fail(MPSGB_EDEVICE, "mpsgb_eigh_noalloc: CUDA error");
  g_err.clear();
  return MPSGB_OK;
}

double mpsgb_initial_theta(double J, double hx, double dtheta) { return std::asin(hx / (4.0 * J)) + dtheta; }

double mpsgb_initial_theta_lattice(mpsgb_lattice lattice, double J, double hx, double dtheta) {
  const double z = lattice == MPSGB_LATTICE_2D_GROUPED ? 4.0 : lattice == MPSGB_LATTICE_3D_SITES ? 6.0 : 0.0;
  if (z == 0.0) return std::nan("");
  return std::asin(hx / (z * J)) + dtheta;
}

double mpsgb_gamma_fit(int temperature, int chi, int n) {
  // Table gamma_scaling: (a, b) for low / mid / high
  static const double a[3] = {2.588, 1.8252, 1.641};
  static const double b[3] = {0.0, 0.0, -0.1298};
  if (temperature < 0 || temperature > 2 || chi < 1 || n < 1) return std::nan("");
  return a[temperature] * std::log2((double)chi) / n + b[temperature];
}

double mpsgb_gamma_fit_lattice(mpsgb_lattice lattice, int temperature, int chi, int n) {
  if (lattice == MPSGB_LATTICE_2D_GROUPED) return mpsgb_gamma_fit(temperature, chi, n);
  if (lattice != MPSGB_LATTICE_3D_SITES) return std::nan("");
  // Table 3d_gamma_scaling: (a, b) for low / mid / high (b = 0 throughout)
  static const double a[3] = {2.654, 2.153, 1.5104};
  if (temperature < 0 || temperature > 2 || chi < 1 || n < 1) return std::nan("");
  return a[temperature] * std::log2((double)chi) / n;
}

int mpsgb_rescale(double z, double z2, double F, double gamma, double out[2]) {
  if (!out) return fail(MPSGB_EINVAL, "null argument");
  out[0] = F * z;
  out[1] = z2 * std::pow(F, gamma);
  return MPSGB_OK;
}

}  // extern "C"
