// Host engine of one grouped-qubit MPS: layout and schedule, gate application with
// the Gram/eigen truncation sweep, centre moves, observables, checkpoints.
//
// Truncation of an inter-block gate exp(-i phi Z_i Z_j) on blocks p < q (Sec. III):
// the gate is written as the rank-2 MPO  sum_v P_v(i) (x) exp(-i phi z_v Z_j)
// (P_v projects qubit i on bit v, z_v = 1 - 2v).  With the orthogonality centre on
// block p and blocks p+1..q right-isometric:
//  1. right environments: at bond q-1 the Gram of the two MPO branches of block q,
//     E = [[Y_0 + Y_1, e^{-2i phi} Y_0 + e^{2i phi} Y_1], [h.c., Y_0 + Y_1]] with
//     Y_w = B_w B_w^H over the columns of block q whose qubit j has bit w; carried to
//     bonds q-2 .. p through the untouched blocks (E -> sum_s C_s E C_s^H per 2x2 block);
//  2. left to right over bonds m = p .. q-1: the left factor L_m (rows: left bond x
//     physical, columns: MPO index x bond) has Gram G = L^H L (block diagonal at m = p:
//     the two row sets of qubit i); with G = U D U^H and Gs = U D^{1/2} (numerical range)
//     the state across bond m has squared singular values eig(H), H = Gs^H E Gs; the k
//     largest (k = min(chi, numerical rank)) are kept, the new left isometry is
//     L_m U D^{-1/2} V_k, the carry to the right is (Gs V_k)^H / sqrt(kept), and the
//     truncation fidelity is f = sum(kept) / sum(all) -- exactly the SVD truncation of the
//     state across the bond;
//  3. the carry multiplies the MPO branches of block q, which becomes the new centre.
// That Gram route (complex64 forms) squares the Schmidt values, so values below about
// sqrt(eps) s_0 are not resolved.  The FP64 form therefore takes the exact route, the plain
// definition of Sec. III with no squaring: the MPO cos(phi) I I - i sin(phi) Z_i Z_j is applied
// to blocks p .. q (spanned bonds doubled), blocks q .. p+1 are made right-isometric, and each
// spanned bond p .. q-1 in turn is truncated by the SVD of the centre block (one-sided Jacobi on
// its conjugate transpose, svd.cu), keeping min(chi, numerical rank) values; centre moves and
// Schmidt spectra use the same SVD.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <type_traits>
#include <vector>

#include "engine.hpp"
#include "kernels.hpp"

namespace mpsgb {

// ------------------------------------------------------------------ layout
namespace {
// gate order (first block, second block, first qubit, second qubit) and the exact bond bounds
void finish_layout(Layout& L) {
  std::sort(L.inter.begin(), L.inter.end(), [](const Layout::Gate& a, const Layout::Gate& b) {
    if (a.p != b.p) return a.p < b.p;
    if (a.q != b.q) return a.q < b.q;
    if (a.qi != b.qi) return a.qi < b.qi;
    return a.qj < b.qj;
  });
  L.bound.assign(L.N - 1, 0);
  int total = 0;
  for (int b = 0; b < L.N; ++b) total += L.k[b];
  int left = 0;
  for (int m = 0; m < L.N - 1; ++m) {
    left += L.k[m];
    L.bound[m] = std::ldexp(1.0, std::min(left, total - left));
  }
}
}  // namespace

bool make_layout(int Lx, int Ly, Layout& L, std::string& err) {
  if (Lx < 2 || Ly < 2 || Lx > 16 || Ly > 10 || Lx * Ly > 160) {
    err = "grid must have 2 <= Lx <= 16, 2 <= Ly <= 10 and at most 160 qubits";
    return false;
  }
  L = Layout();
  L.Lx = Lx; L.Ly = Ly; L.N = 2 * Lx; L.n = Lx * Ly;
  const int h0 = (Ly + 1) / 2;
  L.k.assign(L.N, 0);
  L.qubits.assign(L.N, {});
  L.intra.assign(L.N, {});
  std::vector<std::pair<int, int>> home(L.n);  // qubit -> (block, bit position from MSB)
  for (int r = 0; r < Lx; ++r)
    for (int g = 0; g < 2; ++g) {
      int pos = (r % 2 == 0) ? 2 * r + g : 2 * r + 1 - g;
      int c0 = g == 0 ? 0 : h0, c1 = g == 0 ? h0 : Ly;
      for (int c = c0; c < c1; ++c) {
        home[r * Ly + c] = {pos, (int)L.qubits[pos].size()};
        L.qubits[pos].push_back(r * Ly + c);
      }
      L.k[pos] = c1 - c0;
    }
  L.stag.assign(L.n, 1);
  for (int r = 0; r < Lx; ++r)
    for (int c = 0; c < Ly; ++c) L.stag[r * Ly + c] = ((r + c) & 1) ? -1 : 1;
  std::set<std::pair<int, int>> bonds;
  for (int r = 0; r < Lx; ++r)
    for (int c = 0; c < Ly; ++c) {
      int a = r * Ly + c;
      int nb[2] = {((r + 1) % Lx) * Ly + c, r * Ly + (c + 1) % Ly};
      for (int b : nb)
        if (b != a) bonds.insert({std::min(a, b), std::max(a, b)});
    }
  for (auto& bd : bonds) {
    auto h1 = home[bd.first], h2 = home[bd.second];
    if (h1.first == h2.first) {
      L.intra[h1.first].push_back({std::min(h1.second, h2.second), std::max(h1.second, h2.second)});
    } else {
      Layout::Gate g;
      if (h1.first < h2.first) g = {h1.first, h2.first, bd.first, bd.second, h1.second, h2.second};
      else g = {h2.first, h1.first, bd.second, bd.first, h2.second, h1.second};
      L.inter.push_back(g);
    }
  }
  finish_layout(L);
  return true;
}

// 3D cubic grid with open boundaries, one qubit per site, sites along a snake through the layers
bool make_layout_3d(int Lx, int Ly, int Lz, Layout& L, std::string& err) {
  if (Lx < 2 || Ly < 2 || Lz < 2 || Lx > 16 || Ly > 16 || Lz > 16 || Lx * Ly * Lz > 512) {
    err = "3D grid must have 2 <= Lx, Ly, Lz <= 16 and at most 512 qubits";
    return false;
  }
  L = Layout();
  L.Lx = Lx; L.Ly = Ly; L.Lz = Lz; L.n = Lx * Ly * Lz; L.N = L.n;
  L.k.assign(L.N, 1);
  L.qubits.assign(L.N, {});
  L.intra.assign(L.N, {});
  auto qid = [&](int x, int y, int z) { return (z * Lx + x) * Ly + y; };
  L.stag.assign(L.n, 1);
  for (int z = 0; z < Lz; ++z)
    for (int x = 0; x < Lx; ++x)
      for (int y = 0; y < Ly; ++y) L.stag[qid(x, y, z)] = ((x + y + z) & 1) ? -1 : 1;
  std::vector<int> pos_of(L.n, -1);
  int pos = 0, row = 0;
  for (int z = 0; z < Lz; ++z)
    for (int i = 0; i < Lx; ++i, ++row) {
      const int x = (z % 2 == 0) ? i : Lx - 1 - i;
      for (int j = 0; j < Ly; ++j) {
        const int y = (row % 2 == 0) ? j : Ly - 1 - j;
        pos_of[qid(x, y, z)] = pos;
        L.qubits[pos].push_back(qid(x, y, z));
        ++pos;
      }
    }
  for (int z = 0; z < Lz; ++z)
    for (int x = 0; x < Lx; ++x)
      for (int y = 0; y < Ly; ++y) {
        const int a = qid(x, y, z);
        const int nb[3] = {x + 1 < Lx ? qid(x + 1, y, z) : -1, y + 1 < Ly ? qid(x, y + 1, z) : -1,
                           z + 1 < Lz ? qid(x, y, z + 1) : -1};
        for (int b : nb) {
          if (b < 0) continue;
          const int pa = pos_of[a], pb = pos_of[b];
          L.inter.push_back(pa < pb ? Layout::Gate{pa, pb, a, b, 0, 0} : Layout::Gate{pb, pa, b, a, 0, 0});
        }
      }
  finish_layout(L);
  return true;
}

// open Lx x Ly grid, one qubit per site along the row snake; bonds carry their set of the XY
// model's Trotter step: horizontal bonds starting on an even / odd column (A / B), vertical bonds
// starting on an even / odd row (C / D)
bool make_layout_2d_sites(int Lx, int Ly, Layout& L, std::string& err) {
  if (Lx < 2 || Ly < 2 || Lx > 16 || Ly > 16 || Lx * Ly > 256) {
    err = "2D one-qubit-per-site grid must have 2 <= Lx, Ly <= 16 and at most 256 qubits";
    return false;
  }
  L = Layout();
  L.Lx = Lx; L.Ly = Ly; L.n = Lx * Ly; L.N = L.n;
  L.k.assign(L.N, 1);
  L.qubits.assign(L.N, {});
  L.intra.assign(L.N, {});
  L.stag.assign(L.n, 1);
  std::vector<int> pos_of(L.n, -1);
  int pos = 0;
  for (int r = 0; r < Lx; ++r)
    for (int i = 0; i < Ly; ++i) {
      const int c = (r % 2 == 0) ? i : Ly - 1 - i;
      pos_of[r * Ly + c] = pos;
      L.qubits[pos].push_back(r * Ly + c);
      L.stag[r * Ly + c] = ((r + c) & 1) ? -1 : 1;
      ++pos;
    }
  auto add = [&](int a, int b, int set) {
    const int pa = pos_of[a], pb = pos_of[b];
    Layout::Gate g = pa < pb ? Layout::Gate{pa, pb, a, b, 0, 0} : Layout::Gate{pb, pa, b, a, 0, 0};
    g.set = set;
    L.inter.push_back(g);
  };
  for (int r = 0; r < Lx; ++r)
    for (int c = 0; c < Ly; ++c) {
      if (c + 1 < Ly) add(r * Ly + c, r * Ly + c + 1, c % 2);
      if (r + 1 < Lx) add(r * Ly + c, (r + 1) * Ly + c, 2 + r % 2);
    }
  finish_layout(L);
  return true;
}

bool make_layout(const mpsgb_config& c, Layout& L, std::string& err) {
  if (c.lattice == MPSGB_LATTICE_2D_SITES) {
    if (c.Lz != 0 && c.Lz != 1) {
      err = "the 2D lattice takes Lz = 0 or 1";
      return false;
    }
    return make_layout_2d_sites(c.Lx, c.Ly, L, err);
  }
  if (c.lattice == MPSGB_LATTICE_2D_GROUPED) {
    if (c.Lz != 0 && c.Lz != 1) {
      err = "the 2D lattice takes Lz = 0 or 1";
      return false;
    }
    return make_layout(c.Lx, c.Ly, L, err);
  }
  if (c.lattice == MPSGB_LATTICE_3D_SITES) return make_layout_3d(c.Lx, c.Ly, c.Lz, L, err);
  err = "unknown lattice";
  return false;
}

// ------------------------------------------------------------------ device memory
struct DevMem {
  mpsgb_allocator a{};
  bool custom = false;
  cudaStream_t st = nullptr;
  std::vector<void*> live;
  void* get(size_t bytes) {
    void* p = nullptr;
    if (custom) p = a.alloc(bytes, (void*)st, a.ctx);
    else if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) p = nullptr;
    if (p) live.push_back(p);
    return p;
  }
  void release() {
    for (void* p : live) {
      if (custom) a.free(p, (void*)st, a.ctx);
      else cudaFreeAsync(p, st);
    }
    live.clear();
  }
};

struct Arena {
  char* base = nullptr;
  size_t size = 0, off = 0;
  template <typename T> T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (off + bytes > size) return nullptr;
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

// ------------------------------------------------------------------ engine
template <typename R>
class EngineT : public Engine {
  using C = Cx<R>;

 public:
  DevMem mem;
  std::vector<C*> blk;
  C* spare = nullptr;
  Arena ar;
  C* dU = nullptr;     // per-block d x d unitaries of the current local layer
  double* dsc = nullptr;  // device FP64 scratch (reductions)
  long long cap = 0;   // elements per block buffer
  int chi_eff = 1, dmax = 2;
  double tau = 1e-13;  // numerical-rank threshold on squared singular values (relative)
  std::vector<R> hbuf;
  bool tc = false;        // block-sized contractions on the tensor cores (split forms)
  bool tc_tf32 = false;   // ... with TF32 splits (kind::tf32) instead of BF16
  GraphCache* gcache = new_graph_cache();  // CUDA graphs of this handle's fixed launch sequences
  void* tcws = nullptr;   // BF16 operand planes of the tensor-core GEMM
  size_t tcws_bytes = 0;
  int* derr = nullptr;    // device error word of bounded waits in kernels
  bool exact = false;     // FP64 form: truncation and centre moves by the SVD (one-sided Jacobi)
  long long stats_chol_fallbacks = 0;
  std::vector<int> kpos;  // qubits of the block at each position (L.k except inside a SWAP-routed gate)
  bool swap_route = false;  // truncation cores whose G was too close to singular for Cholesky

  // Block-sized contraction: tensor cores in the split form (when every dimension is at least
  // 64), FP32 / FP64 CUDA cores otherwise.
  void mm(int M, int N, int K, C alpha, View<R> A, View<R> B, C beta, View<R> Cv) {
    if constexpr (std::is_same<R, float>::value) {
      if (tc && M >= 64 && N >= 64 && K >= 64) {
        int s = tc_gemm(stream, M, N, K, alpha, A, B, beta, Cv, tcws, tcws_bytes, derr, tc_tf32);
        if (s != 0) throw Fail{MPSGB_EDEVICE, "tensor-core GEMM set-up failed"};
        return;
      }
    }
    gemm<R>(stream, M, N, K, alpha, A, B, beta, Cv);
  }
  void check_device_error() {
    int h = 0;
    cudaMemcpyAsync(&h, derr, sizeof(int), cudaMemcpyDeviceToHost, stream);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) throw Fail{MPSGB_EDEVICE, std::string("device: ") + cudaGetErrorString(e)};
    if (h != 0) throw Fail{MPSGB_ETIMEDOUT, "a bounded wait in a tensor-core kernel ran out"};
  }

  ~EngineT() override {
    if (stream) cudaStreamSynchronize(stream);
    free_graph_cache(gcache);
    mem.release();
    if (stream) cudaStreamSynchronize(stream);
  }

  void check(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Fail{MPSGB_EDEVICE, std::string(what) + ": " + cudaGetErrorString(e)};
  }
  void synchronize(const char* what) {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) throw Fail{MPSGB_EDEVICE, std::string(what) + ": " + cudaGetErrorString(e)};
    check(what);
  }
  // local dimension of the block at position b (SWAP routing exchanges blocks transiently)
  int d(int b) const { return 1 << kpos[b]; }
  int left(int b) const { return b == 0 ? 1 : dims[b - 1]; }
  int right(int b) const { return b == L.N - 1 ? 1 : dims[b]; }
  int cap_bond(int m) const { return (int)std::min<double>(cfg.chi_max, L.bound[m]); }

  void init(const mpsgb_config& c, const mpsgb_allocator* alloc, cudaStream_t st) {
    cfg = c;
    stream = st;
    mem.st = st;
    if (alloc && alloc->alloc && alloc->free) { mem.a = *alloc; mem.custom = true; }
    std::string err;
    if (!make_layout(c, L, err)) throw Fail{MPSGB_EINVAL, err};
    if (c.chi_max < 1) throw Fail{MPSGB_EINVAL, "chi_max must be >= 1"};
    kpos = L.k;
    swap_route = c.route == MPSGB_ROUTE_SWAP;
    double mb = 1;
    for (double b : L.bound) mb = std::max(mb, b);
    chi_eff = (int)std::min<double>(c.chi_max, mb);
    dmax = 1;
    for (int b = 0; b < L.N; ++b) dmax = std::max(dmax, d(b));
    cap = (long long)chi_eff * chi_eff * dmax;
    tau = sizeof(R) == 8 ? 1e-16 : 1e-12;
    // exact route: a block carries doubled bonds on both sides while an MPO is applied
    const long long cap_blk = exact ? 4 * cap : cap;
    for (int b = 0; b <= L.N; ++b) {
      C* p = (C*)mem.get(sizeof(C) * cap_blk);
      if (!p) throw Fail{MPSGB_ENOMEM, "allocation of block buffers failed"};
      if (b < L.N) blk.push_back(p); else spare = p;
    }
    long long c2 = (long long)chi_eff * chi_eff;
    long long n2 = 2LL * chi_eff;
    size_t phase = sizeof(C) * (3 * cap + 2 * c2 * (L.N + 8) + 14 * n2 * n2) + sizeof(R) * 8 * n2;
    size_t obs = sizeof(C) * (4 * cap + 16 * c2);
    size_t eigws = eigh_workspace_bytes((int)n2, 1, (int)sizeof(R));
    ar.size = std::max(phase, obs) + eigws + (64 << 10);
    if (swap_route) {
      // two-site tensors of SWAP routing: theta and its permuted copy, Vh, U ((chi d)^2 each) and the
      // SVD's working copy; bounded so that a two-site SVD stays a small problem
      const long long w = (long long)chi_eff * dmax;
      if (w > 4096) throw Fail{MPSGB_EINVAL, "SWAP routing needs chi * d <= 4096 (two-site SVD of a (chi d)^2 matrix)"};
      const size_t sw = sizeof(C) * 4 * (size_t)w * w + sizeof(double) * 2 * w +
                        svd_rows_workspace_bytes((int)w, (int)w, 1, (int)sizeof(R)) + (1 << 20);
      ar.size = std::max(ar.size, sw);
    }
    if (exact) {
      // A^H copy, Vh, U, T (<= 4 cap and (2 chi)^2 each) and the SVD's own working copy
      const size_t svdws = svd_rows_workspace_bytes((int)n2, (int)(4 * cap / n2 + 1), 1, (int)sizeof(R));
      ar.size = std::max<size_t>(ar.size, sizeof(C) * (8 * cap + 3 * n2 * n2) + sizeof(double) * 4 * n2 + svdws + (1 << 20));
      ar.size = std::max(ar.size, obs + (size_t)(64 << 10));
    }
    ar.base = (char*)mem.get(ar.size);
    dU = (C*)mem.get(sizeof(C) * 32 * 32 * L.N);
    dsc = (double*)mem.get(sizeof(double) * 16);
    derr = (int*)mem.get(sizeof(int) * 4);
    if (!ar.base || !dU || !dsc || !derr) throw Fail{MPSGB_ENOMEM, "allocation of workspace failed"};
    cudaMemsetAsync(derr, 0, sizeof(int) * 4, stream);
    if (tc) {
      // largest operand pair: the Gram of a left factor (2 chi x chi d) with itself
      tcws_bytes = tc_gemm_workspace_bytes(4LL * chi_eff, 4LL * chi_eff, (long long)chi_eff * dmax, tc_tf32) + (1 << 20);
      tcws = mem.get(tcws_bytes);
      if (!tcws) throw Fail{MPSGB_ENOMEM, "allocation of tensor-core workspace failed"};
    }
    dims.assign(L.N - 1, 1);
    if (c.model == MPSGB_MODEL_XY) {  // |Neel>: the ground state of sum_j s_j Z_j (one qubit per site)
      for (int b = 0; b < L.N; ++b) {
        const bool one = L.stag[L.qubits[b][0]] > 0;
        init_product<R>(stream, blk[b], 1, one ? 0.0 : 1.0, one ? 1.0 : 0.0);
      }
    } else {
      double cth = std::cos(c.theta / 2), sth = std::sin(c.theta / 2);
      for (int b = 0; b < L.N; ++b) init_product<R>(stream, blk[b], L.k[b], cth, sth);
    }
    centre = 0;
    F = 1.0;
    synchronize("create");
  }

  // ---------------------------------------------------------- eigen helper (device in, host eigenvalues out)
  // nvec > 0: only the eigenvectors of the nvec largest eigenvalues are needed (the others are
  // not computed on the tridiagonal route)
  void eig(int n, C* A, R* w, C* V, void* ws, std::vector<double>& hw, int nvec = 0) {
    GraphScope gs(gcache);
    int sw = eigh<R>(stream, n, A, n, 0, w, 0, V, n, 0, 1, ws, nvec);
    stats.eig_calls++;
    if (sw == -1) throw Fail{MPSGB_ETIMEDOUT, "Jacobi eigensolver did not converge within its sweep limit"};
    if (sw == -2) throw Fail{MPSGB_ETIMEDOUT, "eigensolver: a bounded grid barrier of the reduction timed out"};
    if (sw == -3) throw Fail{MPSGB_ESTATE, "eigensolver: dependent eigenvectors could not be orthonormalised"};
    if (sw < 0) throw Fail{MPSGB_EDEVICE, "eigensolver: launch or device error"};
    stats.eig_sweeps += sw;
    hbuf.resize(n);
    cudaMemcpyAsync(hbuf.data(), w, sizeof(R) * n, cudaMemcpyDeviceToHost, stream);
    synchronize("eigensolver");
    hw.assign(hbuf.begin(), hbuf.end());
    if (tc) check_device_error();
  }
  static int count_above(const std::vector<double>& w, double rel, int cap_) {
    if (w.empty() || !(w[0] > 0)) return 0;
    int c = 0;
    while (c < (int)w.size() && c < cap_ && w[c] > rel * w[0]) ++c;
    return c;
  }

  // ---------------------------------------------------------- local layers
  void upload_and_apply(const std::vector<std::vector<std::complex<double>>>& U) {
    std::vector<C> h((size_t)L.N * 1024);
    for (int b = 0; b < L.N; ++b) {
      int dd = d(b);
      for (int i = 0; i < dd * dd; ++i) h[(size_t)b * 1024 + i] = cmake<R>((R)U[b][i].real(), (R)U[b][i].imag());
    }
    cudaMemcpyAsync(dU, h.data(), sizeof(C) * h.size(), cudaMemcpyHostToDevice, stream);  // pageable: host-synchronous
    for (int b = 0; b < L.N; ++b) {
      if (U[b].empty()) continue;
      apply_phys<R>(stream, blk[b], left(b), d(b), right(b), dU + (size_t)b * 1024);
    }
    check("local layer");
  }
  static std::vector<std::complex<double>> rx_kron(int k, double alpha) {
    std::complex<double> c(std::cos(alpha), 0), s(0, -std::sin(alpha));
    std::vector<std::complex<double>> u{1.0};
    int n = 1;
    for (int t = 0; t < k; ++t) {  // kron(u, r1): first factor is the most significant bit
      std::vector<std::complex<double>> v((size_t)4 * n * n);
      std::complex<double> r1[4] = {c, s, s, c};
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          for (int a = 0; a < 2; ++a)
            for (int bb = 0; bb < 2; ++bb) v[(size_t)(2 * i + a) * (2 * n) + (2 * j + bb)] = u[(size_t)i * n + j] * r1[a * 2 + bb];
      u.swap(v);
      n *= 2;
    }
    return u;
  }
  std::vector<std::complex<double>> intra_diag(int b, double phi) const {
    int k = L.k[b], dd = 1 << k;
    std::vector<std::complex<double>> u((size_t)dd * dd, 0.0);
    for (int s = 0; s < dd; ++s) {
      double e = 0;
      for (auto& pr : L.intra[b]) {
        double zt = 1 - 2 * ((s >> (k - 1 - pr.first)) & 1), zu = 1 - 2 * ((s >> (k - 1 - pr.second)) & 1);
        e += zt * zu;
      }
      u[(size_t)s * dd + s] = std::exp(std::complex<double>(0, -phi * e));
    }
    return u;
  }
  static std::vector<std::complex<double>> matmul(const std::vector<std::complex<double>>& a,
                                                  const std::vector<std::complex<double>>& b, int n) {
    std::vector<std::complex<double>> c((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j) c[(size_t)i * n + j] += a[(size_t)i * n + k] * b[(size_t)k * n + j];
    return c;
  }

  int apply_zstag(double alpha) override {
    std::vector<std::vector<std::complex<double>>> U(L.N);
    for (int b = 0; b < L.N; ++b) {
      const int k = L.k[b], dd = 1 << k;
      U[b].assign((size_t)dd * dd, 0.0);
      for (int sidx = 0; sidx < dd; ++sidx) {
        double e = 0;
        for (int t = 0; t < k; ++t) e += L.stag[L.qubits[b][t]] * (1 - 2 * ((sidx >> (k - 1 - t)) & 1));
        U[b][(size_t)sidx * dd + sidx] = std::exp(std::complex<double>(0, -alpha * e));
      }
    }
    upload_and_apply(U);
    return MPSGB_OK;
  }
  int apply_x(double alpha) override {
    if (cfg.model == MPSGB_MODEL_XY) throw Fail{MPSGB_EINVAL, "an X layer is not a layer of the XY model"};
    std::vector<std::vector<std::complex<double>>> U(L.N);
    for (int b = 0; b < L.N; ++b) U[b] = rx_kron(L.k[b], alpha);
    upload_and_apply(U);
    return MPSGB_OK;
  }
  void apply_intra(double phi, double alpha_before) {
    // diag(intra ZZ) * Rx(alpha_before)^{(x)k}; alpha_before = 0 means phases only
    std::vector<std::vector<std::complex<double>>> U(L.N);
    for (int b = 0; b < L.N; ++b) {
      if (L.intra[b].empty() && alpha_before == 0.0) continue;
      U[b] = intra_diag(b, phi);
      if (alpha_before != 0.0) U[b] = matmul(U[b], rx_kron(L.k[b], alpha_before), d(b));
    }
    upload_and_apply(U);
  }
  int apply_zz(double phi) override {
    if (cfg.model == MPSGB_MODEL_XY) throw Fail{MPSGB_EINVAL, "a ZZ layer is not a layer of the XY model"};
    apply_intra(phi, 0.0);
    inter_layer(phi);
    return MPSGB_OK;
  }
  int apply_gates(int first, int count, double phi) override {
    if (cfg.model == MPSGB_MODEL_XY) throw Fail{MPSGB_EINVAL, "ZZ gates are not gates of the XY model"};
    if (first < 0 || count < 0 || first + count > (int)L.inter.size())
      throw Fail{MPSGB_EINVAL, "gate range outside the schedule"};
    last_f_min = 1.0;
    for (int i = first; i < first + count; ++i) any_gate(L.inter[i], phi);
    return MPSGB_OK;
  }
  void inter_layer(double phi) {
    last_f_min = 1.0;
    for (auto& g : L.inter) any_gate(g, phi);
  }
  // the XY model's two-qubit factor exp(-i theta (X X + Y Y)): the identity on |00>, |11> and
  // cos(2 theta) - i sin(2 theta) X on the span of |01>, |10>
  static Gate4 xy_gate(double theta) {
    Gate4 u{};
    for (int i = 0; i < 4; ++i) u.re[5 * i] = 1.0;
    const double c = std::cos(2 * theta), sn = std::sin(2 * theta);
    u.re[5] = u.re[10] = c;
    u.im[6] = u.im[9] = -sn;
    return u;
  }
  // Eq. xy_trotter_step: sets A, B, C at half duration, D whole, C, B, A at half duration
  void xy_step(double g, double dt) {
    static const int sets[7] = {0, 1, 2, 3, 2, 1, 0};
    static const double w[7] = {0.5, 0.5, 0.5, 1.0, 0.5, 0.5, 0.5};
    last_f_min = 1.0;
    for (int l = 0; l < 7; ++l) {
      const Gate4 u = xy_gate(0.5 * g * dt * w[l]);
      for (auto& gt : L.inter)
        if (gt.set == sets[l]) gate_general(gt, u);
    }
  }
  int step(double J, double hx, double dt, int order, int nsteps) override {
    if (cfg.model == MPSGB_MODEL_XY) {
      if (order != 2) throw Fail{MPSGB_EINVAL, "the XY model's Trotter step is second order"};
      for (int s = 0; s < nsteps; ++s) xy_step(J, dt);
      return MPSGB_OK;
    }
    double alpha = order == 2 ? 0.5 * hx * dt : hx * dt, phi = J * dt;
    for (int s = 0; s < nsteps; ++s) {
      apply_intra(phi, alpha);  // X(alpha) then in-block ZZ phases, fused into one pass per block
      inter_layer(phi);
      if (order == 2) apply_x(alpha);
    }
    return MPSGB_OK;
  }


  // ---------------------------------------------------------- exact route (FP64 form)
  // numerical rank of a descending spectrum of a rows x cols matrix: s > s_0 max(rows, cols) eps,
  // eps of the working precision (values below it are rounding noise of the stored blocks)
  static int rank_of(const std::vector<double>& s, long long rows, long long cols, int cap_) {
    if (s.empty() || !(s[0] > 0)) return 0;
    const double eps = sizeof(R) == 8 ? 2.220446049250313e-16 : 1.1920929e-7;
    const double tol = s[0] * (double)std::max(rows, cols) * eps;
    int c = 0;
    while (c < (int)s.size() && c < cap_ && s[c] > tol) ++c;
    return c;
  }
  // X (p x q, row-major) = U diag(s) Vh by Jacobi rotations of the rows; Vh (p x q), U (p x p) and
  // the device copy ds of s are taken from the arena, hs receives s on the host
  void jsvd(const C* X, int p, int q, C*& Vh, C*& U, double*& ds, std::vector<double>& hs) {
    Vh = ar.take<C>((size_t)p * q);
    U = ar.take<C>((size_t)p * p);
    ds = ar.take<double>(p);
    const size_t mark = ar.off;
    void* ws = ar.take<char>(svd_rows_workspace_bytes(p, q, 1, sizeof(R)));
    if (!Vh || !U || !ds || !ws) throw Fail{MPSGB_ENOMEM, "workspace exhausted in the SVD"};
    hs.resize(p);
    const int sw = svd_rows<R>(stream, p, q, X, q, ds, hs.data(), Vh, q, U, p, ws);
    ar.off = mark;
    stats.eig_calls++;
    if (sw == -1) throw Fail{MPSGB_ETIMEDOUT, "Jacobi SVD did not converge within its sweep limit"};
    if (sw == -2) throw Fail{MPSGB_ETIMEDOUT, "Jacobi SVD: a bounded grid barrier timed out"};
    if (sw == -5) throw Fail{MPSGB_ESTATE, "Jacobi SVD: the matrix is not finite"};
    if (sw < 0) throw Fail{MPSGB_EDEVICE, "Jacobi SVD: launch or device error"};
    stats.eig_sweeps += sw;
  }
  // SVD of block m as the (left * d) x right matrix A, through X = A^H = U diag(s) Vh, so that
  // A = Vh^H diag(s) U^H: new left-isometric block Vh[:k]^H; the rest, diag(s_k) * scale * U[:, :k]^H,
  // multiplies block m+1.  k = min(kcap, numerical rank) (at least 1).  Returns k; kept / total are
  // the sums of s^2 over the kept / all values.
  int svd_split_right(int m, int kcap, double scale_pow, double& kept, double& total) {
    ar.off = 0;
    const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    const int l = left(m), dd = d(m), r = dims[m];
    const long long M = (long long)l * dd;
    C* Xt = ar.take<C>((size_t)M * r);
    if (!Xt) throw Fail{MPSGB_ENOMEM, "workspace exhausted in the SVD"};
    copy_view<R, R>(stream, r, (int)M, transposed<R>(blk[m], r, true), rowmajor<R>(Xt, M));
    C *Vh, *U;
    double* ds;
    std::vector<double> s;
    jsvd(Xt, r, (int)M, Vh, U, ds, s);
    const int k = std::max(1, rank_of(s, M, r, kcap));
    kept = 0;
    total = 0;
    for (int i = 0; i < (int)s.size(); ++i) { total += s[i] * s[i]; if (i < k) kept += s[i] * s[i]; }
    if (!(kept > 0)) throw Fail{MPSGB_ESTATE, "zero state at a truncation"};
    copy_view<R, R>(stream, (int)M, k, transposed<R>(Vh, M, true), rowmajor<R>(spare, k));
    std::swap(blk[m], spare);
    C* T = ar.take<C>((size_t)k * r);
    if (!T) throw Fail{MPSGB_ENOMEM, "workspace exhausted in the SVD"};
    copy_view<R, R>(stream, k, r, transposed<R>(U, r, true), rowmajor<R>(T, r));
    scale_rows<R>(stream, k, r, T, r, ds, std::pow(kept, scale_pow));
    const int dn = d(m + 1), rn = right(m + 1);
    gemm<R>(stream, k, dn * rn, r, one, rowmajor<R>(T, r), rowmajor<R>(blk[m + 1], (long long)dn * rn), zero,
            rowmajor<R>(spare, (long long)dn * rn));
    std::swap(blk[m + 1], spare);
    dims[m] = k;
    check("SVD split");
    return k;
  }
  // SVD of block m as the left x (d * right) matrix B = U diag(s) Vh: block m <- Vh[:k] (right-
  // isometric), block m-1 <- block m-1 * U[:, :k] diag(s_k); k = numerical rank (the LQ step)
  void svd_split_left(int m) {
    ar.off = 0;
    const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    const int l = dims[m - 1], dd = d(m), r = right(m);
    const long long row = (long long)dd * r;
    C *Vh, *U;
    double* ds;
    std::vector<double> s;
    jsvd(blk[m], l, (int)row, Vh, U, ds, s);
    const int k = std::max(1, rank_of(s, l, row, l));
    copy_view<R, R>(stream, k, (int)row, rowmajor<R>(Vh, row), rowmajor<R>(spare, row));
    std::swap(blk[m], spare);
    C* T = ar.take<C>((size_t)l * k);
    if (!T) throw Fail{MPSGB_ENOMEM, "workspace exhausted in the SVD"};
    copy_view<R, R>(stream, l, k, rowmajor<R>(U, l), rowmajor<R>(T, k));
    scale_cols<R>(stream, l, k, T, k, ds, 1.0);
    const int lq = left(m - 1), dq = d(m - 1);
    gemm<R>(stream, lq * dq, k, l, one, rowmajor<R>(blk[m - 1], l), rowmajor<R>(T, k), zero, rowmajor<R>(spare, k));
    std::swap(blk[m - 1], spare);
    dims[m - 1] = k;
    check("SVD split");
  }
  // inter-block gate by the plain definition of Sec. III (see the file header)
  void gate_exact(const Layout::Gate& g, double phi) {
    move_centre(g.p);
    const int p = g.p, q = g.q;
    const std::vector<int> od = dims;
    for (int b = p; b <= q; ++b) {
      const int l = b == 0 ? 1 : od[b - 1], r = b == L.N - 1 ? 1 : od[b];
      const int mode = b == p ? 0 : (b == q ? 2 : 1);
      const int shift = b == p ? L.k[p] - 1 - g.ti : (b == q ? L.k[q] - 1 - g.tj : 0);
      mpo_expand<R>(stream, mode, l, d(b), r, blk[b], spare, phi, shift);
      std::swap(blk[b], spare);
    }
    for (int m = p; m < q; ++m) dims[m] = 2 * od[m];
    for (int m = q; m > p; --m) svd_split_left(m);  // right-canonical q .. p+1
    for (int m = p; m < q; ++m) {
      double kept = 0, total = 0;
      svd_split_right(m, cap_bond(m), -0.5, kept, total);
      const double f = kept / total;
      F *= f;
      last_f_min = std::min(last_f_min, f);
      stats.truncations++;
    }
    centre = q;
    stats.gates++;
    check("gate");
  }


  // ---------------------------------------------------------- SWAP routing
  // Two-site update of blocks m, m+1 (the centre on one of them): theta = A B as a (l d_m) x (d_m+1 r)
  // matrix, with a diagonal two-qubit phase exp(-i phi z_a z_b) on the physical indices (bit shift_a
  // of block m, shift_b of block m+1) or with the physical legs exchanged (the blocks swap places),
  // then its SVD truncated to min(chi, numerical rank) values, f = kept / total, renormalised; the
  // singular values go into block m (centre_left) or block m+1.
  void two_site(int m, bool swap, bool with_phase, double phi, int shift_a, int shift_b, bool centre_left,
                const Gate4* gate4 = nullptr) {
    ar.off = 0;
    const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    const int l = left(m), da = d(m), mid = dims[m], db = d(m + 1), r = right(m + 1);
    const long long rowsA = (long long)l * da, colsB = (long long)db * r;
    C* Th = ar.take<C>((size_t)(rowsA * colsB));
    if (!Th) throw Fail{MPSGB_ENOMEM, "workspace exhausted in a two-site update"};
    mm((int)rowsA, (int)colsB, mid, one, rowmajor<R>(blk[m], mid), rowmajor<R>(blk[m + 1], colsB), zero,
       rowmajor<R>(Th, colsB));
    if (with_phase) two_site_phase<R>(stream, l, da, db, r, Th, phi, shift_a, shift_b);
    if (gate4) two_site_gate<R>(stream, l, da, db, r, Th, *gate4, shift_a, shift_b);
    C* X = Th;
    int prow = (int)rowsA, pcol = (int)colsB;
    if (swap) {
      prow = l * db;
      pcol = da * r;
      X = ar.take<C>((size_t)prow * pcol);
      if (!X) throw Fail{MPSGB_ENOMEM, "workspace exhausted in a two-site update"};
      // X[(a, t), (s, b)] = theta[a, s, t, b]
      View<R> src;
      src.ptr = Th;
      src.row = split(db, r, (long long)da * db * r);
      src.col = split(r, 1, (long long)db * r);
      src.conj = false;
      copy_view<R, R>(stream, prow, pcol, src, rowmajor<R>(X, pcol));
    }
    C *Vh, *U;
    double* ds;
    std::vector<double> s;
    jsvd(X, prow, pcol, Vh, U, ds, s);
    const int k = std::max(1, rank_of(s, prow, pcol, std::min(cfg.chi_max, chi_eff)));
    double kept = 0, total = 0;
    for (int i = 0; i < (int)s.size(); ++i) { total += s[i] * s[i]; if (i < k) kept += s[i] * s[i]; }
    if (!(kept > 0)) throw Fail{MPSGB_ESTATE, "zero state at a truncation"};
    const double f = kept / total;
    F *= f;
    last_f_min = std::min(last_f_min, f);
    stats.truncations++;
    const double rs = 1.0 / std::sqrt(kept);
    copy_view<R, R>(stream, prow, k, rowmajor<R>(U, prow), rowmajor<R>(spare, k));
    if (centre_left) scale_cols<R>(stream, prow, k, spare, k, ds, rs);
    std::swap(blk[m], spare);
    copy_view<R, R>(stream, k, pcol, rowmajor<R>(Vh, pcol), rowmajor<R>(spare, pcol));
    if (!centre_left) scale_rows<R>(stream, k, pcol, spare, pcol, ds, rs);
    std::swap(blk[m + 1], spare);
    dims[m] = k;
    if (swap) std::swap(kpos[m], kpos[m + 1]);
    check("two-site update");
  }
  // inter-block gate by SWAP routing: block q travels left next to block p through two-site SWAP
  // updates, the gate is one two-site update with a diagonal phase, and the block travels back
  void gate_swap(const Layout::Gate& g, double phi) {
    const int p = g.p, q = g.q;
    move_centre(q);
    for (int m = q - 1; m > p; --m) two_site(m, true, false, 0.0, 0, 0, true);
    two_site(p, false, true, phi, kpos[p] - 1 - g.ti, kpos[p + 1] - 1 - g.tj, false);
    for (int m = p + 1; m < q; ++m) two_site(m, true, false, 0.0, 0, 0, false);
    centre = q;
    stats.gates++;
  }
  // a general two-qubit gate between blocks p < q by SWAP routing (the XY model's gates)
  void gate_general(const Layout::Gate& g, const Gate4& u) {
    const int p = g.p, q = g.q;
    move_centre(q);
    for (int m = q - 1; m > p; --m) two_site(m, true, false, 0.0, 0, 0, true);
    two_site(p, false, false, 0.0, kpos[p] - 1 - g.ti, kpos[p + 1] - 1 - g.tj, false, &u);
    for (int m = p + 1; m < q; ++m) two_site(m, true, false, 0.0, 0, 0, false);
    centre = q;
    stats.gates++;
  }
  void any_gate(const Layout::Gate& g, double phi) {
    if (swap_route) gate_swap(g, phi);
    else if (exact) gate_exact(g, phi);
    else gate(g, phi);
  }
  // ---------------------------------------------------------- centre moves (QR / LQ through the Gram)
  void move_right(int m) {  // block m becomes left-isometric, centre to m+1
    ar.off = 0;
    int l = left(m), dd = d(m), r = dims[m];
    C* G = ar.take<C>((size_t)r * r);
    C* U = ar.take<C>((size_t)r * r);
    R* w = ar.take<R>(r);
    C* T = ar.take<C>((size_t)r * r);
    void* ws = ar.take<char>(eigh_workspace_bytes(r, 1, sizeof(R)));
    const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    mm(r, r, l * dd, one, transposed<R>(blk[m], r, true), rowmajor<R>(blk[m], r), zero, rowmajor<R>(G, r));
    if (l * dd >= r) {  // QR through the Cholesky factor of the Gram: Q = M C^{-H}, R = C^H
      C* Ci = nullptr;
      if (C* Cf = try_chol(r, G, Ci)) {
        mm(l * dd, r, r, one, rowmajor<R>(blk[m], r), transposed<R>(Ci, r, true), zero, rowmajor<R>(spare, r));
        std::swap(blk[m], spare);
        const int dn = d(m + 1), rn = right(m + 1);
        mm(r, dn * rn, r, one, transposed<R>(Cf, r, true), rowmajor<R>(blk[m + 1], (long long)dn * rn), zero,
           rowmajor<R>(spare, (long long)dn * rn));
        std::swap(blk[m + 1], spare);
        stats.centre_moves++;
        check("move right");
        return;
      }
    }
    std::vector<double> hw;
    eig(r, G, w, U, ws, hw);
    int rp = std::max(1, count_above(hw, tau, std::min(r, l * dd)));
    // T = U[:, :rp] D^{-1/2};  Q = M T
    copy_view<R, R>(stream, r, rp, rowmajor<R>(U, r), rowmajor<R>(T, rp));
    scale_cols_pow<R>(stream, r, rp, T, rp, w, -1);
    mm(l * dd, rp, r, one, rowmajor<R>(blk[m], r), rowmajor<R>(T, rp), zero, rowmajor<R>(spare, rp));
    std::swap(blk[m], spare);
    // Gs = U[:, :rp] D^{1/2};  R = Gs^H;  block m+1 <- R block m+1
    copy_view<R, R>(stream, r, rp, rowmajor<R>(U, r), rowmajor<R>(T, rp));
    scale_cols_pow<R>(stream, r, rp, T, rp, w, +1);
    int dn = d(m + 1), rn = right(m + 1);
    mm(rp, dn * rn, r, one, transposed<R>(T, rp, true), rowmajor<R>(blk[m + 1], (long long)dn * rn), zero,
            rowmajor<R>(spare, (long long)dn * rn));
    std::swap(blk[m + 1], spare);
    dims[m] = rp;
    stats.centre_moves++;
    check("move right");
  }
  void move_left(int m) {  // block m becomes right-isometric, centre to m-1
    ar.off = 0;
    int l = dims[m - 1], dd = d(m), r = right(m);
    long long row = (long long)dd * r;
    C* G = ar.take<C>((size_t)l * l);
    C* U = ar.take<C>((size_t)l * l);
    R* w = ar.take<R>(l);
    C* T = ar.take<C>((size_t)l * l);
    void* ws = ar.take<char>(eigh_workspace_bytes(l, 1, sizeof(R)));
    const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    mm(l, l, (int)row, one, rowmajor<R>(blk[m], row), transposed<R>(blk[m], row, true), zero, rowmajor<R>(G, l));
    if (row >= l) {  // LQ through the Cholesky factor of the Gram: B = C Q, Q = C^{-1} B
      C* Ci = nullptr;
      if (C* Cf = try_chol(l, G, Ci)) {
        mm(l, (int)row, l, one, rowmajor<R>(Ci, l), rowmajor<R>(blk[m], row), zero, rowmajor<R>(spare, row));
        std::swap(blk[m], spare);
        const int lq = left(m - 1), dq = d(m - 1);
        mm(lq * dq, l, l, one, rowmajor<R>(blk[m - 1], l), rowmajor<R>(Cf, l), zero, rowmajor<R>(spare, l));
        std::swap(blk[m - 1], spare);
        stats.centre_moves++;
        check("move left");
        return;
      }
    }
    std::vector<double> hw;
    eig(l, G, w, U, ws, hw);
    int lp = std::max(1, count_above(hw, tau, std::min<long long>(l, row)));
    copy_view<R, R>(stream, l, lp, rowmajor<R>(U, l), rowmajor<R>(T, lp));
    scale_cols_pow<R>(stream, l, lp, T, lp, w, -1);
    mm(lp, (int)row, l, one, transposed<R>(T, lp, true), rowmajor<R>(blk[m], row), zero, rowmajor<R>(spare, row));
    std::swap(blk[m], spare);
    copy_view<R, R>(stream, l, lp, rowmajor<R>(U, l), rowmajor<R>(T, lp));
    scale_cols_pow<R>(stream, l, lp, T, lp, w, +1);
    int lq = left(m - 1), dq = d(m - 1);
    mm(lq * dq, lp, l, one, rowmajor<R>(blk[m - 1], l), rowmajor<R>(T, lp), zero, rowmajor<R>(spare, lp));
    std::swap(blk[m - 1], spare);
    dims[m - 1] = lp;
    stats.centre_moves++;
    check("move left");
  }
  void move_centre(int target) {
    while (centre < target) {
      if (exact) {
        double kept, total;
        svd_split_right(centre, 1 << 30, 0.0, kept, total);
        stats.centre_moves++;
      } else {
        move_right(centre);
      }
      ++centre;
    }
    while (centre > target) {
      if (exact) { svd_split_left(centre); stats.centre_moves++; }
      else move_left(centre);
      --centre;
    }
  }

  // ---------------------------------------------------------- truncation core
  // G: 2r x 2r left Gram, E: 2r x 2r right environment (both overwritten / read).
  // Outputs: k, WL (r2 x k), Kc (k x r2, scaled by 1/sqrt(kept)), kept, total.
  void core(int r2, int rows, int kcap, C* G, C* E, C* WL, C* Kc, int& k, double& kept, double& total,
            bool may_be_full_rank = true) {
    const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    if (may_be_full_rank && rows >= r2 && core_chol(r2, kcap, G, E, WL, Kc, k, kept, total)) return;
    C* U = ar.take<C>((size_t)r2 * r2);
    R* Dv = ar.take<R>(r2);
    C* Gs = ar.take<C>((size_t)r2 * r2);
    C* T1 = ar.take<C>((size_t)r2 * r2);
    C* H = ar.take<C>((size_t)r2 * r2);
    R* Lam = ar.take<R>(r2);
    C* V = ar.take<C>((size_t)r2 * r2);
    size_t save = ar.off;
    void* ws = ar.take<char>(eigh_workspace_bytes(r2, 1, sizeof(R)));
    if (!ws) throw Fail{MPSGB_ENOMEM, "workspace exhausted in truncation core"};
    std::vector<double> hD, hL;
    eig(r2, G, Dv, U, ws, hD);
    int rG = count_above(hD, tau, std::min(r2, rows));
    if (rG == 0) throw Fail{MPSGB_ESTATE, "zero state at a truncation"};
    copy_view<R, R>(stream, r2, rG, rowmajor<R>(U, r2), rowmajor<R>(Gs, rG));
    scale_cols_pow<R>(stream, r2, rG, Gs, rG, Dv, +1);
    gemm<R>(stream, r2, rG, r2, one, rowmajor<R>(E, r2), rowmajor<R>(Gs, rG), zero, rowmajor<R>(T1, rG));
    gemm<R>(stream, rG, rG, r2, one, transposed<R>(Gs, rG, true), rowmajor<R>(T1, rG), zero, rowmajor<R>(H, rG));
    eig(rG, H, Lam, V, ws, hL, std::max(1, std::min(kcap, rG)));  // at most kcap vectors are kept
    total = 0;
    for (double x : hL) total += std::max(x, 0.0);
    k = std::max(1, count_above(hL, tau, kcap));
    kept = 0;
    for (int i = 0; i < k; ++i) kept += std::max(hL[i], 0.0);
    if (!(kept > 0) || !(total > 0)) throw Fail{MPSGB_ESTATE, "non-positive weight at a truncation"};
    ar.off = save;
    // WL = U[:, :rG] D^{-1/2} V[:, :k]
    copy_view<R, R>(stream, r2, rG, rowmajor<R>(U, r2), rowmajor<R>(T1, rG));
    scale_cols_pow<R>(stream, r2, rG, T1, rG, Dv, -1);
    gemm<R>(stream, r2, k, rG, one, rowmajor<R>(T1, rG), rowmajor<R>(V, rG), zero, rowmajor<R>(WL, k));
    // Kc = V_k^H Gs^H / sqrt(kept)
    View<R> vkh; vkh.ptr = V; vkh.row = plain(1); vkh.col = plain(rG); vkh.conj = true;
    gemm<R>(stream, k, r2, rG, cmake<R>((R)(1.0 / std::sqrt(kept)), 0), vkh, transposed<R>(Gs, rG, true), zero,
            rowmajor<R>(Kc, r2));
  }

  // Cholesky factor of the n x n Gram G (copied, G untouched) and its inverse, from the arena: Cf
  // (lower) and Ci = Cf^{-1} (lower); nullptr if G is numerically singular (a pivot at or below
  // 32 eps G_jj), in which case the arena is left as it was.
  C* try_chol(int n, const C* G, C*& Ci) {
    const size_t save = ar.off;
    C* Cf = ar.take<C>((size_t)n * n);
    Ci = ar.take<C>((size_t)n * n);
    const size_t mark = ar.off;
    void* cws = ar.take<char>(chol_workspace_bytes(n, sizeof(R)));
    int* flag = ar.take<int>(4);
    if (!flag) throw Fail{MPSGB_ENOMEM, "workspace exhausted in the Cholesky factorisation"};
    cudaMemcpyAsync(Cf, G, sizeof(C) * (size_t)n * n, cudaMemcpyDeviceToDevice, stream);
    const double rel = 32.0 * (sizeof(R) == 8 ? 2.220446049250313e-16 : 1.1920929e-7);
    GraphScope gs(gcache);
    if (chol_inv<R>(stream, n, Cf, n, Ci, n, rel, cws, flag) != 0) throw Fail{MPSGB_EDEVICE, "Cholesky launch"};
    int hflag = 0;
    cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, stream);
    synchronize("Cholesky");
    if (hflag) {
      stats.chol_fallbacks++;
      ar.off = save;
      return nullptr;
    }
    stats.chol_ok++;
    ar.off = mark;  // keep Cf and Ci, release the scratch
    return Cf;
  }

  // Truncation core with the Cholesky factor of G (G = C C^H, Gs = C): H = C^H E C, new left
  // isometry C^{-H} V_k, carry (C V_k)^H / sqrt(kept).  Returns false, leaving G untouched, if G is
  // numerically singular (a pivot at or below 32 eps G_jj); the eigenvector factor then handles it.
  bool core_chol(int r2, int kcap, C* G, C* E, C* WL, C* Kc, int& k, double& kept, double& total) {
    const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    const size_t save = ar.off;
    C* Ci = nullptr;
    C* Cf = try_chol(r2, G, Ci);
    if (!Cf) return false;
    C* T1 = ar.take<C>((size_t)r2 * r2);
    C* H = ar.take<C>((size_t)r2 * r2);
    R* Lam = ar.take<R>(r2);
    C* V = ar.take<C>((size_t)r2 * r2);
    if (!V) throw Fail{MPSGB_ENOMEM, "workspace exhausted in truncation core"};
    gemm<R>(stream, r2, r2, r2, one, rowmajor<R>(E, r2), rowmajor<R>(Cf, r2), zero, rowmajor<R>(T1, r2));
    gemm<R>(stream, r2, r2, r2, one, transposed<R>(Cf, r2, true), rowmajor<R>(T1, r2), zero, rowmajor<R>(H, r2));
    const size_t save2 = ar.off;
    void* ws = ar.take<char>(eigh_workspace_bytes(r2, 1, sizeof(R)));
    if (!ws) throw Fail{MPSGB_ENOMEM, "workspace exhausted in truncation core"};
    std::vector<double> hL;
    eig(r2, H, Lam, V, ws, hL, std::max(1, std::min(kcap, r2)));
    ar.off = save2;
    total = 0;
    for (double x : hL) total += std::max(x, 0.0);
    k = std::max(1, count_above(hL, tau, kcap));
    kept = 0;
    for (int i = 0; i < k; ++i) kept += std::max(hL[i], 0.0);
    if (!(kept > 0) || !(total > 0)) throw Fail{MPSGB_ESTATE, "non-positive weight at a truncation"};
    // WL = C^{-H} V[:, :k]
    gemm<R>(stream, r2, k, r2, one, transposed<R>(Ci, r2, true), rowmajor<R>(V, r2), zero, rowmajor<R>(WL, k));
    // Kc = V_k^H C^H / sqrt(kept)
    View<R> vkh; vkh.ptr = V; vkh.row = plain(1); vkh.col = plain(r2); vkh.conj = true;
    gemm<R>(stream, k, r2, r2, cmake<R>((R)(1.0 / std::sqrt(kept)), 0), vkh, transposed<R>(Cf, r2, true), zero,
            rowmajor<R>(Kc, r2));
    ar.off = save;
    return true;
  }

  // ---------------------------------------------------------- inter-block gate
  void gate(const Layout::Gate& g, double phi) {
    move_centre(g.p);
    ar.off = 0;
    const int p = g.p, q = g.q;
    const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    const std::vector<int> od = dims;  // bond dims before the gate
    // ---- phase 1: right environments E00/E01 for bonds p .. q-1
    std::vector<C*> E00(L.N), E01(L.N);
    for (int m = p; m < q; ++m) {
      E00[m] = ar.take<C>((size_t)od[m] * od[m]);
      E01[m] = ar.take<C>((size_t)od[m] * od[m]);
    }
    C* X = ar.take<C>((size_t)cap);
    C* Lb = ar.take<C>((size_t)2 * cap);
    C* WL = ar.take<C>((size_t)2 * chi_eff * chi_eff);
    C* Ka = ar.take<C>((size_t)2 * chi_eff * chi_eff);
    C* Kb = ar.take<C>((size_t)2 * chi_eff * chi_eff);
    if (!Kb) throw Fail{MPSGB_ENOMEM, "workspace exhausted in gate"};
    const int lq = od[q - 1], dq = d(q), rq = right(q);
    const int bq = L.k[q] - 1 - g.tj;
    const long long inq = (1LL << bq) * rq, rowq = (long long)dq * rq;
    {
      C* Y0 = X;
      C* Y1 = X + (size_t)lq * lq;
      for (int v = 0; v < 2; ++v) {
        View<R> Bv; Bv.ptr = blk[q] + v * inq; Bv.row = plain(rowq); Bv.col = split(inq, 1, 2 * inq); Bv.conj = false;
        View<R> BvH; BvH.ptr = Bv.ptr; BvH.row = Bv.col; BvH.col = Bv.row; BvH.conj = true;
        mm(lq, lq, (int)(rowq / 2), one, Bv, BvH, zero, rowmajor<R>(v ? Y1 : Y0, lq));
      }
      C ep = cmake<R>((R)std::cos(2 * phi), (R)-std::sin(2 * phi)), em = cmake<R>((R)std::cos(2 * phi), (R)std::sin(2 * phi));
      axpby<R>(stream, lq, lq, one, rowmajor<R>(Y0, lq), one, rowmajor<R>(Y1, lq), rowmajor<R>(E00[q - 1], lq));
      axpby<R>(stream, lq, lq, ep, rowmajor<R>(Y0, lq), em, rowmajor<R>(Y1, lq), rowmajor<R>(E01[q - 1], lq));
    }
    for (int m = q - 1; m > p; --m) {  // E[m-1] = sum_s C_s E[m] C_s^H through block m
      int lm = od[m - 1], dm = d(m), rm_ = od[m];
      long long row = (long long)dm * rm_;
      for (int which = 0; which < 2; ++which) {
        C* Ein = which ? E01[m] : E00[m];
        C* Eout = which ? E01[m - 1] : E00[m - 1];
        mm(lm * dm, rm_, rm_, one, rowmajor<R>(blk[m], rm_), rowmajor<R>(Ein, rm_), zero, rowmajor<R>(X, rm_));
        mm(lm, lm, (int)row, one, rowmajor<R>(X, row), transposed<R>(blk[m], row, true), zero,
                rowmajor<R>(Eout, lm));
      }
    }
    check("gate environments");
    // ---- phase 2: truncation sweep p .. q-1
    C* carry = nullptr;
    C* nextK = Ka;
    int kprev = 0;
    for (int m = p; m < q; ++m) {
      const int r = od[m], r2 = 2 * r, dm = d(m);
      size_t mark = ar.off;
      C* G = ar.take<C>((size_t)r2 * r2);
      C* E = ar.take<C>((size_t)r2 * r2);
      int rows;
      const int bp = L.k[p] - 1 - g.ti;
      const int lp = left(p);
      const long long inp = (1LL << bp);
      if (m == p) {
        rows = lp * dm;
        set_zero<R>(stream, (long long)r2 * r2, G);
        for (int v = 0; v < 2; ++v) {
          View<R> Av; Av.ptr = blk[p] + v * inp * r; Av.row = split(inp, r, 2 * inp * r); Av.col = plain(1); Av.conj = false;
          View<R> AvH; AvH.ptr = Av.ptr; AvH.row = plain(1); AvH.col = Av.row; AvH.conj = true;
          View<R> Gv = rowmajor<R>(G + (size_t)v * r * r2 + (size_t)v * r, r2);
          mm(r, r, rows / 2, one, AvH, Av, zero, Gv);
        }
      } else {
        const int lm = od[m - 1];
        rows = kprev * dm;
        for (int kk = 0; kk < 2; ++kk) {
          View<R> Kk; Kk.ptr = carry + (size_t)kk * lm; Kk.row = plain(2LL * lm); Kk.col = plain(1); Kk.conj = false;
          View<R> Out; Out.ptr = Lb + (size_t)kk * r; Out.row = plain((long long)dm * r2); Out.col = split(r, 1, r2); Out.conj = false;
          mm(kprev, dm * r, lm, one, Kk, rowmajor<R>(blk[m], (long long)dm * r), zero, Out);
        }
        mm(r2, r2, rows, one, transposed<R>(Lb, r2, true), rowmajor<R>(Lb, r2), zero, rowmajor<R>(G, r2));
      }
      env_assemble<R>(stream, r, E00[m], E01[m], E);
      int k = 0;
      double kept = 0, total = 0;
      // G is block diagonal at m = p (two halves of rows / 2 rows each): full rank needs rows / 2 >= r
      core(r2, rows, cap_bond(m), G, E, WL, nextK, k, kept, total, m == p ? rows / 2 >= r : rows >= r2);
      // new left-isometric block m
      if (m == p) {
        for (int v = 0; v < 2; ++v) {
          View<R> Av; Av.ptr = blk[p] + v * inp * r; Av.row = split(inp, r, 2 * inp * r); Av.col = plain(1); Av.conj = false;
          View<R> Out; Out.ptr = spare + v * inp * k; Out.row = split(inp, k, 2 * inp * k); Out.col = plain(1); Out.conj = false;
          mm(rows / 2, k, r, one, Av, rowmajor<R>(WL + (size_t)v * r * k, k), zero, Out);
        }
      } else {
        mm(rows, k, r2, one, rowmajor<R>(Lb, r2), rowmajor<R>(WL, k), zero, rowmajor<R>(spare, k));
      }
      std::swap(blk[m], spare);
      dims[m] = k;
      double f = kept / total;
      F *= f;
      last_f_min = std::min(last_f_min, f);
      stats.truncations++;
      carry = nextK;
      nextK = (nextK == Ka) ? Kb : Ka;
      kprev = k;
      ar.off = mark;
      check("truncation");
    }
    // ---- new centre block q = sum_v M_w B_w with M_w = e^{-i phi z_w} K0 + e^{i phi z_w} K1
    C* Mw = X;
    for (int w = 0; w < 2; ++w) {
      double z = 1 - 2 * w;
      C a = cmake<R>((R)std::cos(phi * z), (R)-std::sin(phi * z)), b = cmake<R>((R)std::cos(phi * z), (R)std::sin(phi * z));
      View<R> K0; K0.ptr = carry; K0.row = plain(2LL * lq); K0.col = plain(1); K0.conj = false;
      View<R> K1 = K0; K1.ptr = carry + lq;
      axpby<R>(stream, kprev, lq, a, K0, b, K1, rowmajor<R>(Mw, lq));
      View<R> Bw; Bw.ptr = blk[q] + w * inq; Bw.row = plain(rowq); Bw.col = split(inq, 1, 2 * inq); Bw.conj = false;
      View<R> Out; Out.ptr = spare + w * inq; Out.row = plain(rowq); Out.col = split(inq, 1, 2 * inq); Out.conj = false;
      mm(kprev, (int)(rowq / 2), lq, one, rowmajor<R>(Mw, lq), Bw, zero, Out);
    }
    std::swap(blk[q], spare);
    centre = q;
    stats.gates++;
    check("gate");
  }

  // ---------------------------------------------------------- whole-chain re-compression
  int truncate(int chi) override {
    if (chi < 1 || chi > cfg.chi_max) throw Fail{MPSGB_EINVAL, "truncate: chi out of range"};
    move_centre(L.N - 1);
    move_centre(0);  // everything right of block 0 is right-isometric
    if (exact) {
      for (int m = 0; m < L.N - 1; ++m) {
        const int r = dims[m];
        double kept = 0, total = 0;
        const int k = svd_split_right(m, std::min(chi, cap_bond(m)), -0.5, kept, total);
        F *= kept / total;
        if (k < r) stats.truncations++;
        centre = m + 1;
      }
      return MPSGB_OK;
    }
    for (int m = 0; m < L.N - 1; ++m) {
      ar.off = 0;
      int l = left(m), dd = d(m), r = dims[m];
      C* G = ar.take<C>((size_t)r * r);
      C* U = ar.take<C>((size_t)r * r);
      R* w = ar.take<R>(r);
      C* T = ar.take<C>((size_t)r * r);
      void* ws = ar.take<char>(eigh_workspace_bytes(r, 1, sizeof(R)));
      const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
      mm(r, r, l * dd, one, transposed<R>(blk[m], r, true), rowmajor<R>(blk[m], r), zero, rowmajor<R>(G, r));
      std::vector<double> hw;
      eig(r, G, w, U, ws, hw);
      int kp = std::max(1, count_above(hw, tau, std::min(std::min(r, l * dd), chi)));
      double tot = 0, kept = 0;
      for (int i = 0; i < (int)hw.size(); ++i) { tot += std::max(hw[i], 0.0); if (i < kp) kept += std::max(hw[i], 0.0); }
      copy_view<R, R>(stream, r, kp, rowmajor<R>(U, r), rowmajor<R>(T, kp));
      scale_cols_pow<R>(stream, r, kp, T, kp, w, -1);
      mm(l * dd, kp, r, one, rowmajor<R>(blk[m], r), rowmajor<R>(T, kp), zero, rowmajor<R>(spare, kp));
      std::swap(blk[m], spare);
      copy_view<R, R>(stream, r, kp, rowmajor<R>(U, r), rowmajor<R>(T, kp));
      scale_cols_pow<R>(stream, r, kp, T, kp, w, +1);
      int dn = d(m + 1), rn = right(m + 1);
      mm(kp, dn * rn, r, cmake<R>((R)(1.0 / std::sqrt(kept)), 0), transposed<R>(T, kp, true),
              rowmajor<R>(blk[m + 1], (long long)dn * rn), zero, rowmajor<R>(spare, (long long)dn * rn));
      std::swap(blk[m + 1], spare);
      dims[m] = kp;
      double f = kept / tot;
      F *= f;
      if (kp < r) stats.truncations++;
      centre = m + 1;
      check("truncate");
    }
    return MPSGB_OK;
  }

  // ---------------------------------------------------------- observables (left-to-right environment sweep)
  int observables(double out[4]) override {
    ar.off = 0;
    const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    C* Y[4];
    for (int i = 0; i < 4; ++i) Y[i] = ar.take<C>((size_t)cap);
    C* Ecur[4];
    C* Enew[4];
    long long c2 = (long long)chi_eff * chi_eff;
    for (int i = 0; i < 4; ++i) { Ecur[i] = ar.take<C>(c2); Enew[i] = ar.take<C>(c2); }
    if (!Enew[3]) throw Fail{MPSGB_ENOMEM, "workspace exhausted in observables"};
    // L0 = [1], L1 = L2 = LX = [0]
    set_identity<R>(stream, 1, Ecur[0], 1);
    for (int i = 1; i < 4; ++i) set_zero<R>(stream, 1, Ecur[i]);
    for (int b = 0; b < L.N; ++b) {
      int l = left(b), dd = d(b), r = right(b);
      long long row = (long long)dd * r;
      for (int i = 0; i < 4; ++i)
        mm(l, (int)row, l, one, rowmajor<R>(Ecur[i], l), rowmajor<R>(blk[b], row), zero, rowmajor<R>(Y[i], row));
      // Y2 <- Y2 + 2 m Y1 + m^2 Y0 ; Y1 <- Y1 + m Y0 ; YX <- YX + X(Y0)
      weighted_phys<R>(stream, 1, l, dd, r, Y[2], Y[1], Y[2], 2.0);
      weighted_phys<R>(stream, 2, l, dd, r, Y[2], Y[0], Y[2], 1.0);
      weighted_phys<R>(stream, 1, l, dd, r, Y[1], Y[0], Y[1], 1.0);
      weighted_phys<R>(stream, 3, l, dd, r, Y[3], Y[0], Y[3], 1.0);
      for (int i = 0; i < 4; ++i)
        mm(r, r, l * dd, one, transposed<R>(blk[b], r, true), rowmajor<R>(Y[i], r), zero, rowmajor<R>(Enew[i], r));
      for (int i = 0; i < 4; ++i) std::swap(Ecur[i], Enew[i]);
    }
    C h[4];
    for (int i = 0; i < 4; ++i) cudaMemcpyAsync(&h[i], Ecur[i], sizeof(C), cudaMemcpyDeviceToHost, stream);
    synchronize("observables");
    if (tc) check_device_error();
    double norm = h[0].x, n = L.n;
    out[0] = h[1].x / (n * norm);
    out[1] = h[2].x / (n * n * norm);
    out[2] = h[3].x / (n * norm);
    out[3] = norm;
    return MPSGB_OK;
  }

  // <X_stag^2> = (1/n^2) <(sum_j s_j X_j)^2> by the same left-to-right sweep with three
  // environments: norm, first moment (sum over the blocks so far of O_b) and second moment, where
  // O_b = sum_{j in b} s_j X_j; per block Y2 <- Y2 + 2 O(Y1) + O(O(Y0)), Y1 <- Y1 + O(Y0)
  int x_stag2(double* out) override {
    ar.off = 0;
    const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    C* Y[3];
    for (int i = 0; i < 3; ++i) Y[i] = ar.take<C>((size_t)cap);
    C* T = ar.take<C>((size_t)cap);
    C* Ecur[3];
    C* Enew[3];
    long long c2 = (long long)chi_eff * chi_eff;
    for (int i = 0; i < 3; ++i) { Ecur[i] = ar.take<C>(c2); Enew[i] = ar.take<C>(c2); }
    if (!Enew[2]) throw Fail{MPSGB_ENOMEM, "workspace exhausted in observables"};
    set_identity<R>(stream, 1, Ecur[0], 1);
    for (int i = 1; i < 3; ++i) set_zero<R>(stream, 1, Ecur[i]);
    for (int b = 0; b < L.N; ++b) {
      const int l = left(b), dd = d(b), r = right(b), k = L.k[b];
      long long row = (long long)dd * r;
      int neg = 0;
      for (int t = 0; t < k; ++t)
        if (L.stag[L.qubits[b][t]] < 0) neg |= 1 << (k - 1 - t);
      for (int i = 0; i < 3; ++i)
        mm(l, (int)row, l, one, rowmajor<R>(Ecur[i], l), rowmajor<R>(blk[b], row), zero, rowmajor<R>(Y[i], row));
      stag_x<R>(stream, 1, l, dd, r, Y[2], Y[1], Y[2], 2.0, neg);
      stag_x<R>(stream, 1, l, dd, r, nullptr, Y[0], T, 1.0, neg);
      stag_x<R>(stream, 1, l, dd, r, Y[2], T, Y[2], 1.0, neg);
      stag_x<R>(stream, 0, l, dd, r, Y[1], T, Y[1], 1.0, 0);
      for (int i = 0; i < 3; ++i)
        mm(r, r, l * dd, one, transposed<R>(blk[b], r, true), rowmajor<R>(Y[i], r), zero, rowmajor<R>(Enew[i], r));
      for (int i = 0; i < 3; ++i) std::swap(Ecur[i], Enew[i]);
    }
    C h[3];
    for (int i = 0; i < 3; ++i) cudaMemcpyAsync(&h[i], Ecur[i], sizeof(C), cudaMemcpyDeviceToHost, stream);
    synchronize("observables");
    if (tc) check_device_error();
    const double n = L.n;
    *out = h[2].x / (n * n * h[0].x);
    return MPSGB_OK;
  }

  int singular_values(int bond, std::vector<double>& s) override {
    if (bond < 0 || bond >= L.N - 1) throw Fail{MPSGB_EINVAL, "bond out of range"};
    move_centre(bond);
    if (exact) {
      ar.off = 0;
      const int l = left(bond), dd = d(bond), r = dims[bond];
      const long long M = (long long)l * dd;
      C* Xt = ar.take<C>((size_t)M * r);
      if (!Xt) throw Fail{MPSGB_ENOMEM, "workspace exhausted in the SVD"};
      copy_view<R, R>(stream, r, (int)M, transposed<R>(blk[bond], r, true), rowmajor<R>(Xt, M));
      C *Vh, *U;
      double* ds;
      jsvd(Xt, r, (int)M, Vh, U, ds, s);
      return MPSGB_OK;
    }
    ar.off = 0;
    int l = left(bond), dd = d(bond), r = dims[bond];
    C* G = ar.take<C>((size_t)r * r);
    C* U = ar.take<C>((size_t)r * r);
    R* w = ar.take<R>(r);
    void* ws = ar.take<char>(eigh_workspace_bytes(r, 1, sizeof(R)));
    const C one = cmake<R>(1, 0), zero = cmake<R>(0, 0);
    mm(r, r, l * dd, one, transposed<R>(blk[bond], r, true), rowmajor<R>(blk[bond], r), zero, rowmajor<R>(G, r));
    std::vector<double> hw;
    eig(r, G, w, U, ws, hw);
    s.resize(hw.size());
    for (size_t i = 0; i < hw.size(); ++i) s[i] = std::sqrt(std::max(hw[i], 0.0));
    return MPSGB_OK;
  }

  // ---------------------------------------------------------- checkpoints
  int save(const char* path) override {
    FILE* fh = std::fopen(path, "wb");
    if (!fh) throw Fail{MPSGB_EINVAL, std::string("cannot open ") + path};
    const char magic[8] = {'M', 'P', 'S', 'G', 'B', 'v', '2', 0};
    int hdr[4] = {(int)sizeof(R), L.N, centre, 0};
    long long st5[5] = {stats.truncations, stats.gates, stats.centre_moves, stats.eig_calls, stats.eig_sweeps};
    bool ok = std::fwrite(magic, 1, 8, fh) == 8 && std::fwrite(&cfg, sizeof(cfg), 1, fh) == 1 &&
              std::fwrite(hdr, sizeof(int), 4, fh) == 4 && std::fwrite(&F, sizeof(double), 1, fh) == 1 &&
              std::fwrite(st5, sizeof(long long), 5, fh) == 5 &&
              std::fwrite(dims.data(), sizeof(int), dims.size(), fh) == dims.size();
    std::vector<C> h;
    for (int b = 0; ok && b < L.N; ++b) {
      size_t cnt = (size_t)left(b) * d(b) * right(b);
      h.resize(cnt);
      cudaMemcpyAsync(h.data(), blk[b], sizeof(C) * cnt, cudaMemcpyDeviceToHost, stream);
      synchronize("save");
      ok = std::fwrite(h.data(), sizeof(C), cnt, fh) == cnt;
    }
    ok = (std::fclose(fh) == 0) && ok;
    if (!ok) throw Fail{MPSGB_EINVAL, std::string("write failed: ") + path};
    return MPSGB_OK;
  }
  int load_blocks(FILE* fh) override {
    int hdr[4];
    long long st5[5];
    bool ok = std::fread(hdr, sizeof(int), 4, fh) == 4 && hdr[0] == (int)sizeof(R) && hdr[1] == L.N &&
              std::fread(&F, sizeof(double), 1, fh) == 1 && std::fread(st5, sizeof(long long), 5, fh) == 5 &&
              std::fread(dims.data(), sizeof(int), dims.size(), fh) == dims.size();
    if (!ok) throw Fail{MPSGB_EINVAL, "checkpoint header does not match its config"};
    for (int m = 0; m < L.N - 1; ++m)
      if (dims[m] < 1 || dims[m] > cap_bond(m)) throw Fail{MPSGB_EINVAL, "checkpoint bond dimension out of range"};
    centre = hdr[2];
    stats.truncations = st5[0]; stats.gates = st5[1]; stats.centre_moves = st5[2]; stats.eig_calls = st5[3]; stats.eig_sweeps = st5[4];
    std::vector<C> h;
    for (int b = 0; b < L.N; ++b) {
      size_t cnt = (size_t)left(b) * d(b) * right(b);
      h.resize(cnt);
      if (std::fread(h.data(), sizeof(C), cnt, fh) != cnt) throw Fail{MPSGB_EINVAL, "checkpoint truncated"};
      cudaMemcpyAsync(blk[b], h.data(), sizeof(C) * cnt, cudaMemcpyHostToDevice, stream);
    }
    synchronize("load");
    return MPSGB_OK;
  }
  int sync() override {
    synchronize("sync");
    return MPSGB_OK;
  }
};

Engine* make_engine(const mpsgb_config& cfg, const mpsgb_allocator* alloc, cudaStream_t st, std::string& err, int& status) {
  Engine* e = nullptr;
  try {
    if (cfg.prec == MPSGB_FP64) {
      auto* x = new EngineT<double>();
      e = x;
      x->exact = true;
      x->init(cfg, alloc, st);
    } else if (cfg.prec == MPSGB_FP32 || cfg.prec == MPSGB_SPLIT_BF16X3 || cfg.prec == MPSGB_SPLIT_TF32X3) {
      auto* x = new EngineT<float>();
      e = x;
      x->tc = cfg.prec == MPSGB_SPLIT_BF16X3 || cfg.prec == MPSGB_SPLIT_TF32X3;
      x->tc_tf32 = cfg.prec == MPSGB_SPLIT_TF32X3;
      x->init(cfg, alloc, st);
    } else {
      throw Fail{MPSGB_EINVAL, "precision not available in this build"};
    }
    status = MPSGB_OK;
    return e;
  } catch (const Fail& f) {
    delete e;
    err = f.msg;
    status = f.status;
    return nullptr;
  }
}

}  // namespace mpsgb
