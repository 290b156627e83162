// Host-side engine of one grouped-qubit MPS (one handle of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/mpsgb.h"
#include "common.cuh"

namespace mpsgb {

// Error carried from the engine to the C ABI, which turns it into a status code.
struct Fail {
  int status;
  std::string msg;
};

// MPS layout of a lattice: row-grouped snake of an Lx x Ly periodic grid (Sec. III, Fig.
// mps_drawing), or one qubit per site along the 3D snake of an open Lx x Ly x Lz grid (the
// Supplemental Material's 3D TFIM section, Fig. 3D_snake).
struct Layout {
  struct Gate {
    int p, q, qi, qj, ti, tj;  // block positions p < q, global qubits, bit positions (0 = MSB)
    int set = -1;              // bond set A..D (0..3) of the XY model's Trotter step, -1 elsewhere
  };
  int Lx = 0, Ly = 0, Lz = 1, N = 0, n = 0;
  std::vector<int> stag;                               // staggered sign s_j (+1 / -1) per global qubit
  std::vector<int> k;                                  // qubits per block
  std::vector<std::vector<int>> qubits;                // global qubit ids per block, MSB first
  std::vector<std::vector<std::pair<int, int>>> intra; // in-block ZZ pairs (bit positions)
  std::vector<Gate> inter;                             // inter-block gates in application order
  std::vector<double> bound;                           // exact bond-dimension bound per bond
};
bool make_layout(int Lx, int Ly, Layout& out, std::string& err);
bool make_layout(const mpsgb_config& cfg, Layout& out, std::string& err);

struct Stats {
  long long truncations = 0;     // bond truncations (one per spanned bond of an inter-block gate)
  long long gates = 0;           // inter-block gates applied
  long long centre_moves = 0;
  long long eig_calls = 0;
  long long eig_sweeps = 0;
  long long chol_ok = 0;         // Gram matrices factorised by Cholesky
  long long chol_fallbacks = 0;  // ... that were too close to singular (eigenvector factor taken instead)
};

class Engine {
 public:
  virtual ~Engine() {}
  virtual int apply_x(double alpha) = 0;                       // prod_j exp(-i alpha X_j)
  virtual int apply_zz(double phi) = 0;                        // prod_<ij> exp(-i phi Z_i Z_j) with truncation
  virtual int step(double J, double h, double dt, int order, int nsteps) = 0;
  virtual int apply_gates(int first, int count, double phi) = 0;  // inter-block gates [first, first+count)
  virtual int truncate(int chi) = 0;
  virtual int observables(double out[4]) = 0;                  // <Z_tot>, <Z_tot^2>, <X_tot>, norm^2
  virtual int singular_values(int bond, std::vector<double>& s) = 0;
  virtual int save(const char* path) = 0;
  virtual int load_blocks(FILE* fh) = 0;
  virtual int sync() = 0;
  virtual int apply_zstag(double alpha) = 0;                   // prod_j exp(-i alpha s_j Z_j)
  virtual int x_stag2(double* out) = 0;                        // <X_stag^2> (Eq. xy_signal)
  double F = 1.0;                     // F_MPS: product of all truncation fidelities
  double last_f_min = 1.0;            // smallest truncation fidelity of the last layer
  Stats stats;
  Layout L;
  mpsgb_config cfg;
  std::vector<int> dims;              // bond dimensions, size N-1
  int centre = 0;
  cudaStream_t stream = nullptr;
};

Engine* make_engine(const mpsgb_config& cfg, const mpsgb_allocator* alloc, cudaStream_t st, std::string& err, int& status);

}  // namespace mpsgb
