// Internal declarations of the GB300 library behind include/maxwell4.h.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/maxwell4.h"

namespace ms {

enum Bc { DIR = 0, NEU = 1 };
enum PadeKind { HALF_TO_NODE = 0, NODE_TO_HALF = 1 };
enum Field { EZ = 0, HX = 1, HY = 2 };

// Shape of one 2D TM_z component in the full staggered layout (rows = y, cols = x).
struct Shape {
  int nx, ny, bcx, bcy;
  size_t size() const { return (size_t)nx * ny; }
};
Shape field_shape(int N, int f);

// Explicit banded form of the Pade derivative W = A^{-1} D1~ of one line type (App. A.1,
// Eq. "eq:lhs"), D1~ the plain two-point difference (M x (M+1)), so that delta f = (1/h) W f.
// Output i uses inputs i-K .. i+K+1.  Rows [0, B) and [M-B, M) are stored explicitly, the
// remaining rows share one Toeplitz row.  Each stored row has 2K+2 weights.
struct PadeTable {
  int M = 0, K = 0, B = 0;
  bool all_explicit = false;        // every row stored (short lines)
  // Generic band form used by the FP64 kernel: `rows` outputs from `n_in` inputs, output i
  // reading inputs i - left .. i - left + 2K + 1.  Forward tables: rows = M, n_in = M + 1,
  // left = K.  Transposed tables (W^T, the reverse pass): rows = M + 1, n_in = M, left = K + 1.
  int rows = 0, n_in = 0, left = 0;
  std::vector<double> w;             // (2B + 1) rows x (2K + 2)
  double* d_w = nullptr;             // device copy (FP64)
  float* d_whi = nullptr;            // device FP32 split: w = whi + wlo exactly to ~2^-48
  float* d_wlo = nullptr;
  int row_stride() const { return 2 * K + 2; }
};
// Build the table for M outputs, closure, kind; tail weights dropped sum below tol * row sum.
int build_pade_table(int M, int closure, int kind, double tol, PadeTable* t, std::string* err,
                     bool of_differences = false);
// Transpose W^T of a forward FP64 table, as the same truncated band: exact transpose of the
// operator the forward kernels apply.
void build_pade_table_T(const PadeTable& fwd, PadeTable* t);
// Exact (untruncated) dense row i of W, for checks.
void pade_dense_row(int M, int closure, int kind, int i, std::vector<double>* row);

// Largest stable CFL number of the 2D scheme from its Fourier symbol (Sec. 4 recurrence).
double stability_limit_2d();

struct Graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int steps = 0;
};

// Kernel kinds reported by ms_step_profiled.
enum KernelKind {
  KK_FILTER64 = 0, KK_PADE64 = 1, KK_P1SWEEP64 = 2, KK_YEE64 = 3, KK_CURL32 = 4, KK_SOLVE32 = 5,
  KK_FILTER3D64 = 6, KK_PADE3D64 = 7, KK_SWEEP3D64 = 8, KK_FILT3D32 = 9, KK_BAND3D32 = 10, KK_SWEEP3D32 = 11,
  KK_NC64 = 12, KK_SRC = 13, KK_TERM3D32 = 14, KK_TSGEMM = 15, KK_TSPACK = 16, KK_TRACKED32 = 17,
  KK_COUNT
};
const char* kernel_kind_name(int k);

// Per-launch event marks of a profiled step.
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> kinds;
  std::vector<double> bytes;  // algorithmic bytes of each launch
  size_t next = 0;
};

}  // namespace ms

struct ms_grid;
namespace ms {
struct Grid3D;  // six-component state of a 3D grid (grid3d.cu)
struct Src3;    // current sources of a 3D grid (k_src3.cu)
struct Adj32;   // FP32 reverse pass of an FP32_REFINED grid (adjoint32.cu)
// Record an event after a launch of the given kind when the grid is being profiled.
void prof_mark(ms_grid* g, int kind, double bytes = 0.0);
// Set the message returned by ms_last_error on this thread.
void set_last_error(const char* msg);
// Every device allocation and release of the library goes through these two (capi.cu), so a test
// can make the n-th allocation fail on the host (ms_debug_fail_alloc) and count what is held.
cudaError_t dev_malloc(void** p, size_t bytes);
void dev_free(void* p);
template <typename T>
cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}
}  // namespace ms

struct ms_grid {
  ms_grid_desc desc{};
  int N = 0;
  double h = 0, ht = 0, kappa2 = 0, beta = 0, c1 = 0, Z = 1;
  long step = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  ms::Shape sh[3];

  // Pade tables: [0] half->node (M = N-1), [1] node->half (M = N)
  ms::PadeTable pade[2];
  int p1_sweeps = 0;  // Richardson sweeps for the FP64 solve
  // FP32 path: tables truncated for FP32 and split hi/lo; Richardson sweeps for FP32
  ms::PadeTable pade32[2];
  int p1_sweeps32 = 0;

  // FP64 state and scratch
  double* f64[3] = {nullptr, nullptr, nullptr};   // E_z, H_x, H_y
  double* de64 = nullptr;                          // tracked Delta E_z (MS_SCHEME_C4_DE)
  float* de_hi = nullptr;                          // the same in MS_FP32_REFINED (float-float)
  float* de_lo = nullptr;
  float* t32[8] = {};                              // its scratch: E^n, y_x, y_y, G~_E (hi, lo each)
  double* s64[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool shared64 = false;  // s64 planes belong to a batch
  // FP32 hi/lo state (MS_FP32_REFINED)
  float* hi[3] = {nullptr, nullptr, nullptr};
  float* lo[3] = {nullptr, nullptr, nullptr};
  float* s32[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};

  // reductions and diagnostics
  double* d_partial = nullptr;  // per-block partial sums
  double* d_result = nullptr;   // final reduction results
  int partial_cap = 0;
  double* d_modetab = nullptr;  // 1D mode tables for exact fields
  size_t modetab_cap = 0;

  ms::Graph graph1, graphk;
  int launches_per_step = 0;

  // reverse pass (adjoint.cu): transposed FP64 Pade tables, adjoint state and scratch, graphs
  ms::PadeTable padeT[2];
  double* adj[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  ms::Graph adj_graph1, adj_graphk;
  int adj_precision = -1;     // arithmetic of the reverse pass (MS_FP64 / MS_FP32_REFINED); -1: the grid's
  ms::Adj32* adj32 = nullptr;  // FP32 reverse pass state (adjoint32.cu)

  // current sources (k_src.cu): per-source constants, sine/cosine tables, device step index
  int nsrc = 0;
  int src_wall = 0;  // some source has a cosine profile (nonzero on a wall)
  void* d_src = nullptr;
  double* d_srctab = nullptr;
  float* d_srctab32 = nullptr;  // float copy of the tables (FP32_REFINED right-hand sides)
  void* d_srcfac = nullptr;     // time factors of the current step (k_src_time)
  double* d_walldata = nullptr;  // FP32 wall terms: wall data of the current step (k_wall_data)
  float* d_wresp = nullptr;      // FP32 wall terms: Pade responses to the end values of a line
  long* d_step = nullptr;

  // 3D grids (desc.dim == 3): components, scratch and kernels live in grid3d.cu
  ms::Grid3D* g3 = nullptr;
  ms::Src3* src3 = nullptr;  // 3D current sources (k_src3.cu), or none
  ms::Prof prof;
};
