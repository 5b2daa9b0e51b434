// Device helpers and launcher declarations shared by the kernels of the library.
#pragma once

#include "ms_internal.h"

namespace ms {

// Interior test on one axis: Dirichlet axes (nodes 0..n-1 with n-1 = N) exclude both ends.
__host__ __device__ __forceinline__ bool interior(int bc, int i, int n) {
  return bc == NEU ? true : (i > 0 && i < n - 1);
}

// Even ghost reflection (u(-1) = u(0), u(n) = u(n-1)); a no-op for in-range indices.
__host__ __device__ __forceinline__ int clampi(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

// Row i of a Pade table (layout of PadeTable).
template <typename T>
__host__ __device__ __forceinline__ const T* pade_row_ptr(const T* tab, int i, int M, int K, int B, int all_explicit) {
  const int rs = 2 * K + 2;
  if (all_explicit) return tab + (size_t)i * rs;
  if (i < B) return tab + (size_t)i * rs;
  if (i >= M - B) return tab + (size_t)(B + i - (M - B)) * rs;
  return tab + (size_t)(2 * B) * rs;
}

void launch_filter64(const double* u, double* G, const Shape& s, double beta, cudaStream_t st);
void launch_pade64(int axis, const double* in, double* out, int n_lines, int in_ld, int out_len, int out_ld,
                   int out_off, int line_lo, int line_hi, const PadeTable& t, double scale, int accumulate,
                   cudaStream_t st);
void launch_p1_sweep64(const double* b, const double* xin, double* xout, const Shape& s, double c1h2, double omega,
                       double bscale, int first, double* upd, double upd_scale, cudaStream_t st);
void launch_p1_apply64(const double* x, double* out, const Shape& s, double c1h2, double out_scale, cudaStream_t st);
void launch_yee_e64(double* ez, const double* hx, const double* hy, int N, double c_e, cudaStream_t st);
void launch_yee_h64(const double* ez, double* hx, double* hy, int N, double c_h, cudaStream_t st);
// Tracked-Delta-E variant (k_tracked.cu): DE += kappa^2 h_tau E* - (24/h_tau) c / kappa^2 with
// c = kappa^2 Z curl_h H, then G_E = beta E + (h^2/12) DE; and DE = Delta_h E for initial data.
void launch_de_update64(double* de, const double* es, const double* c, const double* e, double* ge, int N, double ht,
                        double k2, double beta, double h, cudaStream_t st);
void launch_lap_e64(const double* e, double* de, int N, double h, cudaStream_t st);
// Current sources (k_src.cu): host tables and constants; launches that add P(J) to an E right-hand
// side and curl d_t J to the H right-hand sides (scaled by `scale`), and the device step tick.
// J_z = amp X(pi m x) Y(pi n y) sin(omega t), X = sin (px = 0) or cos (px = 1), Y likewise by py.
struct SrcSpec {
  int m, n, px, py;
  double amp, omega;
};
int build_sources(ms_grid* g, const SrcSpec* src, int nsrc, std::vector<unsigned char>* dev_blob,
                  std::vector<double>* tabs);
// The time factors of a step (first source launch of the step; FP32 factors in the units of the tile
// solve, scale_e for E and scale_h for H), then the point kernels that read them.
size_t src_factor_bytes();
void launch_src_time(ms_grid* g, double scale_e, double scale_h);
void launch_src_e64(ms_grid* g, double* R);
void launch_src_h64(ms_grid* g, double* Rx, double* Ry);
void launch_src_e32(ms_grid* g, float* R, double scale_e);
void launch_src_h32(ms_grid* g, float* Rx, float* Ry, double scale_h);
// FP32 wall terms: the wall data of a step (launched after launch_src_time) and, on the host, the
// Pade responses to the end values of a line.
void launch_wall_data(ms_grid* g);
size_t wall_data_doubles(int N);
void wall_responses(int N, std::vector<float>* wr);
void launch_tick(ms_grid* g);
// Boundary data of sources that do not vanish on the walls (FP64 step): the H-filter ghosts of
// Step 1, G_E on the boundary nodes, and the ghost part of P1 in the H right-hand sides of Step 2.
void launch_wall_hfilter64(ms_grid* g, double* Gx, double* Gy);
void launch_wall_ge64(ms_grid* g, double* GE);
void launch_wall_hsolve64(ms_grid* g, double* Rx, double* Ry);
// Non-compact fourth-order comparator NC (k_nc.cu)
void launch_nc_e64(double* ez, const double* hx, const double* hy, int N, double c_e, cudaStream_t st);
void launch_nc_h64(const double* ez, double* hx, double* hy, int N, double c_h, cudaStream_t st);

// x = P1^{-1} b for field f by the FP64 Richardson sweeps (scratch planes s64[3], s64[4]); the
// last sweep writes `out` and, when upd != nullptr, adds upd_scale * x to upd (capi.cu).
void p1_solve64(ms_grid* g, int f, const double* b, double* out, double* upd, double upd_scale, int* nl);
// Reverse pass (adjoint.cu): releases the transposed tables, adjoint planes and graphs.
void adjoint_teardown(ms_grid* g);

// Diagnostics (k_diag.cu)
void launch_mode_field(double* out, const Shape& s, const double* tab_x, const double* tab_y, const double* coef,
                       int nmodes, cudaStream_t st);
// Reductions over n points: results[0..3] = sum (a-b)^2, sum b^2, max |a-b|, sum |a-b| (accumulated
// over calls when accumulate != 0).  partial must hold 4 * blocks doubles.
void launch_err_reduce(const double* a, const double* b, size_t n, double* partial, int blocks, double* results,
                       int accumulate, cudaStream_t st);
// results[slot] (+)= sum a*b
void launch_dot(const double* a, const double* b, size_t n, double* partial, int blocks, double* results, int slot,
                int accumulate, cudaStream_t st);
// FP32 hi/lo <-> FP64 conversion
void launch_split(const double* v, float* hi, float* lo, size_t n, cudaStream_t st);
void launch_join(const float* hi, const float* lo, double* v, size_t n, cudaStream_t st);
void launch_zero_dirichlet64(double* u, const Shape& s, cudaStream_t st);
int reduce_blocks(size_t n);

}  // namespace ms
