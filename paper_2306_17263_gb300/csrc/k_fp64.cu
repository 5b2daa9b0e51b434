// FP64 kernels of the compact scheme (MS_FP64): one operator per launch.
//
// GB300 runs FP64 at about 1/60 of its FP32 rate, so this path is bound by the FP64 pipe,
// not by HBM; it exists as the full-precision form of the step.  Every kernel is an
// independent-output stencil over a 2D field with coalesced x-fastest access.
#include "k_fp64.cuh"

namespace ms {

// ---------------------------------------------------------------------------------------
// Right-hand-side filter of Eq. "eq:ell": G = beta u + (1/12) L u with L = h^2 Delta_h,
// Dirichlet boundary points (stored zeros) and even Neumann ghosts (index clamping,
// Corollary "cor:ghost_cor").  G = 0 on Dirichlet boundary points.
__global__ void k_filter64(const double* __restrict__ u, double* __restrict__ G, int nx, int ny, int bcx, int bcy,
                           double beta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const size_t p = (size_t)j * nx + i;
  if (!interior(bcx, i, nx) || !interior(bcy, j, ny)) {
    G[p] = 0.0;
    return;
  }
  const int im = clampi(i - 1, nx), ip = clampi(i + 1, nx), jm = clampi(j - 1, ny), jp = clampi(j + 1, ny);
  const double c = u[p];
  const double lap = u[(size_t)j * nx + im] + u[(size_t)j * nx + ip] + u[(size_t)jm * nx + i] +
                     u[(size_t)jp * nx + i] - 4.0 * c;
  G[p] = beta * c + lap * (1.0 / 12.0);
}

// ---------------------------------------------------------------------------------------
// Pade derivative (App. A.1, delta = A^{-1} D1) applied as the explicit band of W = A^{-1} D1~
// (or of its transpose W^T in the reverse pass):
//   out[line, o] (+)= scale * sum_{t} W(i, t) in[line, i - left + t],  o = i + out_off,
// for the M output rows i of the table and inputs 0 .. n_in - 1.
// AXIS 0: lines are rows (x contiguous); AXIS 1: lines are columns.  Every point of the
// output array is written: outputs outside [out_off, out_off + M) or lines outside
// [line_lo, line_hi) receive 0 (or are left unchanged when accumulating).
template <int AXIS>
__global__ void k_pade64(const double* __restrict__ in, double* __restrict__ out, int n_lines, int M, int in_ld,
                         int out_len, int out_ld, int out_off, int line_lo, int line_hi, const double* __restrict__ tab,
                         int K, int B, int all_explicit, double scale, int accumulate, int n_in, int left) {
  int o, line;
  if (AXIS == 0) {
    o = blockIdx.x * blockDim.x + threadIdx.x;
    line = blockIdx.y * blockDim.y + threadIdx.y;
  } else {
    line = blockIdx.x * blockDim.x + threadIdx.x;
    o = blockIdx.y * blockDim.y + threadIdx.y;
  }
  if (o >= out_len || line >= n_lines) return;
  const size_t po = (AXIS == 0) ? (size_t)line * out_ld + o : (size_t)o * out_ld + line;
  const int i = o - out_off;
  double v = 0.0;
  if (i >= 0 && i < M && line >= line_lo && line < line_hi) {
    const double* w = pade_row_ptr(tab, i, M, K, B, all_explicit);
    const int k0 = i - left;
    for (int t = 0; t < 2 * K + 2; ++t) {
      const int k = k0 + t;
      if (k < 0 || k >= n_in) continue;
      const double f = (AXIS == 0) ? in[(size_t)line * in_ld + k] : in[(size_t)k * in_ld + line];
      v = fma(w[t], f, v);
    }
    v *= scale;
  }
  if (accumulate) out[po] += v;
  else out[po] = v;
}

// ---------------------------------------------------------------------------------------
// One Richardson sweep for P~ x = b~, P~ = h^2 P1 = c1h2 - Lx - Ly - (1/6) Lx Ly (Def.
// "def:operatorsP" with L = h^2 D_2 per axis, Dirichlet zeros and even Neumann ghosts):
//   x_out = x_in + omega (bscale * b - P~ x_in),  omega = 2 / (lambda_min + lambda_max).
// first != 0: x_in is taken as 0 (x_in not read).  upd != nullptr: upd += upd_scale * x_out.
__global__ void k_p1_sweep64(const double* __restrict__ b, const double* __restrict__ xin, double* __restrict__ xout,
                             int nx, int ny, int bcx, int bcy, double c1h2, double omega, double bscale, int first,
                             double* __restrict__ upd, double upd_scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const size_t p = (size_t)j * nx + i;
  if (!interior(bcx, i, nx) || !interior(bcy, j, ny)) {
    xout[p] = 0.0;
    return;
  }
  double x;
  if (first) {
    x = omega * bscale * b[p];
  } else {
    const int im = clampi(i - 1, nx), ip = clampi(i + 1, nx), jm = clampi(j - 1, ny), jp = clampi(j + 1, ny);
    const double* r0 = xin + (size_t)jm * nx;
    const double* r1 = xin + (size_t)j * nx;
    const double* r2 = xin + (size_t)jp * nx;
    const double c = r1[i];
    const double lx = r1[im] - 2.0 * c + r1[ip];
    const double ly = r0[i] - 2.0 * c + r2[i];
    // Lx Ly x: [1,-2,1] (x) [1,-2,1] on the ghost-mapped neighbourhood
    const double lxm = r0[im] - 2.0 * r0[i] + r0[ip];
    const double lxp = r2[im] - 2.0 * r2[i] + r2[ip];
    const double lxly = lxm - 2.0 * lx + lxp;
    const double px = c1h2 * c - lx - ly - lxly * (1.0 / 6.0);
    x = c + omega * (bscale * b[p] - px);
  }
  xout[p] = x;
  if (upd) upd[p] += upd_scale * x;
}

// P~ x (the matrix-free operator alone), scaled by out_scale.
__global__ void k_p1_apply64(const double* __restrict__ xin, double* __restrict__ out, int nx, int ny, int bcx,
                             int bcy, double c1h2, double out_scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const size_t p = (size_t)j * nx + i;
  if (!interior(bcx, i, nx) || !interior(bcy, j, ny)) {
    out[p] = 0.0;
    return;
  }
  const int im = clampi(i - 1, nx), ip = clampi(i + 1, nx), jm = clampi(j - 1, ny), jp = clampi(j + 1, ny);
  const double* r0 = xin + (size_t)jm * nx;
  const double* r1 = xin + (size_t)j * nx;
  const double* r2 = xin + (size_t)jp * nx;
  const double c = r1[i];
  const double lx = r1[im] - 2.0 * c + r1[ip];
  const double ly = r0[i] - 2.0 * c + r2[i];
  const double lxm = r0[im] - 2.0 * r0[i] + r0[ip];
  const double lxp = r2[im] - 2.0 * r2[i] + r2[ip];
  const double lxly = lxm - 2.0 * lx + lxp;
  out[p] = out_scale * (c1h2 * c - lx - ly - lxly * (1.0 / 6.0));
}

// ---------------------------------------------------------------------------------------
// Plain second-order Yee step pieces (Sec. 5.2, stencil S with c = 1).
__global__ void k_yee_e64(double* __restrict__ ez, const double* __restrict__ hx, const double* __restrict__ hy, int N,
                          double c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i < 1 || j < 1 || i >= N || j >= N) return;
  const double dxhy = hy[(size_t)j * N + i] - hy[(size_t)j * N + i - 1];
  const double dyhx = hx[(size_t)j * (N + 1) + i] - hx[(size_t)(j - 1) * (N + 1) + i];
  ez[(size_t)j * (N + 1) + i] += c * (dxhy - dyhx);
}

__global__ void k_yee_h64(const double* __restrict__ ez, double* __restrict__ hx, double* __restrict__ hy, int N,
                          double c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > N || j > N) return;
  if (j < N && i >= 1 && i < N)
    hx[(size_t)j * (N + 1) + i] -= c * (ez[(size_t)(j + 1) * (N + 1) + i] - ez[(size_t)j * (N + 1) + i]);
  if (i < N && j >= 1 && j < N)
    hy[(size_t)j * N + i] += c * (ez[(size_t)j * (N + 1) + i + 1] - ez[(size_t)j * (N + 1) + i]);
}

// ---------------------------------------------------------------------------------------
// Host launchers

static inline dim3 grid2(int nx, int ny, dim3 blk) { return dim3((nx + blk.x - 1) / blk.x, (ny + blk.y - 1) / blk.y); }

void launch_filter64(const double* u, double* G, const Shape& s, double beta, cudaStream_t st) {
  dim3 blk(32, 8);
  k_filter64<<<grid2(s.nx, s.ny, blk), blk, 0, st>>>(u, G, s.nx, s.ny, s.bcx, s.bcy, beta);
}

void launch_pade64(int axis, const double* in, double* out, int n_lines, int in_ld, int out_len, int out_ld,
                   int out_off, int line_lo, int line_hi, const PadeTable& t, double scale, int accumulate,
                   cudaStream_t st) {
  dim3 blk(32, 8);
  if (axis == 0) {
    k_pade64<0><<<grid2(out_len, n_lines, blk), blk, 0, st>>>(in, out, n_lines, t.rows, in_ld, out_len, out_ld,
                                                              out_off, line_lo, line_hi, t.d_w, t.K, t.B,
                                                              t.all_explicit, scale, accumulate, t.n_in, t.left);
  } else {
    k_pade64<1><<<grid2(n_lines, out_len, blk), blk, 0, st>>>(in, out, n_lines, t.rows, in_ld, out_len, out_ld,
                                                              out_off, line_lo, line_hi, t.d_w, t.K, t.B,
                                                              t.all_explicit, scale, accumulate, t.n_in, t.left);
  }
}

void launch_p1_sweep64(const double* b, const double* xin, double* xout, const Shape& s, double c1h2, double omega,
                       double bscale, int first, double* upd, double upd_scale, cudaStream_t st) {
  dim3 blk(32, 8);
  k_p1_sweep64<<<grid2(s.nx, s.ny, blk), blk, 0, st>>>(b, xin, xout, s.nx, s.ny, s.bcx, s.bcy, c1h2, omega, bscale,
                                                        first, upd, upd_scale);
}

void launch_p1_apply64(const double* x, double* out, const Shape& s, double c1h2, double out_scale, cudaStream_t st) {
  dim3 blk(32, 8);
  k_p1_apply64<<<grid2(s.nx, s.ny, blk), blk, 0, st>>>(x, out, s.nx, s.ny, s.bcx, s.bcy, c1h2, out_scale);
}

void launch_yee_e64(double* ez, const double* hx, const double* hy, int N, double c_e, cudaStream_t st) {
  dim3 blk(32, 8);
  k_yee_e64<<<grid2(N + 1, N + 1, blk), blk, 0, st>>>(ez, hx, hy, N, c_e);
}

void launch_yee_h64(const double* ez, double* hx, double* hy, int N, double c_h, cudaStream_t st) {
  dim3 blk(32, 8);
  k_yee_h64<<<grid2(N + 1, N + 1, blk), blk, 0, st>>>(ez, hx, hy, N, c_h);
}

}  // namespace ms
