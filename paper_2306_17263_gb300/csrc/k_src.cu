// Current sources of the 2D TM_z problem (J = J_z z, div J = 0): a sum of driven modes
//   J_z = a X(m pi x) Y(n pi y) sin(w t),   X, Y = sin or cos,
// The modified Helmholtz equations of Eq. "eq:mh" gain
//   E:  P(J)^{n+1/2} = -Z (kappa^2 - w^2) J^{n+1/2},    H:  (curl d_t J)^{n+1} = (d_y d_t J_z, -d_x d_t J_z),
// (from the Taylor expansion of Sec. 3.1 with Faraday's and Ampere's laws), each through the
// right-hand-side filter of Eq. "eq:ell" with the exact Laplacian of the source, factor
// f = beta - (h^2/12) pi^2 (m^2 + n^2).  The kernels add these terms to a right-hand side before
// the solve; the step index is read from device memory so that captured graphs stay valid.
//
// Sine profiles vanish on the walls with every derivative the Neumann data of Sec. 3.3 use, so the
// even ghosts stay exact.  A cosine profile does not, and three boundary data of the step change
// (Method 2 of Sec. 3.3, the wall data from Ampere's law on the PEC walls):
//   - the ghosts half a cell beyond a Neumann wall: u(-1) = u(0) - g_lo, u(n) = u(n-1) + g_hi with
//     g = h d_n u + (h^3/24) d_nnn u on the wall, where on x = 0, 1 (H_y)
//       d_x H_y = J_z,   d_xxx H_y = (d_tt + d_xx - d_yy) J_z,
//     and on y = 0, 1 (H_x)  d_y H_x = -J_z,  d_yyy H_x = -(d_tt + d_yy - d_xx) J_z.
//     In the H filter of Step 1 (data of H at t^{n+1/2}) the ghost adds -g_lo/12 or +g_hi/12 to G
//     next to the wall; in the H solves of Step 2 (data of H* = (H^{n+3/2} - H^{n+1/2}) / h_tau)
//     the right-hand side loses P1 applied to the ghosts alone, which is nonzero next to the wall;
//   - G_E on the boundary nodes is (h^2/12) Delta E_z = (h^2/12) Z d_t J_z at t^{n+1}.
// The FP64 step applies them with k_wall_hfilter64 / k_wall_ge64 / k_wall_hsolve64.  The FP32 tile
// curl never forms G, so there the filter's ghost terms and G_E on the walls enter b as their Pade
// responses (the curl is linear in G), added by the FP32 source kernels with the ghost part of P1.
#include <cmath>
#include <cstring>
#include <vector>

#include "k_fp64.cuh"

namespace ms {
namespace {

// Per source: ce = -Z (kappa^2 - w^2) f a,  ch = f a w,  kx = pi m,  ky = pi n,  w, and for the
// wall data: gy = a (h + (h^3/24)(pi^2 n^2 - pi^2 m^2 - w^2)) (ghosts of H_y on x = 0, 1),
// gx = -a (h + (h^3/24)(pi^2 m^2 - pi^2 n^2 - w^2)) (ghosts of H_x on y = 0, 1), ge = (h^2/12) Z a w.
struct SrcDev {
  double ce, ch, kx, ky, w, gy, gx, ge;
};

// The time factors are the same at every point: a one-block kernel at the start of each step
// forms them (k_src_time), and the point kernels read them.  FP64: v = sum_q (ce_q sin(w_q t))
// X_q(i) Y_q(j), the product taken in the order of the plain definition.  FP32 (right-hand sides of
// the tile solve): the factors are scaled to the tile's units and rounded to float, and the sum is
// taken in float from the float copy of the tables.
constexpr int kMaxSrc = 64;
struct SrcFac {
  double e[kMaxSrc], hx[kMaxSrc], hy[kMaxSrc];
  float e32[kMaxSrc], hx32[kMaxSrc], hy32[kMaxSrc];
};

// e_q = ce_q sin(w_q t_E), t_E = (n + 1/2) h_tau;  hx_q = ch_q cos(w_q t_H) ky_q, hy_q = ch_q cos(w_q t_H) kx_q,
// t_H = (n + 1) h_tau; the float copies scaled by scale_e and scale_h.
__global__ void k_src_time(const SrcDev* __restrict__ s, int nsrc, const long* __restrict__ d_step, double ht,
                           double scale_e, double scale_h, SrcFac* __restrict__ fac) {
  const int q = threadIdx.x;
  if (q >= nsrc) return;
  const double te = ((double)*d_step + 0.5) * ht, th = ((double)*d_step + 1.0) * ht;
  const double fe = s[q].ce * sin(s[q].w * te);
  const double c = s[q].ch * cos(s[q].w * th);
  const double fx = c * s[q].ky, fy = c * s[q].kx;
  fac->e[q] = fe;
  fac->hx[q] = fx;
  fac->hy[q] = fy;
  fac->e32[q] = (float)(scale_e * fe);
  fac->hx32[q] = (float)(scale_h * fx);
  fac->hy32[q] = (float)(scale_h * fy);
}

// Wall data of one step (k_wall_data), 12 arrays of N + 1: the ghost data of H at t^{n+1/2}
// (H_y on x = 0, 1 by row; H_x on y = 0, 1 by column), G_E on the walls at t^{n+1} (x = 0, x = 1 by
// row; y = 0, y = 1 by column), and the ghost data of H* on the four walls.
enum { WD_GY_LO, WD_GY_HI, WD_GX_LO, WD_GX_HI, WD_V_X0, WD_V_X1, WD_V_Y0, WD_V_Y1,
       WD_SY_LO, WD_SY_HI, WD_SX_LO, WD_SX_HI, WD_COUNT };
// Pade responses to one end value (float, zero beyond kWallReach outputs from that end):
// half-node lines (N inputs, N - 1 outputs) to input 0 and to input N - 1, node lines (N + 1 inputs,
// N outputs) to input 0 and to input N.
constexpr int kWallReach = 64;
struct WallView {
  const double* wd;  // nullptr: no wall terms
  const float* hn0;
  const float* hn1;
  const float* nh0;
  const float* nh1;
};
__host__ __device__ inline WallView wall_view(const double* wd, const float* wr, int N) {
  return WallView{wd, wr, wr + (N - 1), wr + 2 * (N - 1), wr + 2 * (N - 1) + N};
}

// Point kernels: a block is 32 columns by kSrcBy rows, and each thread takes kSrcRows rows kSrcBy
// apart, all loads of a thread issued before its first update (one point per thread left the kernel
// waiting on one memory round trip per wave).  Per point the arithmetic is that of the plain sum.
constexpr int kSrcBy = 8;
constexpr int kSrcRows = 8;

// R += sum_q e_q X_q(i) Y_q(j) at the interior E_z nodes.  FP32 with wall data: plus, in the units of
// R scaled by cE / (kappa^2 Z / h), the Pade responses to the filter's ghost terms of Step 1,
//   kappa^2 Z / h (W_{i-1,0} (-g^y_lo(j) / 12) + W_{i-1,N-1} g^y_hi(j) / 12
//                  - W_{j-1,0} (-g^x_lo(i) / 12) - W_{j-1,N-1} g^x_hi(i) / 12)   (W = A^{-1} D1 per line).
template <typename T>
__global__ void __launch_bounds__(32 * kSrcBy) k_src_e(T* __restrict__ R, int N, int nsrc, const double* __restrict__ tab,
                                                       const float* __restrict__ tab32, const SrcFac* __restrict__ fac,
                                                       WallView wv, float cE) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j0 = blockIdx.y * (kSrcBy * kSrcRows) + threadIdx.y;
  if (i < 1 || i >= N) return;
  const size_t per = 4 * (size_t)(N + 1);  // per-source table block: X, Y at nodes, X', Y' at half-nodes
  T old[kSrcRows], v[kSrcRows];
#pragma unroll
  for (int r = 0; r < kSrcRows; ++r) {
    const int j = j0 + r * kSrcBy;
    old[r] = (j >= 1 && j < N) ? R[(size_t)j * (N + 1) + i] : (T)0;
    v[r] = (T)0;
  }
  for (int q = 0; q < nsrc; ++q) {
    if constexpr (sizeof(T) == 8) {
      const double* tq = tab + q * per;
      const double fx = fac->e[q] * tq[i];
#pragma unroll
      for (int r = 0; r < kSrcRows; ++r) {
        const int j = min(j0 + r * kSrcBy, N);
        v[r] += fx * tq[(N + 1) + j];
      }
    } else {
      const float* tq = tab32 + q * per;
      const float fx = fac->e32[q] * tq[i];
#pragma unroll
      for (int r = 0; r < kSrcRows; ++r) {
        const int j = min(j0 + r * kSrcBy, N);
        v[r] = fmaf(fx, tq[(N + 1) + j], v[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kSrcRows; ++r) {
    const int j = j0 + r * kSrcBy;
    if (j < 1 || j >= N) continue;
    if constexpr (sizeof(T) == 4) {
      const int M = N - 1;
      if (wv.wd && (i - 1 < kWallReach || i - 1 >= M - kWallReach || j - 1 < kWallReach || j - 1 >= M - kWallReach)) {
        const double* wd = wv.wd;
        const size_t L = N + 1;
        const float ax = wv.hn0[i - 1] * (float)(-wd[WD_GY_LO * L + j]) + wv.hn1[i - 1] * (float)wd[WD_GY_HI * L + j];
        const float ay = wv.hn0[j - 1] * (float)(-wd[WD_GX_LO * L + i]) + wv.hn1[j - 1] * (float)wd[WD_GX_HI * L + i];
        v[r] = fmaf(cE * (1.0f / 12.0f), ax - ay, v[r]);
      }
    }
    R[(size_t)j * (N + 1) + i] = old[r] + v[r];
  }
}

// Ghost part of P1 next to a wall with data g (zero at the Dirichlet end points k = 0, N):
// g_k / h^2 + (g_{k-1} - 2 g_k + g_{k+1}) / (6 h^2), in units of h^2.
__device__ __forceinline__ double ghost_p1(const double* g, int k) {
  return g[k] + (g[k - 1] - 2.0 * g[k] + g[k + 1]) * (1.0 / 6.0);
}

// R_x += sum_q hx_q X_q(i) Y'_q(j)/ky_q;  R_y -= sum_q hy_q X'_q(i)/kx_q Y_q(j).  FP32 with wall data:
// plus the Pade responses to G_E on the walls, -cH (W_{j,0} v(i, 0) + W_{j,N} v(i, N)) on R_x and
// +cH (W_{i,0} v(0, j) + W_{i,N} v(N, j)) on R_y (cH = scale kappa^2 / (Z h)), minus the ghost part of
// P1 with the data of H* next to the walls (times sP = scale / h^2).
template <typename T>
__global__ void __launch_bounds__(32 * kSrcBy) k_src_h(T* __restrict__ Rx, T* __restrict__ Ry, int N, int nsrc,
                                                       const double* __restrict__ tab, const float* __restrict__ tab32,
                                                       const SrcFac* __restrict__ fac, WallView wv, float cH, double sP) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j0 = blockIdx.y * (kSrcBy * kSrcRows) + threadIdx.y;
  if (i > N) return;
  const size_t per = 4 * (size_t)(N + 1);
  const bool ix = i >= 1 && i < N;  // H_x column (interior in x)
  const bool iy = i < N;            // H_y column
  T ox[kSrcRows], oy[kSrcRows], vx[kSrcRows], vy[kSrcRows];
#pragma unroll
  for (int r = 0; r < kSrcRows; ++r) {
    const int j = j0 + r * kSrcBy;
    ox[r] = (ix && j < N) ? Rx[(size_t)j * (N + 1) + i] : (T)0;
    oy[r] = (iy && j >= 1 && j < N) ? Ry[(size_t)j * N + i] : (T)0;
    vx[r] = (T)0;
    vy[r] = (T)0;
  }
  const int ic = min(i, N - 1);  // X' is tabulated at the N half-nodes
  for (int q = 0; q < nsrc; ++q) {
    if constexpr (sizeof(T) == 8) {
      const double* tq = tab + q * per;
      const double fx = fac->hx[q] * tq[i], fy = fac->hy[q] * tq[2 * (N + 1) + ic];
#pragma unroll
      for (int r = 0; r < kSrcRows; ++r) {
        const int j = min(j0 + r * kSrcBy, N);
        vx[r] += fx * tq[3 * (N + 1) + min(j, N - 1)];
        vy[r] += fy * tq[(N + 1) + j];
      }
    } else {
      const float* tq = tab32 + q * per;
      const float fx = fac->hx32[q] * tq[i], fy = fac->hy32[q] * tq[2 * (N + 1) + ic];
#pragma unroll
      for (int r = 0; r < kSrcRows; ++r) {
        const int j = min(j0 + r * kSrcBy, N);
        vx[r] = fmaf(fx, tq[3 * (N + 1) + min(j, N - 1)], vx[r]);
        vy[r] = fmaf(fy, tq[(N + 1) + j], vy[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kSrcRows; ++r) {
    const int j = j0 + r * kSrcBy;
    if (ix && j < N) {
      if constexpr (sizeof(T) == 4) {
        if (wv.wd && (j < kWallReach || j >= N - kWallReach)) {
          const double* wd = wv.wd;
          const size_t L = N + 1;
          vx[r] = fmaf(-cH, wv.nh0[j] * (float)wd[WD_V_Y0 * L + i] + wv.nh1[j] * (float)wd[WD_V_Y1 * L + i], vx[r]);
          if (j == 0) vx[r] -= (float)(sP * ghost_p1(wd + WD_SX_LO * L, i));
          if (j == N - 1) vx[r] += (float)(sP * ghost_p1(wd + WD_SX_HI * L, i));
        }
      }
      Rx[(size_t)j * (N + 1) + i] = ox[r] + vx[r];
    }
    if (iy && j >= 1 && j < N) {
      if constexpr (sizeof(T) == 4) {
        if (wv.wd && (i < kWallReach || i >= N - kWallReach)) {
          const double* wd = wv.wd;
          const size_t L = N + 1;
          vy[r] = fmaf(-cH, wv.nh0[i] * (float)wd[WD_V_X0 * L + j] + wv.nh1[i] * (float)wd[WD_V_X1 * L + j], vy[r]);
          if (i == 0) vy[r] += (float)(sP * ghost_p1(wd + WD_SY_LO * L, j));
          if (i == N - 1) vy[r] -= (float)(sP * ghost_p1(wd + WD_SY_HI * L, j));
        }
      }
      Ry[(size_t)j * N + i] = oy[r] - vy[r];
    }
  }
}

__global__ void k_tick(long* d_step) { *d_step += 1; }

// Table layout per source (4 (N + 1) doubles): X at nodes i = 0..N, Y at nodes j = 0..N,
// X'/(pi m) at half-nodes i = 0..N-1, Y'/(pi n) at half-nodes j = 0..N-1.
__device__ __forceinline__ double wall_sum_hy(const SrcDev* s, int nsrc, const double* tab, int N, int side, int j,
                                              double t0, double t1, double inv_dt) {
  // ghost datum of H_y on wall x = side at row j: sum_q gy_q X_q(side) Y_q(j) T_q
  if (j <= 0 || j >= N) return 0.0;
  const size_t per = 4 * (size_t)(N + 1);
  double v = 0.0;
  for (int q = 0; q < nsrc; ++q) {
    const double* tq = tab + q * per;
    const double T = inv_dt > 0.0 ? (sin(s[q].w * t1) - sin(s[q].w * t0)) * inv_dt : sin(s[q].w * t1);
    v += s[q].gy * T * tq[side ? N : 0] * tq[(N + 1) + j];
  }
  return v;
}
__device__ __forceinline__ double wall_sum_hx(const SrcDev* s, int nsrc, const double* tab, int N, int side, int i,
                                              double t0, double t1, double inv_dt) {
  // ghost datum of H_x on wall y = side at column i: sum_q gx_q X_q(i) Y_q(side) T_q
  if (i <= 0 || i >= N) return 0.0;
  const size_t per = 4 * (size_t)(N + 1);
  double v = 0.0;
  for (int q = 0; q < nsrc; ++q) {
    const double* tq = tab + q * per;
    const double T = inv_dt > 0.0 ? (sin(s[q].w * t1) - sin(s[q].w * t0)) * inv_dt : sin(s[q].w * t1);
    v += s[q].gx * T * tq[i] * tq[(N + 1) + (side ? N : 0)];
  }
  return v;
}

// The wall data of a step for the FP32 source kernels (layout WD_*); thread k = 0..N.
__global__ void k_wall_data(double* __restrict__ wd, int N, const SrcDev* __restrict__ s, int nsrc,
                            const double* __restrict__ tab, const long* __restrict__ d_step, double ht) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > N) return;
  const size_t L = N + 1, per = 4 * L;
  const double th = ((double)*d_step + 0.5) * ht, t1 = th + 0.5 * ht, t32 = th + ht, idt = 1.0 / ht;
  wd[WD_GY_LO * L + k] = wall_sum_hy(s, nsrc, tab, N, 0, k, th, th, 0.0);
  wd[WD_GY_HI * L + k] = wall_sum_hy(s, nsrc, tab, N, 1, k, th, th, 0.0);
  wd[WD_GX_LO * L + k] = wall_sum_hx(s, nsrc, tab, N, 0, k, th, th, 0.0);
  wd[WD_GX_HI * L + k] = wall_sum_hx(s, nsrc, tab, N, 1, k, th, th, 0.0);
  wd[WD_SY_LO * L + k] = wall_sum_hy(s, nsrc, tab, N, 0, k, th, t32, idt);
  wd[WD_SY_HI * L + k] = wall_sum_hy(s, nsrc, tab, N, 1, k, th, t32, idt);
  wd[WD_SX_LO * L + k] = wall_sum_hx(s, nsrc, tab, N, 0, k, th, t32, idt);
  wd[WD_SX_HI * L + k] = wall_sum_hx(s, nsrc, tab, N, 1, k, th, t32, idt);
  double v[4] = {0.0, 0.0, 0.0, 0.0};  // G_E at (0, k), (N, k), (k, 0), (k, N)
  for (int q = 0; q < nsrc; ++q) {
    const double* tq = tab + q * per;
    const double c = s[q].ge * cos(s[q].w * t1);
    v[0] += c * tq[0] * tq[L + k];
    v[1] += c * tq[N] * tq[L + k];
    v[2] += c * tq[k] * tq[L];
    v[3] += c * tq[k] * tq[L + N];
  }
  wd[WD_V_X0 * L + k] = v[0];
  wd[WD_V_X1 * L + k] = v[1];
  wd[WD_V_Y0 * L + k] = v[2];
  wd[WD_V_Y1 * L + k] = v[3];
}

// Step 1: the ghosts of H^{n+1/2} in the filter, G -= g_lo / 12 next to the low wall and
// G += g_hi / 12 next to the high wall.  Thread k = 1..N-1 takes row k of G_y and column k of G_x.
__global__ void k_wall_hfilter64(double* __restrict__ Gx, double* __restrict__ Gy, int N, const SrcDev* __restrict__ s,
                                 int nsrc, const double* __restrict__ tab, const long* __restrict__ d_step, double ht) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < 1 || k >= N) return;
  const double t = ((double)*d_step + 0.5) * ht;
  Gy[(size_t)k * N] -= wall_sum_hy(s, nsrc, tab, N, 0, k, t, t, 0.0) * (1.0 / 12.0);
  Gy[(size_t)k * N + N - 1] += wall_sum_hy(s, nsrc, tab, N, 1, k, t, t, 0.0) * (1.0 / 12.0);
  Gx[k] -= wall_sum_hx(s, nsrc, tab, N, 0, k, t, t, 0.0) * (1.0 / 12.0);
  Gx[(size_t)(N - 1) * (N + 1) + k] += wall_sum_hx(s, nsrc, tab, N, 1, k, t, t, 0.0) * (1.0 / 12.0);
}

// Step 2: G_E on the boundary nodes = sum_q ge_q cos(w_q t) X_q(i) Y_q(j), t = (n + 1) h_tau.
// Thread k = 0..N takes nodes (k, 0) and (k, N), and for 0 < k < N also (0, k) and (N, k).
__global__ void k_wall_ge64(double* __restrict__ GE, int N, const SrcDev* __restrict__ s, int nsrc,
                            const double* __restrict__ tab, const long* __restrict__ d_step, double ht) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > N) return;
  const double t = ((double)*d_step + 1.0) * ht;
  const size_t per = 4 * (size_t)(N + 1);
  const int ni = (k > 0 && k < N) ? 4 : 2;
  for (int e = 0; e < ni; ++e) {
    const int i = e < 2 ? k : (e == 2 ? 0 : N);
    const int j = e < 2 ? (e == 0 ? 0 : N) : k;
    double v = 0.0;
    for (int q = 0; q < nsrc; ++q) {
      const double* tq = tab + q * per;
      v += s[q].ge * cos(s[q].w * t) * tq[i] * tq[(N + 1) + j];
    }
    GE[(size_t)j * (N + 1) + i] = v;
  }
}

// Step 2: the right-hand sides of the H solves lose P1 applied to the ghosts of H* alone (zero
// field inside): next to a low wall with datum g (g = 0 at the Dirichlet end points),
//   P1_g 0 = g / h^2 + (g_{-} - 2 g + g_{+}) / (6 h^2),   and the negative of it with g_hi next to a
// high wall.  Thread k = 1..N-1 takes column k of R_x (rows 0 and N-1) and row k of R_y.
__global__ void k_wall_hsolve64(double* __restrict__ Rx, double* __restrict__ Ry, int N, const SrcDev* __restrict__ s,
                                int nsrc, const double* __restrict__ tab, const long* __restrict__ d_step, double ht,
                                double ih2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < 1 || k >= N) return;
  const double t0 = ((double)*d_step + 0.5) * ht, t1 = t0 + ht, idt = 1.0 / ht;
  for (int side = 0; side < 2; ++side) {
    const double sg = side ? -1.0 : 1.0;
    {
      const double gm = wall_sum_hx(s, nsrc, tab, N, side, k - 1, t0, t1, idt);
      const double g0 = wall_sum_hx(s, nsrc, tab, N, side, k, t0, t1, idt);
      const double gp = wall_sum_hx(s, nsrc, tab, N, side, k + 1, t0, t1, idt);
      const double c = sg * ih2 * (g0 + (gm - 2.0 * g0 + gp) * (1.0 / 6.0));
      Rx[(size_t)(side ? N - 1 : 0) * (N + 1) + k] -= c;
    }
    {
      const double gm = wall_sum_hy(s, nsrc, tab, N, side, k - 1, t0, t1, idt);
      const double g0 = wall_sum_hy(s, nsrc, tab, N, side, k, t0, t1, idt);
      const double gp = wall_sum_hy(s, nsrc, tab, N, side, k + 1, t0, t1, idt);
      const double c = sg * ih2 * (g0 + (gm - 2.0 * g0 + gp) * (1.0 / 6.0));
      Ry[(size_t)k * N + (side ? N - 1 : 0)] -= c;
    }
  }
}

}  // namespace

// Host tables: per source, X(pi m i / N) (i = 0..N), Y(pi n j / N), X'/(pi m) at (i + 1/2) / N
// (i = 0..N-1), Y'/(pi n) at (j + 1/2) / N, with the arguments reduced exactly in integers (so the
// wall values are exact: sin 0, cos 0 = 1, cos(pi m) = (-1)^m).
int build_sources(ms_grid* g, const SrcSpec* src, int nsrc, std::vector<unsigned char>* dev_blob,
                  std::vector<double>* tabs) {
  const int N = g->N;
  const double h = g->h, pi = M_PI;
  std::vector<SrcDev> sd(nsrc);
  tabs->assign((size_t)nsrc * 4 * (N + 1), 0.0);
  auto at_node = [&](int p, int k, int i) {  // sin or cos of pi k i / N
    const long q = ((long)k * i) % (2L * N);
    if (p) return std::cos(pi * (double)q / N);
    if (i == 0 || i == N) return 0.0;
    return std::sin(pi * (double)q / N);
  };
  auto dunit_half = [&](int p, int k, int i) {  // d/dx of the profile at (i + 1/2) / N, over pi k
    const long q = ((long)k * (2L * i + 1)) % (4L * N);
    return p ? -std::sin(pi * (double)q / (2.0 * N)) : std::cos(pi * (double)q / (2.0 * N));
  };
  for (int q = 0; q < nsrc; ++q) {
    const int m = src[q].m, n = src[q].n;
    const double a = src[q].amp, w = src[q].omega;
    const double pm2 = pi * pi * (double)m * m, pn2 = pi * pi * (double)n * n, h3 = h * h * h / 24.0;
    const double f = g->beta - (h * h / 12.0) * pi * pi * ((double)m * m + (double)n * n);
    sd[q].ce = -g->Z * (g->kappa2 - w * w) * f * a;
    sd[q].ch = f * a * w;
    sd[q].kx = pi * m;
    sd[q].ky = pi * n;
    sd[q].w = w;
    sd[q].gy = a * (h + h3 * (pn2 - pm2 - w * w));
    sd[q].gx = -a * (h + h3 * (pm2 - pn2 - w * w));
    sd[q].ge = h * h / 12.0 * g->Z * a * w;
    double* tq = tabs->data() + (size_t)q * 4 * (N + 1);
    for (int i = 0; i <= N; ++i) tq[i] = at_node(src[q].px, m, i);
    for (int j = 0; j <= N; ++j) tq[(N + 1) + j] = at_node(src[q].py, n, j);
    for (int i = 0; i < N; ++i) tq[2 * (N + 1) + i] = dunit_half(src[q].px, m, i);
    for (int j = 0; j < N; ++j) tq[3 * (N + 1) + j] = dunit_half(src[q].py, n, j);
  }
  dev_blob->resize(sd.size() * sizeof(SrcDev));
  std::memcpy(dev_blob->data(), sd.data(), dev_blob->size());
  return (int)sizeof(SrcDev);
}

size_t src_factor_bytes() { return sizeof(SrcFac); }

void launch_src_time(ms_grid* g, double scale_e, double scale_h) {
  k_src_time<<<1, kMaxSrc, 0, g->stream>>>((const SrcDev*)g->d_src, g->nsrc, g->d_step, g->ht, scale_e, scale_h,
                                           (SrcFac*)g->d_srcfac);
}
static dim3 src_grid(int N) { return dim3((N + 1 + 31) / 32, (N + 1 + kSrcBy * kSrcRows - 1) / (kSrcBy * kSrcRows)); }

void launch_src_e64(ms_grid* g, double* R) {
  dim3 blk(32, kSrcBy), grd = src_grid(g->N);
  k_src_e<double><<<grd, blk, 0, g->stream>>>(R, g->N, g->nsrc, g->d_srctab, g->d_srctab32,
                                               (const SrcFac*)g->d_srcfac, WallView{}, 0.0f);
}
void launch_src_h64(ms_grid* g, double* Rx, double* Ry) {
  dim3 blk(32, kSrcBy), grd = src_grid(g->N);
  k_src_h<double><<<grd, blk, 0, g->stream>>>(Rx, Ry, g->N, g->nsrc, g->d_srctab, g->d_srctab32,
                                               (const SrcFac*)g->d_srcfac, WallView{}, 0.0f, 0.0);
}
void launch_src_e32(ms_grid* g, float* R, double scale_e) {
  dim3 blk(32, kSrcBy), grd = src_grid(g->N);
  const WallView wv = g->d_walldata ? wall_view(g->d_walldata, g->d_wresp, g->N) : WallView{};
  const float cE = (float)(scale_e * g->kappa2 * g->Z / g->h);
  k_src_e<float><<<grd, blk, 0, g->stream>>>(R, g->N, g->nsrc, g->d_srctab, g->d_srctab32,
                                              (const SrcFac*)g->d_srcfac, wv, cE);
}
void launch_src_h32(ms_grid* g, float* Rx, float* Ry, double scale_h) {
  dim3 blk(32, kSrcBy), grd = src_grid(g->N);
  const WallView wv = g->d_walldata ? wall_view(g->d_walldata, g->d_wresp, g->N) : WallView{};
  const float cH = (float)(scale_h * g->kappa2 / (g->Z * g->h));
  k_src_h<float><<<grd, blk, 0, g->stream>>>(Rx, Ry, g->N, g->nsrc, g->d_srctab, g->d_srctab32,
                                              (const SrcFac*)g->d_srcfac, wv, cH, scale_h / (g->h * g->h));
}
void launch_wall_data(ms_grid* g) {
  k_wall_data<<<(g->N + 1 + 127) / 128, 128, 0, g->stream>>>(g->d_walldata, g->N, (const SrcDev*)g->d_src, g->nsrc,
                                                             g->d_srctab, g->d_step, g->ht);
}
size_t wall_data_doubles(int N) { return (size_t)WD_COUNT * (N + 1); }

// Pade responses for the FP32 wall terms (PAPER closure): rows of W = A^{-1} D1 within kWallReach of
// either end, the entries of their first and last inputs.
void wall_responses(int N, std::vector<float>* wr) {
  wr->assign((size_t)2 * (N - 1) + 2 * N, 0.0f);
  if (N < 5) return;  // the end rows of the PAPER closure need 4 outputs per line (grids are larger)
  std::vector<double> row;
  for (int kind = 0; kind < 2; ++kind) {
    const int M = kind == HALF_TO_NODE ? N - 1 : N;
    float* c0 = wr->data() + (kind == HALF_TO_NODE ? 0 : 2 * (N - 1));
    float* c1 = c0 + M;
    for (int i = 0; i < M; ++i) {
      if (i >= kWallReach && i < M - kWallReach) continue;
      pade_dense_row(M, MS_CLOSURE_PAPER, kind, i, &row);
      c0[i] = (float)row[0];
      c1[i] = (float)row[M];
    }
  }
}
void launch_tick(ms_grid* g) { k_tick<<<1, 1, 0, g->stream>>>(g->d_step); }

void launch_wall_hfilter64(ms_grid* g, double* Gx, double* Gy) {
  k_wall_hfilter64<<<(g->N + 127) / 128, 128, 0, g->stream>>>(Gx, Gy, g->N, (const SrcDev*)g->d_src, g->nsrc,
                                                              g->d_srctab, g->d_step, g->ht);
}
void launch_wall_ge64(ms_grid* g, double* GE) {
  k_wall_ge64<<<(g->N + 1 + 127) / 128, 128, 0, g->stream>>>(GE, g->N, (const SrcDev*)g->d_src, g->nsrc, g->d_srctab,
                                                              g->d_step, g->ht);
}
void launch_wall_hsolve64(ms_grid* g, double* Rx, double* Ry) {
  k_wall_hsolve64<<<(g->N + 127) / 128, 128, 0, g->stream>>>(Rx, Ry, g->N, (const SrcDev*)g->d_src, g->nsrc,
                                                             g->d_srctab, g->d_step, g->ht, 1.0 / (g->h * g->h));
}

}  // namespace ms
