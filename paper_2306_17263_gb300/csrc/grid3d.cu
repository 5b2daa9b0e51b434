// Three-dimensional compact scheme: six components on the staggered unit cube (Eq. "eq:meshes"),
// boundary types of Table "tab:bc", Step 1 / Step 2 of Sec. 3.4 with
//   curl_h = [[0, -d_z, d_y], [d_z, 0, -d_x], [-d_y, d_x, 0]],
// the 7-point filter of Eq. "eq:ell" (Delta_h = D_xx + D_yy + D_zz) and the 19-point
// P1 = -(Delta_h + (h^2/6) Upsilon_h) + kappa^2 (1 + 2/r^2), Upsilon_h = D_zz D_xx + D_yy D_zz
// + D_xx D_yy (Def. "def:operatorsP").  Every component is Dirichlet (stored wall zeros) along
// the axes on which it sits on nodes and Neumann (even ghosts) along its half-node axes.
//
// MS_FP64: one operator per launch in FP64 (filter, Pade band along one axis, Richardson sweep).
// MS_FP32_REFINED: the arithmetic of the 2D FP32 path (k_mixed.cu) carried to 3D: float-float
// state; each half-step first filters its three source components once into float-float
// G = 12 beta u + L u (k_ffilt3d32), then per Pade term one tile kernel (k_term3d32) forms the
// first differences of G along the line (the filter commutes with the difference under the ghost
// rules) and applies A^{-1} (interior rows by two first-order recurrences, rows near a wall by the
// explicit band rows, farthest taps first), accumulating the right-hand side (a difference kernel
// and a band kernel take over for tables wider than the tile holds); the solve
// (k_sweep3d32) is the Richardson iteration on 6 h^2 P1 with the exact-product residual and
// the split last correction, each sweep one launch that marches tiles along z.
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "grid3d.cuh"
#include "k_fp64.cuh"
#include "k_tiled.cuh"
#include "k_src3.cuh"
#include "k_transform.cuh"

namespace ms {

Shape3 field_shape3(int N, int c) {
  Shape3 s;
  for (int a = 0; a < 3; ++a) {
    const bool node = (c < 3) ? (a != c % 3) : (a == c % 3);
    s.bc[a] = node ? DIR : NEU;
    s.n[a] = node ? N + 1 : N;
  }
  return s;
}

struct Grid3D {
  Shape3 sh[6];
  double* f64[6] = {};
  float* hi[6] = {};
  float* lo[6] = {};
  double* s64[7] = {};  // FP64: G[3], R, sweep ping-pong [2], solve output; FP32 grids use [0], [1]
  float* s32[4] = {};   // FP32: differences, R, sweep ping-pong [2]
  float* gh[3] = {};    // FP32: filtered components G~ (hi, lo) of one half-step, slot c % 3
  float* gl[3] = {};
  double* dview[6] = {};  // FP32_REFINED grids: FP64 copy of the state for the diagnostics
  size_t nmax = 0;      // points of the largest component
  int solver = MS_SOLVER_RICHARDSON;  // FP32_REFINED: P1 solve by Richardson sweeps or by transforms
  TransformSolver* ts = nullptr;       // made when the transform solver is first selected
  int ts_sweeps = 0;                   // refinement sweeps after a transform solve
};

namespace {

thread_local std::string g_err3;

ms_status fail3(ms_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

#define MS3_CUDA(call)                                                                            \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail3(MS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define MS3_TRY(expr)           \
  do {                          \
    ms_status s_ = (expr);      \
    if (s_ != MS_OK) return s_; \
  } while (0)

__device__ __forceinline__ bool unk3(const Shape3& s, int i, int j, int k) {
  return interior(s.bc[0], i, s.n[0]) && interior(s.bc[1], j, s.n[1]) && interior(s.bc[2], k, s.n[2]);
}

__device__ __forceinline__ size_t at3(const Shape3& s, int i, int j, int k) {
  return ((size_t)k * s.n[1] + j) * s.n[0] + i;
}

dim3 grid3(const Shape3& s, dim3 blk) {
  return dim3((s.n[0] + blk.x - 1) / blk.x, (s.n[1] + blk.y - 1) / blk.y, s.n[2]);
}

// ---------------------------------------------------------------------------------------
// FP64 kernels

// G = beta u + (1/12) L u, L = h^2 Delta_h (7 points), 0 at wall points.
__global__ void k_filter3d64(const double* __restrict__ u, double* __restrict__ G, Shape3 s, double beta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= s.n[0] || j >= s.n[1]) return;
  const size_t p = at3(s, i, j, k);
  if (!unk3(s, i, j, k)) {
    G[p] = 0.0;
    return;
  }
  const double c = u[p];
  const double lap = (u[at3(s, clampi(i - 1, s.n[0]), j, k)] + u[at3(s, clampi(i + 1, s.n[0]), j, k)]) +
                     (u[at3(s, i, clampi(j - 1, s.n[1]), k)] + u[at3(s, i, clampi(j + 1, s.n[1]), k)]) +
                     (u[at3(s, i, j, clampi(k - 1, s.n[2]))] + u[at3(s, i, j, clampi(k + 1, s.n[2]))]) - 6.0 * c;
  G[p] = beta * c + lap * (1.0 / 12.0);
}

// Pade band along AXIS (App. A.1): out[o] (+)= scale * sum_t W(r, t) in[r - left + t], r = o - out_off,
// at every point of the output component; the two other coordinates are shared with the input.
template <int AXIS>
__global__ void k_pade3d64(const double* __restrict__ in, double* __restrict__ out, Shape3 so, Shape3 si,
                           const double* __restrict__ tab, int rows, int n_in, int left, int K, int B,
                           int all_explicit, int out_off, double scale, int accumulate) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  if (x >= so.n[0] || y >= so.n[1]) return;
  const size_t po = at3(so, x, y, z);
  const int o = AXIS == 0 ? x : (AXIS == 1 ? y : z);
  const int r = o - out_off;
  double v = 0.0;
  if (r >= 0 && r < rows) {
    const double* w = pade_row_ptr(tab, r, rows, K, B, all_explicit);
    size_t base, stride;
    if (AXIS == 0) {
      base = at3(si, 0, y, z);
      stride = 1;
    } else if (AXIS == 1) {
      base = at3(si, x, 0, z);
      stride = (size_t)si.n[0];
    } else {
      base = at3(si, x, y, 0);
      stride = (size_t)si.n[0] * si.n[1];
    }
    const int k0 = r - left;
    for (int t = 0; t < 2 * K + 2; ++t) {
      const int kk = k0 + t;
      if (kk < 0 || kk >= n_in) continue;
      v = fma(w[t], in[base + (size_t)kk * stride], v);
    }
    v *= scale;
  }
  out[po] = accumulate ? out[po] + v : v;
}

// One Richardson sweep for P~ x = bscale b, P~ = h^2 P1 = c1h2 - (Lx + Ly + Lz) - (1/6)(LxLy + LyLz + LzLx)
// (19 points); first != 0: x_in = 0.  upd != nullptr: upd += upd_scale * x_out.
__global__ void k_sweep3d64(const double* __restrict__ b, const double* __restrict__ xin, double* __restrict__ xout,
                            Shape3 s, double c1h2, double omega, double bscale, int first, double* __restrict__ upd,
                            double upd_scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= s.n[0] || j >= s.n[1]) return;
  const size_t p = at3(s, i, j, k);
  if (!unk3(s, i, j, k)) {
    xout[p] = 0.0;
    return;
  }
  double x;
  if (first) {
    x = omega * bscale * b[p];
  } else {
    const int im = clampi(i - 1, s.n[0]), ip = clampi(i + 1, s.n[0]);
    const int jm = clampi(j - 1, s.n[1]), jp = clampi(j + 1, s.n[1]);
    const int km = clampi(k - 1, s.n[2]), kp = clampi(k + 1, s.n[2]);
    auto X = [&](int a, int bb, int c) { return xin[at3(s, a, bb, c)]; };
    auto LX = [&](int bb, int c) { return X(im, bb, c) - 2.0 * X(i, bb, c) + X(ip, bb, c); };
    auto LY = [&](int a, int c) { return X(a, jm, c) - 2.0 * X(a, j, c) + X(a, jp, c); };
    const double c0 = X(i, j, k);
    const double lx = LX(j, k), ly = LY(i, k);
    const double lz = X(i, j, km) - 2.0 * c0 + X(i, j, kp);
    const double lxly = LX(jm, k) - 2.0 * lx + LX(jp, k);
    const double lxlz = LX(j, km) - 2.0 * lx + LX(j, kp);
    const double lylz = LY(i, km) - 2.0 * ly + LY(i, kp);
    const double px = c1h2 * c0 - (lx + ly + lz) - (lxly + lylz + lxlz) * (1.0 / 6.0);
    x = c0 + omega * (bscale * b[p] - px);
  }
  xout[p] = x;
  if (upd) upd[p] += upd_scale * x;
}

__global__ void k_zero_walls3d64(double* __restrict__ u, Shape3 s) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= s.n[0] || j >= s.n[1]) return;
  if (!unk3(s, i, j, k)) u[at3(s, i, j, k)] = 0.0;
}

// Superposition of separable modes: out = sum_q coef[q] tx[q][i] ty[q][j] tz[q][k].
__global__ void k_mode_field3(double* __restrict__ out, Shape3 s, const double* __restrict__ tx,
                              const double* __restrict__ ty, const double* __restrict__ tz,
                              const double* __restrict__ coef, int nm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= s.n[0] || j >= s.n[1]) return;
  double v = 0.0;
  for (int q = 0; q < nm; ++q)
    v += coef[q] * tx[(size_t)q * s.n[0] + i] * ty[(size_t)q * s.n[1] + j] * tz[(size_t)q * s.n[2] + k];
  out[at3(s, i, j, k)] = unk3(s, i, j, k) ? v : 0.0;
}

// ---------------------------------------------------------------------------------------
// FP32_REFINED kernels

// (hi, lo) += (s_hi + s_lo) x with error-free transformations (two-product by FMA, Knuth two-sum).
__device__ __forceinline__ void ff_add_scaled3(float& hi, float& lo, float x, float s_hi, float s_lo) {
  const float p = __fmul_rn(s_hi, x);
  float e = fmaf(s_hi, x, -p);
  e = fmaf(s_lo, x, e);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float l = __fadd_rn(lo, __fadd_rn(err, e));
  const float h2 = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(h2, s));
  hi = h2;
}

// Interior row of A^{-1} at offsets -KB3 .. KB3+1 (hi) and the lo parts of offsets -1, 0, 1: the
// same Toeplitz row for every grid, 24 (-rho) rho^|d| / (1 - rho^2), rho = -11 + sqrt(120).
constexpr int KB3 = 7;
__constant__ float c_w3[2 * KB3 + 2];
__constant__ float c_wl3[3];
// The interior rows as the recurrences A factors into: rho (FP32), 1 / (1 - rho), and the scale
// (1 - rho_f) / (1 + rho_f) (hi, lo) that gives them a DC gain of exactly 1.
__constant__ float c_rec3[4];

// Paired FP32 arithmetic (two correctly rounded operations per instruction, sm_100 and later):
// bitwise the same as the scalar operations on each half.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// ff_add_scaled3 on two independent pairs at once.
__device__ __forceinline__ void ff_add_scaled3_2(float2& hi, float2& lo, float2 x, float2 s_hi, float2 s_lo) {
  const float2 p = mul2(s_hi, x);
  float2 e = fma2(s_hi, x, neg2(p));
  e = fma2(s_lo, x, e);
  const float2 s = add2(hi, p);
  const float2 bb = sub2(s, hi);
  const float2 err = add2(sub2(hi, sub2(s, bb)), sub2(p, bb));
  const float2 l = add2(lo, add2(err, e));
  const float2 h2 = add2(s, l);
  lo = sub2(l, sub2(h2, s));
  hi = h2;
}

// Float-float filter of one component, Eq. "eq:ell" in the units of the FP32 step:
//   G = 12 beta u + L u,  L = h^2 Delta_h (7 points),
// with even ghosts on Neumann axes and the stored wall zeros on Dirichlet axes; G = 0 at wall
// points.  12 beta u is an exact two-product of the hi parts plus the cross terms; L u, a sum of
// first differences each taken of the float-float values (so FP32 holds it to its own relative
// accuracy), joins the low word, and two-sum renormalises the pair.  The Pade terms below then
// difference G: D1 G = (12 beta + L') D1 u, the filter commuting with the difference under the
// ghost rules (zero differences beyond the ends of a Neumann line, even ones on a Dirichlet line).
// The layout is that of the sweep below: a block of 32 x 8 threads takes a 32 x 16 tile, a thread
// rows j and j + 8 of one column as a pair (paired FP32 instructions), marching FZ3 planes along
// z with the planes z-1, z, z+1 (hi and lo, one-point halo in x and y, clamped) in a ring in
// shared memory; the next plane is fetched into registers while the current one is computed.
constexpr int FZ3 = 16;
constexpr int FTX = 32, FTT = 8, FTY = 2 * FTT;
constexpr int FXP = FTX + 2, FRP = FTT + 2, FN = FRP * FXP;
static_assert(FN <= 2 * FTX * FTT, "two staged pairs per thread");
__global__ void __launch_bounds__(FTX * FTT, 6) k_ffilt3d32(const float* __restrict__ hi, const float* __restrict__ lo,
                                                            Shape3 s, float* __restrict__ gh, float* __restrict__ gl,
                                                            float cb_hi, float cb_lo) {
  __shared__ float2 hs[3][FRP][FXP];
  __shared__ float2 ls[3][FRP][FXP];
  const int n0 = s.n[0], n1 = s.n[1], n2 = s.n[2];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = blockIdx.x * FTX + tx, j = blockIdx.y * FTY + ty;  // rows j and j + FTT
  const int k0 = blockIdx.z * FZ3, k1 = min(k0 + FZ3, n2);
  const bool in0 = i < n0 && j < n1, in1 = i < n0 && j + FTT < n1;
  const bool ux = i < n0 && interior(s.bc[0], i, n0);
  const bool unk0 = in0 && ux && interior(s.bc[1], j, n1), unk1 = in1 && ux && interior(s.bc[1], j + FTT, n1);
  const int sz = n0 * n1;
  const int t1 = ty * FTX + tx, t2 = t1 + FTX * FTT;
  const bool has2 = t2 < FN;
  auto pair_off = [&](int e, int half) {
    const int row = e / FXP, col = e - row * FXP;
    return clampi(blockIdx.y * FTY + row - 1 + half * FTT, n1) * n0 + clampi(blockIdx.x * FTX + col - 1, n0);
  };
  const int o1a = pair_off(t1, 0), o1b = pair_off(t1, 1);
  const int o2a = pair_off(has2 ? t2 : t1, 0), o2b = pair_off(has2 ? t2 : t1, 1);
  float2 ha, la, hb, lb;
  auto fetch = [&](int kk) {
    const int q = clampi(kk, n2) * sz;
    ha = make_float2(hi[q + o1a], hi[q + o1b]);
    la = make_float2(lo[q + o1a], lo[q + o1b]);
    if (has2) {
      hb = make_float2(hi[q + o2a], hi[q + o2b]);
      lb = make_float2(lo[q + o2a], lo[q + o2b]);
    }
  };
  auto stage = [&](int slot) {
    (&hs[slot][0][0])[t1] = ha;
    (&ls[slot][0][0])[t1] = la;
    if (has2) {
      (&hs[slot][0][0])[t2] = hb;
      (&ls[slot][0][0])[t2] = lb;
    }
  };
  fetch(k0 - 1);
  stage(0);
  fetch(k0);
  stage(1);
  fetch(k0 + 1);
  int zm = 0, z0 = 1, zp = 2;
  int p = k0 * sz + j * n0 + i;
  const int dj = FTT * n0;
  const int c0 = tx + 1, r0 = ty + 1;
  const float2 cbh = bc2(cb_hi), cbl = bc2(cb_lo);
  for (int k = k0; k < k1; ++k, p += sz) {
    stage(zp);
    __syncthreads();
    if (k + 1 < k1) fetch(k + 2);
    const float2 hc = hs[z0][r0][c0], lc = ls[z0][r0][c0];
    auto dv = [&](int pl, int rr, int cc) { return add2(sub2(hs[pl][rr][cc], hc), sub2(ls[pl][rr][cc], lc)); };
    const float2 lap = add2(add2(add2(dv(z0, r0, c0 - 1), dv(z0, r0, c0 + 1)), add2(dv(z0, r0 - 1, c0), dv(z0, r0 + 1, c0))),
                            add2(dv(zm, r0, c0), dv(zp, r0, c0)));
    const float2 pr = mul2(cbh, hc);
    float2 e = fma2(cbh, hc, neg2(pr));
    e = fma2(cbh, lc, e);
    e = fma2(cbl, hc, e);
    const float2 t = add2(e, lap);
    const float2 g_hi = add2(pr, t);
    const float2 bb = sub2(g_hi, pr);
    const float2 g_lo = add2(sub2(pr, sub2(g_hi, bb)), sub2(t, bb));
    const bool uz = interior(s.bc[2], k, n2);
    if (in0) {
      const bool u = unk0 && uz;
      gh[p] = u ? g_hi.x : 0.0f;
      gl[p] = u ? g_lo.x : 0.0f;
    }
    if (in1) {
      const bool u = unk1 && uz;
      gh[p + dj] = u ? g_hi.y : 0.0f;
      gl[p + dj] = u ? g_lo.y : 0.0f;
    }
    __syncthreads();  // the slot of plane k - 1 is staged again as plane k + 2
    const int t0 = zm;
    zm = z0;
    z0 = zp;
    zp = t0;
  }
}

// First differences of G along AXIS at the destination points (fallback for Pade tables wider
// than the term tile holds): d = (gh_{m+1} - gh_m) + (gl_{m+1} - gl_m) at o = m + out_off, 0 at
// the other points.  Indices are 32-bit (n <= 512: at most 513^3 points per component).
template <int AXIS>
__global__ void k_diff3d32(const float* __restrict__ gh, const float* __restrict__ gl, Shape3 ss, float* __restrict__ d,
                           Shape3 sd, int out_off, int M) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  if (x >= sd.n[0] || y >= sd.n[1]) return;
  const int pd = (z * sd.n[1] + y) * sd.n[0] + x;
  const int m = (AXIS == 0 ? x : (AXIS == 1 ? y : z)) - out_off;
  if (m < 0 || m >= M) {
    d[pd] = 0.0f;
    return;
  }
  const int st[3] = {1, ss.n[0], ss.n[0] * ss.n[1]};
  const int cx = AXIS == 0 ? m : x, cy = AXIS == 1 ? m : y, cz = AXIS == 2 ? m : z;
  const int ps = (cz * ss.n[1] + cy) * ss.n[0] + cx;
  d[pd] = (gh[ps + st[AXIS]] - gh[ps]) + (gl[ps + st[AXIS]] - gl[ps]);
}

// y = A^{-1} d along AXIS, then R (+)= sign * y at the unknowns of the destination component.
// Rows away from the line ends use the interior row from constant memory (taps -KB3 .. KB3+1);
// the end rows use the explicit FP32 hi + lo table rows.  Taps are summed farthest first (see
// the 2D curl tile for why the order matters).
template <int AXIS>
__global__ void k_band3d32(const float* __restrict__ d, float* __restrict__ R, Shape3 sd, int out_off, int M,
                           const float* __restrict__ whi, const float* __restrict__ wlo, int K, int B,
                           int all_explicit, float sign, int accumulate) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y, z = blockIdx.z;
  if (x >= sd.n[0] || y >= sd.n[1]) return;
  const int pd = (z * sd.n[1] + y) * sd.n[0] + x;
  const int r = (AXIS == 0 ? x : (AXIS == 1 ? y : z)) - out_off;
  if (!unk3(sd, x, y, z) || r < 0 || r >= M) {
    if (!accumulate) R[pd] = 0.0f;
    return;
  }
  const int stride = AXIS == 0 ? 1 : (AXIS == 1 ? sd.n[0] : sd.n[0] * sd.n[1]);
  const float* dc = d + pd;  // dc[t * stride] = d_{r + t}
  float acc;
  if (!all_explicit && r >= B && r < M - B && r >= KB3 && r + KB3 + 1 < M) {
    acc = c_w3[2 * KB3 + 1] * dc[(KB3 + 1) * stride];
#pragma unroll
    for (int dist = KB3; dist >= 1; --dist) {
      acc = fmaf(c_w3[KB3 + dist], dc[dist * stride], acc);
      acc = fmaf(c_w3[KB3 - dist], dc[-dist * stride], acc);
    }
    acc = fmaf(c_wl3[0], dc[-stride], acc);
    acc = fmaf(c_wl3[2], dc[stride], acc);
    acc = fmaf(c_wl3[1], dc[0], acc);
    acc = fmaf(c_w3[KB3], dc[0], acc);
  } else {
    const float* wh = pade_row_ptr(whi, r, M, K, B, all_explicit);
    const float* wl = pade_row_ptr(wlo, r, M, K, B, all_explicit);
    float lo = 0.0f;
    acc = 0.0f;
    for (int dist = K + 1; dist >= 1; --dist) {
      for (int side = 1; side >= -1; side -= 2) {
        const int mm = r + side * dist, t = mm - r + K;
        if (t < 0 || t > 2 * K + 1 || mm < 0 || mm >= M) continue;
        const float dm = dc[(mm - r) * stride];
        acc = fmaf(__ldg(wh + t), dm, acc);
        lo = fmaf(__ldg(wl + t), dm, lo);
      }
    }
    lo = fmaf(__ldg(wl + K), dc[0], lo);
    acc = fmaf(__ldg(wh + K), dc[0], acc + lo);
  }
  R[pd] = accumulate ? R[pd] + sign * acc : sign * acc;
}

constexpr int T3O = 64;             // band rows per tile
constexpr int K3H = 13;             // reach held in shared memory (table half-width <= 12)
constexpr int D3L = T3O + 2 * K3H;  // differences per line

// Interior row of the band at row r, d[t] = delta_{r - KB3 + t} (t = 0 .. 2 KB3 + 1), taps summed
// farthest first, the lo parts of the three central taps before the central hi tap (rows of a
// run that also holds end rows; whole interior runs take rec_rows3).
__device__ __forceinline__ float band_fast3(const float* d) {
  float acc = c_w3[2 * KB3 + 1] * d[2 * KB3 + 1];
#pragma unroll
  for (int dist = KB3; dist >= 1; --dist) {
    acc = fmaf(c_w3[KB3 + dist], d[KB3 + dist], acc);
    acc = fmaf(c_w3[KB3 - dist], d[KB3 - dist], acc);
  }
  acc = fmaf(c_wl3[0], d[KB3 - 1], acc);
  acc = fmaf(c_wl3[2], d[KB3 + 1], acc);
  acc = fmaf(c_wl3[1], d[KB3], acc);
  return fmaf(c_w3[KB3], d[KB3], acc);
}

// Eight interior rows rb .. rb + 7 of A^{-1} d (v[t] = d_{rb + t}, t = -KR3 - 1 .. 8 + KR3).
// A = (1/24) tridiag(1, 22, 1) = (1 - rho E^-1)(1 - rho E) / (1 - rho)^2 with rho^2 + 22 rho + 1 = 0,
// and by partial fractions 1 / ((1 - rho E^-1)(1 - rho E)) = (F + G - 1) / (1 - rho^2) with
// F = (1 - rho E^-1)^-1, G = (1 - rho E)^-1: A^{-1} d = (1 - rho) / (1 + rho) (f + g - d) for
// the forward recurrence f_i = d_i + rho f_{i-1} and the backward one g_i = d_i + rho g_{i+1}.
// The two are independent chains over d (half the dependent depth of running one after the
// other).  Each starts KR3 + 1 rows outside the eight from the steady state d / (1 - rho), an
// error damped by |rho|^(KR3+1) ~ 4e-10 times the change of d over those rows; every product
// enters through one FMA.
constexpr int KR3 = 6;
template <typename Emit>
__device__ __forceinline__ void rec_rows3(const float* v, Emit emit) {
  const float rho = c_rec3[0], inv1mr = c_rec3[1];
  float fs[8];
  float f = v[-KR3 - 1] * inv1mr;
#pragma unroll
  for (int t = -KR3; t < 8; ++t) {
    f = fmaf(rho, f, v[t]);
    if (t >= 0) fs[t] = f;
  }
  float g = v[8 + KR3] * inv1mr;
#pragma unroll
  for (int t = 7 + KR3; t >= 0; --t) {
    g = fmaf(rho, g, v[t]);
    if (t < 8) {
      const float u = (fs[t] + g) - v[t];
      emit(t, fmaf(c_rec3[2], u, c_rec3[3] * u));
    }
  }
}

// Explicit table row r (hi + lo), dc[t] = delta_{r + t}, taps farthest first as in the interior
// row, hi and lo products summed apart.  The loop is unrolled to the largest half-width the tile
// holds, the taps beyond K predicated off; taps outside the line read the zeros stored there.
__device__ __forceinline__ float band_gen3(const float* dc, int r, int M, const float* __restrict__ whi,
                                           const float* __restrict__ wlo, int K, int B, int all_explicit) {
  const float* wh = pade_row_ptr(whi, r, M, K, B, all_explicit) + K;  // wh[d]: tap of delta_{r + d}
  const float* wl = pade_row_ptr(wlo, r, M, K, B, all_explicit) + K;
  float acc = 0.0f, lo2 = 0.0f;
#pragma unroll
  for (int dist = K3H; dist >= 1; --dist) {
    if (dist <= K + 1) {
      const float d = dc[dist];
      acc = fmaf(__ldg(wh + dist), d, acc);
      lo2 = fmaf(__ldg(wl + dist), d, lo2);
    }
    if (dist <= K) {
      const float d = dc[-dist];
      acc = fmaf(__ldg(wh - dist), d, acc);
      lo2 = fmaf(__ldg(wl - dist), d, lo2);
    }
  }
  lo2 = fmaf(__ldg(wl), dc[0], lo2);
  return fmaf(__ldg(wh), dc[0], acc + lo2);
}

// One Pade term y = A^{-1} D1 G along AXIS, R (+)= sign y, on a tile of T3O band rows r0 ..
// r0 + T3O - 1 of 32 lines along the transverse axis P (y for x lines, x otherwise), at one
// coordinate q of the other transverse axis Q.  The first differences of G over the rows' reach
// (K3H on each side) go to shared memory, a row per line; a thread then takes eight consecutive
// rows of one line (lanes across the lines, so every lane of a warp is at the same rows and the
// end rows of the table take their path together).  x lines are read and written along x by whole
// warps, the results passing through shared memory; y and z lines are read and written with the
// lanes across x.  Runs of rows away from the line ends take the recurrences (rec_rows3); runs
// that hold end rows take the explicit FP32 hi + lo table rows there and the interior band row
// from constant memory elsewhere.  Wall lines
// need no test: G is 0 on them, so y is 0 there.  Without accumulation the first and last tiles of
// a line also write the wall points beyond the band rows (0).
template <int AXIS>
struct TermGeo {
  static constexpr int P = AXIS == 0 ? 1 : 0;  // in-tile transverse axis
  static constexpr int Q = AXIS == 2 ? 1 : 2;  // the other transverse axis
};
constexpr int DP3 = D3L | 1;  // odd row pitch: lanes across the rows are conflict-free

template <int AXIS>
__global__ void __launch_bounds__(256, AXIS == 0 ? 4 : 5) k_term3d32(const float* __restrict__ gh, const float* __restrict__ gl, Shape3 ss,
                                                     float* __restrict__ R, Shape3 sd, int out_off, int M,
                                                     const float* __restrict__ whi, const float* __restrict__ wlo, int K,
                                                     int B, int all_explicit, float sign, int accumulate) {
  constexpr int P = TermGeo<AXIS>::P, Q = TermGeo<AXIS>::Q;
  __shared__ float dd[32 * DP3];
  int tr, p0, q;
  if (AXIS == 0) { tr = blockIdx.x; p0 = blockIdx.y * 32; q = blockIdx.z; }
  else if (AXIS == 1) { p0 = blockIdx.x * 32; tr = blockIdx.y; q = blockIdx.z; }
  else { p0 = blockIdx.x * 32; tr = blockIdx.y; q = blockIdx.z; }  // tiles along z a few blocks apart
  const int r0 = tr * T3O;  // first band row of the tile
  const int st[3] = {1, ss.n[0], ss.n[0] * ss.n[1]};
  const int sdt[3] = {1, sd.n[0], sd.n[0] * sd.n[1]};
  const int nA = sd.n[AXIS], nP = sd.n[P];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool last_tile = r0 + T3O >= M;
  const int mb = r0 - K3H;  // m of difference column 0
  auto fast = [&](int r) { return !all_explicit && r >= B && r < M - B && r >= KB3 && r + KB3 + 1 < M; };
  // x lines: warp w reads and writes lines 4 w .. 4 w + 3 of the tile along x
  float racc[8];  // R at this thread's outputs when accumulating, fetched first
  if (AXIS == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = p0 + 4 * warp + i, ld = p * sdt[P] + q * sdt[Q];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int r = r0 + lane + 32 * c;
        racc[2 * i + c] = (accumulate && p < nP && r < M) ? R[ld + r + out_off] : 0.0f;
      }
    }
    // G at source points mb + lane + 32 c of the warp's four lines, every load issued first
    // (lines past the grid read the last line, unused)
    const int ns = ss.n[0];
    const bool inner = mb >= 0 && mb + 96 <= ns;  // block-uniform: no tests along the line
    float h[4][3], l[4][3];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int pl = min(p0 + 4 * warp + i, nP - 1);
      const float* hr = gh + pl * st[P] + q * st[Q] + mb + lane;
      const float* lr = gl + pl * st[P] + q * st[Q] + mb + lane;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int sidx = mb + lane + 32 * c;
        const bool ok = inner || (sidx >= 0 && sidx < ns);
        h[i][c] = ok ? hr[32 * c] : 0.0f;
        l[i][c] = ok ? lr[32 * c] : 0.0f;
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int ll = 4 * warp + i;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float h1 = __shfl_down_sync(0xffffffffu, h[i][c], 1), l1 = __shfl_down_sync(0xffffffffu, l[i][c], 1);
        const float hn = __shfl_sync(0xffffffffu, c < 2 ? h[i][c < 2 ? c + 1 : 0] : 0.0f, 0);
        const float ln = __shfl_sync(0xffffffffu, c < 2 ? l[i][c < 2 ? c + 1 : 0] : 0.0f, 0);
        if (lane == 31) {
          h1 = hn;
          l1 = ln;
        }
        const int j = lane + 32 * c, m = mb + j;
        if (j < D3L) dd[ll * DP3 + j] = (m >= 0 && m < M) ? (h1 - h[i][c]) + (l1 - l[i][c]) : 0.0f;
      }
    }
  }
  const int p = p0 + lane;  // the line of this thread in the band phase
  const bool live = p < nP;
  const int ob = 8 * warp, rb = r0 + ob;
  const int sA = sdt[AXIS];
  const int ld = p * sdt[P] + q * sdt[Q];
  if (AXIS != 0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) racc[u] = (accumulate && live && rb + u < M) ? R[ld + (rb + u + out_off) * sA] : 0.0f;
    // differences j in [w RJ, (w + 1) RJ) of the lane's line, all loads issued first
    constexpr int RJ = (D3L + 7) / 8;
    const int sa = st[AXIS];
    const int ja = warp * RJ;
    const int pc = live ? p : nP - 1;  // lanes past the tile's lines read the last line, unused
    const float* gph = gh + pc * st[P] + q * st[Q];
    const float* gpl = gl + pc * st[P] + q * st[Q];
    float hv[RJ + 1], lv[RJ + 1];
    float* row = dd + lane * DP3;
    if (mb + ja >= 0 && mb + ja + RJ < M) {
      // the warp's run lies inside the line: no tests (warp-uniform)
      const float* hr = gph + (mb + ja) * sa;
      const float* lr = gpl + (mb + ja) * sa;
#pragma unroll
      for (int i = 0; i <= RJ; ++i) {
        hv[i] = hr[i * sa];
        lv[i] = lr[i * sa];
      }
#pragma unroll
      for (int i = 0; i < RJ; ++i)
        if (ja + i < D3L) row[ja + i] = (hv[i + 1] - hv[i]) + (lv[i + 1] - lv[i]);
    } else {
#pragma unroll
      for (int i = 0; i <= RJ; ++i) {
        const int sidx = mb + ja + i;  // source point
        const bool ok = sidx >= 0 && sidx <= M;
        hv[i] = ok ? gph[sidx * sa] : 0.0f;
        lv[i] = ok ? gpl[sidx * sa] : 0.0f;
      }
#pragma unroll
      for (int i = 0; i < RJ; ++i) {
        const int j = ja + i, m = mb + j;
        if (j < D3L) row[j] = (m >= 0 && m < M) ? (hv[i + 1] - hv[i]) + (lv[i + 1] - lv[i]) : 0.0f;
      }
    }
  }
  __syncthreads();
  if (AXIS != 0) {
    // y and z lines: each result goes straight to R
    if (!live) return;
    const float* row = dd + lane * DP3;
    float* Rp = R + ld + (rb + out_off) * sA;
    auto put = [&](int u, float v) { Rp[u * sA] = accumulate ? racc[u] + sign * v : sign * v; };
    if (rb + 7 < M && fast(rb) && fast(rb + 7)) {
      rec_rows3(row + ob + K3H, put);
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int rr = rb + u;
        const float* dc = row + rr - r0 + K3H;
        if (rr < M) put(u, fast(rr) ? band_fast3(dc - KB3) : band_gen3(dc, rr, M, whi, wlo, K, B, all_explicit));
      }
    }
    if (!accumulate && warp == 0) {
      if (tr == 0)
        for (int od = 0; od < out_off; ++od) R[ld + od * sA] = 0.0f;
      if (last_tile)
        for (int od = M + out_off; od < nA; ++od) R[ld + od * sA] = 0.0f;
    }
    return;
  }
  float y[8];
  if (live) {
    const float* row = dd + lane * DP3;
    if (rb + 7 < M && fast(rb) && fast(rb + 7)) {
      rec_rows3(row + ob + K3H, [&](int u, float v) { y[u] = v; });
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int rr = rb + u;
        const float* dc = row + rr - r0 + K3H;
        y[u] = rr >= M ? 0.0f : (fast(rr) ? band_fast3(dc - KB3) : band_gen3(dc, rr, M, whi, wlo, K, B, all_explicit));
      }
    }
  }
  // x lines: y through shared memory (row = line, column = band row), written along x
  __syncthreads();
  if (live) {
#pragma unroll
    for (int u = 0; u < 8; ++u) dd[lane * DP3 + ob + u] = y[u];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int ll = 4 * warp + i, pl = p0 + ll;
    if (pl >= nP) break;
    const int ldl = pl * sdt[P] + q * sdt[Q];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int o = lane + 32 * c, r = r0 + o;
      if (r < M) {
        const float yv = dd[ll * DP3 + o];
        R[ldl + r + out_off] = accumulate ? racc[2 * i + c] + sign * yv : sign * yv;
      }
    }
    if (!accumulate) {
      if (tr == 0 && lane < out_off) R[ldl + lane] = 0.0f;
      if (last_tile && M + out_off + lane < nA) R[ldl + M + out_off + lane] = 0.0f;
    }
  }
}

// One sweep of the FP32 Richardson iteration on 6 h^2 P1 x = b (6h^2 P1 = d - 6(Lx + Ly + Lz)
// - (LxLy + LyLz + LzLx), d = 6 c1 h^2 as hi + lo), x_{k+1} = x_k + omega (b - 6 h^2 P1 x_k) from
// x_1 = omega b.  FIRST: the sweep from x_1, read as omega b.  LAST: the state (hi, lo) += s x +
// s corr (two separate error-free additions) instead of writing x.
// A block of SWX x SWT threads takes a tile of SWX x SWY points and marches SWZ planes along z;
// a thread takes rows j and j + SWT of one column, and every operation acts on that pair at once
// (paired FP32 instructions).  The iterate on planes z-1, z, z+1 over the tile with a one-point
// halo in x and y sits in a ring in shared memory as pairs: pair row pr holds tile rows pr - 1 and
// pr - 1 + SWT, so a shift in x or y is the same shift of both halves.  The next plane is
// fetched into registers, and the per-point operands (b, the state) of the next plane too, while
// the current one is computed.  Tiles cover the unknowns only: halo points past a Neumann end
// are its even ghosts (clamped), walls of a Dirichlet axis are taken as zeros without a load, so
// no sweep reads or writes a wall point.
constexpr int SWX = 32, SWT = 8, SWY = 2 * SWT, SWZ = 16;
constexpr int SWXP = SWX + 2, SWRP = SWT + 2;  // pair rows of a staged plane
constexpr int SWN = SWRP * SWXP;               // staged pairs per plane
static_assert(SWN <= 2 * SWX * SWT, "two staged pairs per thread");

template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(SWX * SWT, LAST ? 4 : 5) k_sweep3d32(const float* __restrict__ b, const float* __restrict__ xin,
                                                            float* __restrict__ xout, Shape3 s, float d_hi, float d_lo,
                                                            float omega, float* __restrict__ shi,
                                                            float* __restrict__ slo, float s_hi, float s_lo) {
  __shared__ float2 xs[3][SWRP][SWXP];
  const int n0 = s.n[0], n1 = s.n[1], n2 = s.n[2];
  // tiles cover the unknowns only: index u along an axis is point u + lo (lo = 1 on a Dirichlet
  // axis, whose walls are read as the zeros they hold, without a load)
  const int lo0 = s.bc[0] == DIR, lo1 = s.bc[1] == DIR, lo2 = s.bc[2] == DIR;
  const int nu0 = n0 - 2 * lo0, nu1 = n1 - 2 * lo1, nu2 = n2 - 2 * lo2;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int iu = blockIdx.x * SWX + tx, ju = blockIdx.y * SWY + ty;  // rows ju and ju + SWT
  const int k0 = blockIdx.z * SWZ, k1 = min(k0 + SWZ, nu2);
  const bool in0 = iu < nu0 && ju < nu1, in1 = iu < nu0 && ju + SWT < nu1;
  const int sz = n0 * n1;
  const float* X0 = FIRST ? b : xin;
  // position q along an axis of n points: false where the value is a wall zero, else the point
  // (even ghosts of a Neumann axis clamped)
  auto place = [](int q, int n, int dir, int* at) {
    if (dir) {
      *at = q;
      return q > 0 && q < n - 1;
    }
    *at = clampi(q, n);
    return true;
  };
  // plane loader: thread t stages pairs t and t + 256 (< SWN), at offsets fixed for the march
  const int t1 = ty * SWX + tx, t2 = t1 + SWX * SWT;
  const bool has2 = t2 < SWN;
  auto pair_off = [&](int e, int half, bool* live) {
    const int row = e / SWXP, col = e - row * SWXP;
    int y, x;
    const bool ly = place(lo1 + blockIdx.y * SWY + row - 1 + half * SWT, n1, lo1, &y);
    const bool lx = place(lo0 + blockIdx.x * SWX + col - 1, n0, lo0, &x);
    *live = ly && lx;
    return *live ? y * n0 + x : 0;
  };
  bool v1a, v1b, v2a, v2b;
  const int o1a = pair_off(t1, 0, &v1a), o1b = pair_off(t1, 1, &v1b);
  const int o2a = pair_off(has2 ? t2 : t1, 0, &v2a), o2b = pair_off(has2 ? t2 : t1, 1, &v2b);
  float2 ra = make_float2(0.0f, 0.0f), rb = make_float2(0.0f, 0.0f);
  auto fetch = [&](int ku) {  // plane of unknown index ku (-1 .. nu2)
    int z;
    const bool lz = place(lo2 + ku, n2, lo2, &z);
    const float* P = X0 + (lz ? z : 0) * sz;
    ra = make_float2(lz && v1a ? P[o1a] : 0.0f, lz && v1b ? P[o1b] : 0.0f);
    if (has2) rb = make_float2(lz && v2a ? P[o2a] : 0.0f, lz && v2b ? P[o2b] : 0.0f);
  };
  const float2 om2 = bc2(omega);
  auto stage = [&](float2(*pl)[SWXP]) {
    float2* f = &pl[0][0];
    f[t1] = FIRST ? mul2(om2, ra) : ra;
    if (has2) f[t2] = FIRST ? mul2(om2, rb) : rb;
  };
  // per-point operands of the next plane
  float2 bq = make_float2(0.0f, 0.0f), hq = bq, lq = bq;
  const int dj = SWT * n0;
  auto fetch_pt = [&](int p) {
    if (in0) {
      bq.x = b[p];
      if (LAST) {
        hq.x = shi[p];
        lq.x = slo[p];
      }
    }
    if (in1) {
      bq.y = b[p + dj];
      if (LAST) {
        hq.y = shi[p + dj];
        lq.y = slo[p + dj];
      }
    }
  };
  float2(*Zm)[SWXP] = xs[0];
  float2(*Z0)[SWXP] = xs[1];
  float2(*Zp)[SWXP] = xs[2];
  fetch(k0 - 1);
  stage(Zm);
  fetch(k0);
  stage(Z0);
  fetch(k0 + 1);
  int p = (lo2 + k0) * sz + (lo1 + ju) * n0 + lo0 + iu;
  fetch_pt(p);
  const int c0 = tx + 1, r0 = ty + 1;  // halo coordinates in the pair layout
  const float2 m2 = bc2(-2.0f), m6 = bc2(-6.0f), ndh2 = bc2(-d_hi), ndl2 = bc2(-d_lo), sh2 = bc2(s_hi), sl2 = bc2(s_lo);
  for (int k = k0; k < k1; ++k, p += sz) {
    stage(Zp);
    __syncthreads();
    if (k + 1 < k1) fetch(k + 2);
    const float2 bc = bq, hc = hq, lc = lq;
    if (k + 1 < k1) fetch_pt(p + sz);
    // second differences as a + b - 2 v: the residual's dominant term d x enters exactly, so
    // the rounding of these sums is far below an ulp of the residual
    auto LX = [&](const float2(*Pl)[SWXP], int rr) { return fma2(m2, Pl[rr][c0], add2(Pl[rr][c0 - 1], Pl[rr][c0 + 1])); };
    auto LY = [&](const float2(*Pl)[SWXP]) { return fma2(m2, Pl[r0][c0], add2(Pl[r0 - 1][c0], Pl[r0 + 1][c0])); };
    const float2 x = Z0[r0][c0];
    const float2 lx = LX(Z0, r0), ly = LY(Z0);
    const float2 lz = fma2(m2, x, add2(Zm[r0][c0], Zp[r0][c0]));
    const float2 lxly = fma2(m2, lx, add2(LX(Z0, r0 - 1), LX(Z0, r0 + 1)));
    const float2 lxlz = fma2(m2, lx, add2(LX(Zm, r0), LX(Zp, r0)));
    const float2 lylz = fma2(m2, ly, add2(LY(Zm), LY(Zp)));
    const float2 rest = fma2(m6, add2(add2(lx, ly), lz), neg2(add2(add2(lxly, lylz), lxlz)));
    // b - d x with the product exact: b - d_hi x, then - d_lo x, one rounding each
    const float2 res = sub2(fma2(ndl2, x, fma2(ndh2, x, bc)), rest);
    if (LAST) {
      const float2 corr = mul2(om2, res);
      float2 h = hc, l = lc;
      ff_add_scaled3_2(h, l, x, sh2, sl2);
      ff_add_scaled3_2(h, l, corr, sh2, sl2);
      if (in0) {
        shi[p] = h.x;
        slo[p] = l.x;
      }
      if (in1) {
        shi[p + dj] = h.y;
        slo[p + dj] = l.y;
      }
    } else {
      const float2 xn = fma2(om2, res, x);
      if (in0) xout[p] = xn.x;
      if (in1) xout[p + dj] = xn.y;
    }
    __syncthreads();  // the slot of plane k - 1 is staged again as plane k + 2
    float2(*t)[SWXP] = Zm;
    Zm = Z0;
    Z0 = Zp;
    Zp = t;
  }
}

// S = 1: the single iterate x = omega b is the correction, state += s omega b.
__global__ void k_single3d32(const float* __restrict__ b, Shape3 s, float omega, float* __restrict__ shi,
                             float* __restrict__ slo, float s_hi, float s_lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= s.n[0] || j >= s.n[1] || !unk3(s, i, j, k)) return;
  const int p = (k * s.n[1] + j) * s.n[0] + i;
  float h = shi[p], l = slo[p];
  ff_add_scaled3(h, l, omega * b[p], s_hi, s_lo);
  shi[p] = h;
  slo[p] = l;
}

dim3 sweep_grid3(const Shape3& s) {  // tiles over the unknowns
  const int nu0 = s.n[0] - 2 * (s.bc[0] == DIR), nu1 = s.n[1] - 2 * (s.bc[1] == DIR), nu2 = s.n[2] - 2 * (s.bc[2] == DIR);
  return dim3((nu0 + SWX - 1) / SWX, (nu1 + SWY - 1) / SWY, (nu2 + SWZ - 1) / SWZ);
}

__global__ void k_split3(const double* __restrict__ v, float* __restrict__ hi, float* __restrict__ lo, size_t n) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float h = (float)v[p];
  hi[p] = h;
  lo[p] = (float)(v[p] - (double)h);
}

__global__ void k_join3(const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ v, size_t n) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  v[p] = (double)hi[p] + (double)lo[p];
}

// ---------------------------------------------------------------------------------------
// Host launchers

const dim3 kBlk(32, 8, 1);

void filter3d64(ms_grid* g, int c, const double* u, double* G) {
  const Shape3& s = g->g3->sh[c];
  k_filter3d64<<<grid3(s, kBlk), kBlk, 0, g->stream>>>(u, G, s, g->beta);
  prof_mark(g, KK_FILTER3D64, 16.0 * (double)s.size());
}

// out (+)= scale * delta_axis(in), in of component cs, out of component cd
void pade3d64(ms_grid* g, int axis, int cs, int cd, const double* in, double* out, double scale, int accumulate) {
  const Shape3& si = g->g3->sh[cs];
  const Shape3& so = g->g3->sh[cd];
  const int kind = (si.bc[axis] == NEU) ? HALF_TO_NODE : NODE_TO_HALF;
  const PadeTable& t = g->pade[kind];
  const int off = (kind == HALF_TO_NODE) ? 1 : 0;
  const dim3 grd = grid3(so, kBlk);
  if (axis == 0)
    k_pade3d64<0><<<grd, kBlk, 0, g->stream>>>(in, out, so, si, t.d_w, t.rows, t.n_in, t.left, t.K, t.B,
                                                t.all_explicit, off, scale, accumulate);
  else if (axis == 1)
    k_pade3d64<1><<<grd, kBlk, 0, g->stream>>>(in, out, so, si, t.d_w, t.rows, t.n_in, t.left, t.K, t.B,
                                                t.all_explicit, off, scale, accumulate);
  else
    k_pade3d64<2><<<grd, kBlk, 0, g->stream>>>(in, out, so, si, t.d_w, t.rows, t.n_in, t.left, t.K, t.B,
                                                t.all_explicit, off, scale, accumulate);
  prof_mark(g, KK_PADE3D64, 8.0 * ((double)si.size() + (accumulate ? 2.0 : 1.0) * (double)so.size()));
}

// x = P1^{-1} b for component c; the last sweep adds upd_scale * x to upd.
void solve3d64(ms_grid* g, int c, const double* b, double* upd, double upd_scale, int* nl) {
  const Shape3& s = g->g3->sh[c];
  const double c1h2 = g->c1 * g->h * g->h, om = 2.0 / (2.0 * c1h2 + 16.0 / 3.0), h2 = g->h * g->h;
  double* buf[2] = {g->g3->s64[4], g->g3->s64[5]};
  const double* xin = nullptr;
  for (int k = 0; k < g->p1_sweeps; ++k) {
    const bool last = (k == g->p1_sweeps - 1);
    double* xo = last ? g->g3->s64[6] : buf[k & 1];
    k_sweep3d64<<<grid3(s, kBlk), kBlk, 0, g->stream>>>(b, xin, xo, s, c1h2, om, h2, k == 0, last ? upd : nullptr,
                                                         upd_scale);
    prof_mark(g, KK_SWEEP3D64, 8.0 * (double)s.size() * ((k == 0 ? 2 : 3) + (last ? 2 : 0)));
    xin = xo;
  }
  *nl += g->p1_sweeps;
}

ms_status step3d64(ms_grid* g) {
  Grid3D* G3 = g->g3;
  int nl = 0;
  double** G = G3->s64;  // G[0..2]
  double* R = G3->s64[3];
  const double s_he = g->kappa2 * g->Z / g->h, s_eh = g->kappa2 / (g->Z * g->h);
  if (g->src3) {  // time factors of this step's source terms
    src3_time(g);
    prof_mark(g, KK_SRC, 0.0);
    nl += 1;
  }
  // Step 1: R_e = kappa^2 Z (d_{e+1} G_{e+2} - d_{e+2} G_{e+1}) on E_e, P1 E* = R, E += h_tau E*
  for (int c = 0; c < 3; ++c) filter3d64(g, 3 + c, G3->f64[3 + c], G[c]);
  nl += 3;
  for (int e = 0; e < 3; ++e) {
    const int p1 = (e + 1) % 3, p2 = (e + 2) % 3;
    pade3d64(g, p1, 3 + p2, e, G[p2], R, s_he, 0);
    pade3d64(g, p2, 3 + p1, e, G[p1], R, -s_he, 1);
    nl += 2;
    if (g->src3) {
      src3_add(g, e, R);
      prof_mark(g, KK_SRC, 16.0 * (double)G3->sh[e].size());
      nl += 1;
    }
    solve3d64(g, e, R, G3->f64[e], g->ht, &nl);
  }
  // Step 2: R_h = -(kappa^2/Z)(d_{h+1} G_{E,h+2} - d_{h+2} G_{E,h+1}) on H_h
  for (int c = 0; c < 3; ++c) filter3d64(g, c, G3->f64[c], G[c]);
  nl += 3;
  for (int hc = 0; hc < 3; ++hc) {
    const int p1 = (hc + 1) % 3, p2 = (hc + 2) % 3;
    pade3d64(g, p1, p2, 3 + hc, G[p2], R, -s_eh, 0);
    pade3d64(g, p2, p1, 3 + hc, G[p1], R, s_eh, 1);
    nl += 2;
    if (g->src3) {
      src3_add(g, 3 + hc, R);
      prof_mark(g, KK_SRC, 16.0 * (double)G3->sh[3 + hc].size());
      nl += 1;
    }
    solve3d64(g, 3 + hc, R, G3->f64[3 + hc], g->ht, &nl);
  }
  if (g->src3) {  // the device step index advances with the step
    launch_tick(g);
    prof_mark(g, KK_SRC, 0.0);
    nl += 1;
  }
  g->launches_per_step = nl;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail3(MS_ECUDA, std::string("3D FP64 step: ") + cudaGetErrorString(e));
  return MS_OK;
}

// FP32_REFINED: G (hi, lo) = 12 beta u + L u of component c into the filter buffers of slot c % 3.
void filter3d32(ms_grid* g, int c, float cb_hi, float cb_lo) {
  Grid3D* G3 = g->g3;
  const Shape3& s = G3->sh[c];
  const dim3 grd((s.n[0] + FTX - 1) / FTX, (s.n[1] + FTY - 1) / FTY, (s.n[2] + FZ3 - 1) / FZ3), blk(FTX, FTT, 1);
  k_ffilt3d32<<<grd, blk, 0, g->stream>>>(G3->hi[c], G3->lo[c], s, G3->gh[c % 3], G3->gl[c % 3], cb_hi, cb_lo);
  // state hi + lo in, G hi + lo out
  prof_mark(g, KK_FILT3D32, 16.0 * (double)s.size());
}

// FP32_REFINED: one Pade term y = A^{-1} D1 G of source component cs (G made by filter3d32) along
// axis, added with `sign` into R on component cd.  Returns the number of launches issued.
int term3d32(ms_grid* g, int axis, int cs, int cd, float sign, int accumulate) {
  Grid3D* G3 = g->g3;
  const Shape3& ss = G3->sh[cs];
  const Shape3& sd = G3->sh[cd];
  const int kind = (ss.bc[axis] == NEU) ? HALF_TO_NODE : NODE_TO_HALF;
  const PadeTable& t = g->pade32[kind];
  const int off = (kind == HALF_TO_NODE) ? 1 : 0;
  const float* gh = G3->gh[cs % 3];
  const float* gl = G3->gl[cs % 3];
  float* R = G3->s32[1];
  if (t.K + 1 <= K3H) {
    // differences and band in one tiled kernel
    const int nt = (t.M + T3O - 1) / T3O;
    if (axis == 0) {
      const dim3 grd(nt, (sd.n[1] + 31) / 32, sd.n[2]);
      k_term3d32<0><<<grd, 256, 0, g->stream>>>(gh, gl, ss, R, sd, off, t.M, t.d_whi, t.d_wlo, t.K, t.B, t.all_explicit,
                                                 sign, accumulate);
    } else if (axis == 1) {
      const dim3 grd((sd.n[0] + 31) / 32, nt, sd.n[2]);
      k_term3d32<1><<<grd, 256, 0, g->stream>>>(gh, gl, ss, R, sd, off, t.M, t.d_whi, t.d_wlo, t.K, t.B, t.all_explicit,
                                                 sign, accumulate);
    } else {
      const dim3 grd((sd.n[0] + 31) / 32, nt, sd.n[1]);
      k_term3d32<2><<<grd, 256, 0, g->stream>>>(gh, gl, ss, R, sd, off, t.M, t.d_whi, t.d_wlo, t.K, t.B, t.all_explicit,
                                                 sign, accumulate);
    }
    // G hi + lo in, R out (read too when accumulating)
    prof_mark(g, KK_TERM3D32, 4.0 * (2.0 * (double)ss.size() + (accumulate ? 2.0 : 1.0) * (double)sd.size()));
    return 1;
  }
  float* d = G3->s32[0];
  const dim3 grd = grid3(sd, kBlk);
  if (axis == 0)
    k_diff3d32<0><<<grd, kBlk, 0, g->stream>>>(gh, gl, ss, d, sd, off, t.M);
  else if (axis == 1)
    k_diff3d32<1><<<grd, kBlk, 0, g->stream>>>(gh, gl, ss, d, sd, off, t.M);
  else
    k_diff3d32<2><<<grd, kBlk, 0, g->stream>>>(gh, gl, ss, d, sd, off, t.M);
  if (axis == 0)
    k_band3d32<0><<<grd, kBlk, 0, g->stream>>>(d, R, sd, off, t.M, t.d_whi, t.d_wlo, t.K, t.B, t.all_explicit, sign,
                                                accumulate);
  else if (axis == 1)
    k_band3d32<1><<<grd, kBlk, 0, g->stream>>>(d, R, sd, off, t.M, t.d_whi, t.d_wlo, t.K, t.B, t.all_explicit, sign,
                                                accumulate);
  else
    k_band3d32<2><<<grd, kBlk, 0, g->stream>>>(d, R, sd, off, t.M, t.d_whi, t.d_wlo, t.K, t.B, t.all_explicit, sign,
                                                accumulate);
  // G hi + lo in, d out; d in, R out (read too when accumulating)
  prof_mark(g, KK_BAND3D32,
            4.0 * (2.0 * (double)ss.size() + (double)sd.size()) + 4.0 * (double)sd.size() * (accumulate ? 3.0 : 2.0));
  return 2;
}

// Transform solve (tensor cores) of component c followed by ts_sweeps Richardson sweeps with the
// exact residual, the last of which updates the state.
void solve3d32_ts(ms_grid* g, int c, float d_hi, float d_lo, float omega, float s_hi, float s_lo, int* nl) {
  Grid3D* G3 = g->g3;
  const Shape3& s = G3->sh[c];
  const float* b = G3->s32[1];
  float* buf[2] = {G3->s32[2], G3->s32[3]};
  *nl += ts_solve(*G3->ts, s, b, buf[0], 6.0f * (float)(g->c1 * g->h * g->h), g->stream, g);
  const dim3 grd = sweep_grid3(s), blk(SWX, SWT, 1);
  const int R = G3->ts_sweeps;
  for (int k = 0; k < R; ++k) {
    const float* xin = buf[k & 1];
    float* xo = buf[(k + 1) & 1];
    if (k == R - 1)
      k_sweep3d32<false, true><<<grd, blk, 0, g->stream>>>(b, xin, xo, s, d_hi, d_lo, omega, G3->hi[c], G3->lo[c],
                                                           s_hi, s_lo);
    else
      k_sweep3d32<false, false><<<grd, blk, 0, g->stream>>>(b, xin, xo, s, d_hi, d_lo, omega, G3->hi[c], G3->lo[c],
                                                            s_hi, s_lo);
    prof_mark(g, KK_SWEEP3D32, 4.0 * (double)s.size() * (2.0 + (k == R - 1 ? 4.0 : 1.0)));
  }
  *nl += R;
}

void solve3d32(ms_grid* g, int c, float d_hi, float d_lo, float omega, float s_hi, float s_lo, int S, int* nl) {
  Grid3D* G3 = g->g3;
  if (G3->solver == MS_SOLVER_TRANSFORM_TC) {
    solve3d32_ts(g, c, d_hi, d_lo, omega, s_hi, s_lo, nl);
    return;
  }
  const Shape3& s = G3->sh[c];
  const float* b = G3->s32[1];
  float* buf[2] = {G3->s32[2], G3->s32[3]};
  // launch k (k = 1 .. S-1, or one launch when S = 1) produces iterate k + 1 from iterate k
  const float* xin = nullptr;
  const int L = S > 1 ? S - 1 : 1;
  for (int k = 0; k < L; ++k) {
    const bool last = (k == L - 1);
    float* xo = buf[k & 1];
    const dim3 grd = sweep_grid3(s), blk(SWX, SWT, 1);
    float* hi = G3->hi[c];
    float* lo = G3->lo[c];
    if (S == 1)
      k_single3d32<<<grid3(s, kBlk), kBlk, 0, g->stream>>>(b, s, omega, hi, lo, s_hi, s_lo);
    else if (k == 0 && last)
      k_sweep3d32<true, true><<<grd, blk, 0, g->stream>>>(b, xin, xo, s, d_hi, d_lo, omega, hi, lo, s_hi, s_lo);
    else if (k == 0)
      k_sweep3d32<true, false><<<grd, blk, 0, g->stream>>>(b, xin, xo, s, d_hi, d_lo, omega, hi, lo, s_hi, s_lo);
    else if (last)
      k_sweep3d32<false, true><<<grd, blk, 0, g->stream>>>(b, xin, xo, s, d_hi, d_lo, omega, hi, lo, s_hi, s_lo);
    else
      k_sweep3d32<false, false><<<grd, blk, 0, g->stream>>>(b, xin, xo, s, d_hi, d_lo, omega, hi, lo, s_hi, s_lo);
    prof_mark(g, KK_SWEEP3D32, 4.0 * (double)s.size() * ((k == 0 ? 1.0 : 2.0) + (last ? 4.0 : 1.0)));
    xin = xo;
  }
  *nl += L;
}

ms_status step3d32(ms_grid* g) {
  const MixedConsts k = mixed_consts(g);
  int nl = 0;
  Grid3D* G3 = g->g3;
  if (g->src3) {
    src3_time(g);
    prof_mark(g, KK_SRC, 0.0);
    nl += 1;
  }
  auto add_src = [&](int c) {  // source term in the units of b, before the solve of component c
    if (!g->src3) return;
    src3_add(g, c, G3->s32[1]);
    prof_mark(g, KK_SRC, 8.0 * (double)G3->sh[c].size());
    nl += 1;
  };
  // Step 1: G~ of H_x, H_y, H_z, then per E component its two Pade terms and its solve
  for (int c = 3; c < 6; ++c) filter3d32(g, c, k.cb_hi, k.cb_lo);
  nl += 3;
  for (int e = 0; e < 3; ++e) {
    const int p1 = (e + 1) % 3, p2 = (e + 2) % 3;
    nl += term3d32(g, p1, 3 + p2, e, 1.0f, 0);
    nl += term3d32(g, p2, 3 + p1, e, -1.0f, 1);
    add_src(e);
    solve3d32(g, e, k.d_hi, k.d_lo, k.omega, k.sE_hi, k.sE_lo, k.S, &nl);
  }
  // Step 2: G~ of the updated E components, then per H component
  for (int c = 0; c < 3; ++c) filter3d32(g, c, k.cb_hi, k.cb_lo);
  nl += 3;
  for (int hc = 0; hc < 3; ++hc) {
    const int p1 = (hc + 1) % 3, p2 = (hc + 2) % 3;
    nl += term3d32(g, p1, p2, 3 + hc, -1.0f, 0);
    nl += term3d32(g, p2, p1, 3 + hc, 1.0f, 1);
    add_src(3 + hc);
    solve3d32(g, 3 + hc, k.d_hi, k.d_lo, k.omega, k.sH_hi, k.sH_lo, k.S, &nl);
  }
  if (g->src3) {
    launch_tick(g);
    prof_mark(g, KK_SRC, 0.0);
    nl += 1;
  }
  g->launches_per_step = nl;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail3(MS_ECUDA, std::string("3D FP32 step: ") + cudaGetErrorString(e));
  return MS_OK;
}

// Largest |h_tau lambda|^2 / 4 over the 3D Fourier symbol at CFL number r (units h = 1).
double max_amp2_3d(double r) {
  const double k2 = 24.0 / (r * r), beta = 1.0 + 2.0 / (r * r);
  const int n = 48;
  std::vector<double> mu(n), dd(n);
  for (int a = 0; a < n; ++a) {
    const double t = M_PI * (a + 1) / n;
    mu[a] = 4.0 * std::sin(t / 2) * std::sin(t / 2);
    const double d = 2.0 * std::sin(t / 2) * 12.0 / (11.0 + std::cos(t));
    dd[a] = d * d;
  }
  double worst = 0.0;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c) {
        const double s1 = mu[a] + mu[b] + mu[c], s2 = mu[a] * mu[b] + mu[b] * mu[c] + mu[c] * mu[a];
        const double gg = k2 * (beta - s1 / 12.0) / (k2 * beta + s1 - s2 / 6.0);
        const double v = r * r * gg * gg * (dd[a] + dd[b] + dd[c]);
        if (v > worst) worst = v;
      }
  return worst;
}

// Interior row of A^{-1} in closed form (long double), split hi + lo, and the constants of its
// recurrences, into constant memory.
int upload_band_row() {
  const long double rho = -11.0L + std::sqrt(120.0L);
  float w[2 * KB3 + 2], wl[3];
  for (int t = 0; t < 2 * KB3 + 2; ++t) {
    const int dd = t - KB3;
    long double v = 24.0L * (-rho) / (1.0L - rho * rho);
    for (int q = 0; q < (dd < 0 ? -dd : dd); ++q) v *= rho;
    w[t] = (float)v;
    if (dd >= -1 && dd <= 1) wl[dd + 1] = (float)(v - (long double)w[t]);
  }
  if (cudaMemcpyToSymbol(c_w3, w, sizeof w) != cudaSuccess || cudaMemcpyToSymbol(c_wl3, wl, sizeof wl) != cudaSuccess)
    return -1;
  const float rho_f = (float)rho;
  const long double one_m = 1.0L - (long double)rho_f;
  const long double scale = one_m / (1.0L + (long double)rho_f);
  float rec[4];
  rec[0] = rho_f;
  rec[1] = (float)(1.0L / one_m);
  rec[2] = (float)scale;
  rec[3] = (float)(scale - (long double)rec[2]);
  if (cudaMemcpyToSymbol(c_rec3, rec, sizeof rec) != cudaSuccess) return -1;
  return 0;
}

template <typename T>
ms_status alloc3(T** p, size_t n) {
  cudaError_t e = dev_malloc((void**)p, n * sizeof(T) + 256);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail3(MS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return MS_OK;
}

ms_status store3(ms_grid* g, int c, const double* dev) {
  Grid3D* G3 = g->g3;
  const Shape3& s = G3->sh[c];
  if (g->desc.precision == MS_FP64) {
    if (dev != G3->f64[c])
      MS3_CUDA(cudaMemcpyAsync(G3->f64[c], dev, s.size() * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    k_zero_walls3d64<<<grid3(s, kBlk), kBlk, 0, g->stream>>>(G3->f64[c], s);
  } else {
    double* tmp = G3->s64[0];
    if (dev != tmp) MS3_CUDA(cudaMemcpyAsync(tmp, dev, s.size() * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    k_zero_walls3d64<<<grid3(s, kBlk), kBlk, 0, g->stream>>>(tmp, s);
    k_split3<<<(unsigned)((s.size() + 255) / 256), 256, 0, g->stream>>>(tmp, G3->hi[c], G3->lo[c], s.size());
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail3(MS_ECUDA, std::string("store: ") + cudaGetErrorString(e));
  return MS_OK;
}

// FP64 view of component c: the FP64 array, or hi + lo joined into dst.
const double* view3(ms_grid* g, int c, double* dst) {
  Grid3D* G3 = g->g3;
  if (g->desc.precision == MS_FP64) return G3->f64[c];
  const size_t n = G3->sh[c].size();
  k_join3<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(G3->hi[c], G3->lo[c], dst, n);
  return dst;
}

// Exact modes (component c) into out, t_E / t_H (see the oracle's mode: sine on node axes,
// cosine on half axes; H = -(1/(Z omega)) curl(E shape) sin(omega t)).
ms_status exact3(ms_grid* g, const ms_mode3* modes, int nm, double tE, double tH, int c, double* out) {
  const int N = g->N;
  const Shape3& s = g->g3->sh[c];
  std::vector<double> host;
  const size_t ox = 0, oy = (size_t)nm * s.n[0], oz = oy + (size_t)nm * s.n[1], oc = oz + (size_t)nm * s.n[2];
  host.assign(oc + nm, 0.0);
  auto sin_node = [&](int k, int i) {
    if (i == 0 || i == N) return 0.0;
    long q = ((long)k * i) % (2L * N);
    return std::sin(M_PI * (double)q / N);
  };
  auto cos_half = [&](int k, int i) {
    long q = ((long)k * (2L * i + 1)) % (4L * N);
    return std::cos(M_PI * (double)q / (2.0 * N));
  };
  for (int q = 0; q < nm; ++q) {
    const int kk[3] = {modes[q].m, modes[q].n, modes[q].p};
    const size_t off[3] = {ox, oy, oz};
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < s.n[a]; ++i)
        host[off[a] + (size_t)q * s.n[a] + i] = (s.bc[a] == DIR) ? sin_node(kk[a], i) : cos_half(kk[a], i);
    const double a = M_PI * kk[0], b = M_PI * kk[1], cc = M_PI * kk[2];
    const double w = std::sqrt(a * a + b * b + cc * cc);
    const double Ax = modes[q].ax, Ay = modes[q].ay, Az = modes[q].az;
    const double ce = std::cos(w * tE), sh = -std::sin(w * tH) / (g->Z * w);
    const double amp[6] = {Ax * ce, Ay * ce, Az * ce, sh * (Az * b - Ay * cc), sh * (Ax * cc - Az * a),
                           sh * (Ay * a - Ax * b)};
    host[oc + q] = amp[c];
  }
  if (host.size() > g->modetab_cap) {
    dev_free(g->d_modetab);
    g->d_modetab = nullptr;
    g->modetab_cap = 0;
    MS3_TRY(alloc3(&g->d_modetab, host.size()));
    g->modetab_cap = host.size();
  }
  MS3_CUDA(cudaMemcpyAsync(g->d_modetab, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  k_mode_field3<<<grid3(s, kBlk), kBlk, 0, g->stream>>>(out, s, g->d_modetab + ox, g->d_modetab + oy,
                                                         g->d_modetab + oz, g->d_modetab + oc, nm);
  MS3_CUDA(cudaGetLastError());
  MS3_CUDA(cudaStreamSynchronize(g->stream));  // the host table is released on return
  return MS_OK;
}

ms_status check_modes3(const ms_mode3* modes, int nm) {
  if (nm < 0 || (nm > 0 && !modes)) return fail3(MS_EINVAL, "invalid modes");
  for (int q = 0; q < nm; ++q) {
    const ms_mode3& m = modes[q];
    if (m.m < 1 || m.n < 1 || m.p < 1) return fail3(MS_EINVAL, "mode indices must be >= 1");
    const double dot = m.ax * m.m + m.ay * m.n + m.az * m.p;
    const double scale = std::fabs(m.ax * m.m) + std::fabs(m.ay * m.n) + std::fabs(m.az * m.p);
    if (std::fabs(dot) > 1e-12 * (scale > 0 ? scale : 1.0))
      return fail3(MS_EINVAL, "mode polarisation must satisfy A . (m, n, p) = 0 (divergence-free E)");
  }
  return MS_OK;
}

}  // namespace

// Rows of 3D sources: indices >= 0 with at least two >= 1, (ax, ay, az) . (m, n, p) = 0, finite
// values; off resonance (omega^2 != pi^2 |k|^2) when a driven solution is asked for.
ms_status check_sources3(const ms_source3* src, int nsrc, bool need_off_resonance) {
  if (nsrc < 0 || nsrc > 64 || (nsrc > 0 && !src)) return fail3(MS_EINVAL, "invalid sources (0 <= nsrc <= 64)");
  for (int q = 0; q < nsrc; ++q) {
    const ms_source3& s = src[q];
    if (s.m < 0 || s.n < 0 || s.p < 0 || s.m > 1000000 || s.n > 1000000 || s.p > 1000000)
      return fail3(MS_EINVAL, "source indices must be in [0, 1e6]");
    if ((s.m > 0) + (s.n > 0) + (s.p > 0) < 2) return fail3(MS_EINVAL, "a source needs at least two nonzero indices");
    if (!std::isfinite(s.ax) || !std::isfinite(s.ay) || !std::isfinite(s.az) || !std::isfinite(s.omega))
      return fail3(MS_EINVAL, "non-finite source");
    const double dot = s.ax * s.m + s.ay * s.n + s.az * s.p;
    const double scale = std::fabs(s.ax * s.m) + std::fabs(s.ay * s.n) + std::fabs(s.az * s.p);
    if (std::fabs(dot) > 1e-12 * (scale > 0 ? scale : 1.0))
      return fail3(MS_EINVAL, "source polarisation must satisfy (ax, ay, az) . (m, n, p) = 0 (div J = 0)");
    if (need_off_resonance) {
      const double k2 = M_PI * M_PI * ((double)s.m * s.m + (double)s.n * s.n + (double)s.p * s.p);
      if (std::fabs(s.omega * s.omega - k2) <= 1e-12 * (k2 > 1 ? k2 : 1.0) || s.omega == 0.0)
        return fail3(MS_EINVAL, "driven solution needs 0 < omega^2 != pi^2 (m^2 + n^2 + p^2)");
    }
  }
  return MS_OK;
}

ms_status mode_field3_tables(ms_grid* g, int c, const std::vector<double>& tq, const std::vector<double>& coef,
                             double* out) {
  const Shape3& s = g->g3->sh[c];
  const int nm = (int)coef.size(), per = s.n[0] + s.n[1] + s.n[2];
  const size_t oy = (size_t)nm * s.n[0], oz = oy + (size_t)nm * s.n[1], oc = oz + (size_t)nm * s.n[2];
  std::vector<double> host(oc + nm, 0.0);
  for (int q = 0; q < nm; ++q) {
    for (int i = 0; i < s.n[0]; ++i) host[(size_t)q * s.n[0] + i] = tq[(size_t)q * per + i];
    for (int j = 0; j < s.n[1]; ++j) host[oy + (size_t)q * s.n[1] + j] = tq[(size_t)q * per + s.n[0] + j];
    for (int k = 0; k < s.n[2]; ++k) host[oz + (size_t)q * s.n[2] + k] = tq[(size_t)q * per + s.n[0] + s.n[1] + k];
    host[oc + q] = coef[q];
  }
  if (host.size() > g->modetab_cap) {
    dev_free(g->d_modetab);
    g->d_modetab = nullptr;
    g->modetab_cap = 0;
    MS3_TRY(alloc3(&g->d_modetab, host.size()));
    g->modetab_cap = host.size();
  }
  MS3_CUDA(cudaMemcpyAsync(g->d_modetab, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  k_mode_field3<<<grid3(s, kBlk), kBlk, 0, g->stream>>>(out, s, g->d_modetab, g->d_modetab + oy, g->d_modetab + oz,
                                                         g->d_modetab + oc, nm);
  MS3_CUDA(cudaGetLastError());
  MS3_CUDA(cudaStreamSynchronize(g->stream));  // the host table is released on return
  return MS_OK;
}


double stability_limit_3d() {
  static double cached = 0.0;
  if (cached > 0.0) return cached;
  double lo = 0.3, hi = 1.0;
  for (int it = 0; it < 50; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (max_amp2_3d(mid) <= 4.0) lo = mid;
    else hi = mid;
  }
  cached = lo;
  return cached;
}

ms_status create_grid3d(const ms_grid_desc* d, ms_grid** out) {
  if (d->n < 4 || d->n > 512) return fail3(MS_EINVAL, "3D grids need 4 <= n <= 512");
  if (!(d->z_imp > 0.0) || !std::isfinite(d->z_imp)) return fail3(MS_EINVAL, "z_imp must be positive");
  if (!(d->r > 0.0) || !std::isfinite(d->r)) return fail3(MS_EINVAL, "r must be positive");
  if (d->precision != MS_FP64 && d->precision != MS_FP32_REFINED) return fail3(MS_EINVAL, "unknown precision");
  if (d->closure != MS_CLOSURE_PAPER && d->closure != MS_CLOSURE_REFLECT) return fail3(MS_EINVAL, "unknown closure");
  if (d->scheme != MS_SCHEME_C4) return fail3(MS_EUNSUPPORTED, "3D grids run the compact scheme only");
  const double rmax = stability_limit_3d();
  if (d->r >= rmax) {
    char buf[160];
    snprintf(buf, sizeof buf, "r = %.6g is at or above the stability limit %.6g of the 3D scheme", d->r, rmax);
    return fail3(MS_ECFL, buf);
  }
  ms_grid* g = new ms_grid();
  g->g3 = new Grid3D();
  Grid3D* G3 = g->g3;
  g->desc = *d;
  g->N = d->n;
  g->Z = d->z_imp;
  g->h = 1.0 / d->n;
  g->ht = d->r * g->h;
  g->kappa2 = 24.0 / (g->ht * g->ht);
  g->beta = 1.0 + g->kappa2 * g->h * g->h / 12.0;
  g->c1 = g->kappa2 * g->beta;
  auto cleanup = [&](ms_status s) {
    ms_destroy(g);
    return s;
  };
  for (int c = 0; c < 6; ++c) {
    G3->sh[c] = field_shape3(g->N, c);
    if (G3->sh[c].size() > G3->nmax) G3->nmax = G3->sh[c].size();
  }
  if (d->stream) {
    g->stream = (cudaStream_t)d->stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(fail3(MS_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e)));
    g->own_stream = true;
  }
  std::string err;
  ms_status s = MS_OK;
  if (d->precision == MS_FP64) {
    for (int kind = 0; kind < 2 && s == MS_OK; ++kind) {
      const int M = (kind == HALF_TO_NODE) ? g->N - 1 : g->N;
      PadeTable& t = g->pade[kind];
      if (build_pade_table(M, d->closure, kind, 1e-18, &t, &err) != 0) return cleanup(fail3(MS_EINVAL, err));
      s = alloc3(&t.d_w, t.w.size());
      if (s == MS_OK && cudaMemcpy(t.d_w, t.w.data(), t.w.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        s = fail3(MS_ECUDA, "copy of Pade tables failed");
    }
    if (s == MS_OK) s = ms_solver_sweeps(3, d->r, MS_FP64, 1e-17, &g->p1_sweeps);
    for (int c = 0; c < 6 && s == MS_OK; ++c) s = alloc3(&G3->f64[c], G3->sh[c].size());
    for (int k = 0; k < 7 && s == MS_OK; ++k) s = alloc3(&G3->s64[k], G3->nmax);
  } else {
    for (int kind = 0; kind < 2 && s == MS_OK; ++kind) {
      const int M = (kind == HALF_TO_NODE) ? g->N - 1 : g->N;
      PadeTable& t = g->pade32[kind];
      if (build_pade_table(M, d->closure, kind, 1e-12, &t, &err, /*of_differences=*/true) != 0)
        return cleanup(fail3(MS_EINVAL, err));
      std::vector<float> whi(t.w.size()), wlo(t.w.size());
      for (size_t q = 0; q < t.w.size(); ++q) {
        whi[q] = (float)t.w[q];
        wlo[q] = (float)(t.w[q] - (double)whi[q]);
      }
      s = alloc3(&t.d_whi, whi.size());
      if (s == MS_OK) s = alloc3(&t.d_wlo, wlo.size());
      if (s == MS_OK && (cudaMemcpy(t.d_whi, whi.data(), whi.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemcpy(t.d_wlo, wlo.data(), wlo.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess))
        s = fail3(MS_ECUDA, "copy of FP32 Pade tables failed");
    }
    if (s == MS_OK && upload_band_row() != 0) s = fail3(MS_ECUDA, "cannot upload the interior band row");
    // Richardson sweeps to 1e-10 (below the FP32 rounding noise, which is not coherent)
    if (s == MS_OK) s = ms_solver_sweeps(3, d->r, MS_FP32_REFINED, 1e-10, &g->p1_sweeps32);
    for (int c = 0; c < 6 && s == MS_OK; ++c) s = alloc3(&G3->hi[c], G3->sh[c].size());
    for (int c = 0; c < 6 && s == MS_OK; ++c) s = alloc3(&G3->lo[c], G3->sh[c].size());
    for (int k = 0; k < 4 && s == MS_OK; ++k) s = alloc3(&G3->s32[k], G3->nmax);
    for (int k = 0; k < 3 && s == MS_OK; ++k) s = alloc3(&G3->gh[k], G3->nmax);
    for (int k = 0; k < 3 && s == MS_OK; ++k) s = alloc3(&G3->gl[k], G3->nmax);
    for (int k = 0; k < 2 && s == MS_OK; ++k) s = alloc3(&G3->s64[k], G3->nmax);
  }
  if (s == MS_OK) s = alloc3(&g->d_result, 8);
  if (s == MS_OK) {
    const int b = reduce_blocks(G3->nmax);
    s = alloc3(&g->d_partial, (size_t)b * 4);
    g->partial_cap = b;
  }
  if (s != MS_OK) return cleanup(s);
  for (int c = 0; c < 6; ++c) {
    const size_t n = G3->sh[c].size();
    if (G3->f64[c]) cudaMemsetAsync(G3->f64[c], 0, n * sizeof(double), g->stream);
    if (G3->hi[c]) cudaMemsetAsync(G3->hi[c], 0, n * sizeof(float), g->stream);
    if (G3->lo[c]) cudaMemsetAsync(G3->lo[c], 0, n * sizeof(float), g->stream);
  }
  for (int k = 0; k < 7; ++k)
    if (G3->s64[k]) cudaMemsetAsync(G3->s64[k], 0, G3->nmax * sizeof(double), g->stream);
  for (int k = 0; k < 4; ++k)
    if (G3->s32[k]) cudaMemsetAsync(G3->s32[k], 0, G3->nmax * sizeof(float), g->stream);
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cleanup(fail3(MS_ECUDA, std::string("create: ") + cudaGetErrorString(e)));
  *out = g;
  return MS_OK;
}

// Accuracy of one transform solve relative to the solution (bf16 three-product split: about 16
// correct bits per pass over six passes, measured at up to 2e-5 on random data), which fixes the
// refinement sweeps: ts_accuracy * rho^R <= 1e-10, the target of the Richardson solve.
constexpr double kTsAccuracy = 5e-5;

ms_status set_solver3d(ms_grid* g, int solver) {
  Grid3D* G3 = g->g3;
  if (solver == MS_SOLVER_RICHARDSON) {
    G3->solver = solver;
    return MS_OK;
  }
  if (!G3->ts) {
    G3->ts = new TransformSolver();
    std::string err;
    const int rc = ts_setup(g->N, G3->ts, &err);
    if (rc != 0) {
      ts_free(G3->ts);
      delete G3->ts;
      G3->ts = nullptr;
      return fail3(rc == -2 ? MS_ENOMEM : MS_ECUDA, err);
    }
  }
  int R = 0;
  MS3_TRY(ms_solver_sweeps(3, g->desc.r, MS_FP32_REFINED, 1e-10 / kTsAccuracy, &R));
  G3->ts_sweeps = R;
  G3->solver = solver;
  return MS_OK;
}

ms_status transform_solve3d(ms_grid* g, int c, const float* b, float* x) {
  Grid3D* G3 = g->g3;
  if (!G3->ts) {  // set the solver up without selecting it
    const int keep = G3->solver;
    MS3_TRY(set_solver3d(g, MS_SOLVER_TRANSFORM_TC));
    G3->solver = keep;
  }
  ts_solve(*G3->ts, G3->sh[c], b, x, 6.0f * (float)(g->c1 * g->h * g->h), g->stream, g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail3(MS_ECUDA, std::string("transform solve: ") + cudaGetErrorString(e));
  return MS_OK;
}

ms_status transform_status3d(ms_grid* g) {
  Grid3D* G3 = g->g3;
  if (!G3 || !G3->ts) return MS_OK;
  int flag = 0;
  if (cudaMemcpy(&flag, G3->ts->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail3(MS_ECUDA, "reading the transform solver's status failed");
  if (flag) {
    cudaMemset(G3->ts->d_err, 0, sizeof(int));
    return fail3(MS_ETIMEOUT, "a transform GEMM gave up waiting for its tensor-core MMAs; its output is invalid");
  }
  return MS_OK;
}

void destroy_grid3d(ms_grid* g) {
  Grid3D* G3 = g->g3;
  if (!G3) return;
  src3_free(g);
  if (G3->ts) {
    ts_free(G3->ts);
    delete G3->ts;
    G3->ts = nullptr;
  }
  for (int c = 0; c < 6; ++c) {
    dev_free(G3->f64[c]);
    dev_free(G3->hi[c]);
    dev_free(G3->lo[c]);
    dev_free(G3->dview[c]);
  }
  for (int k = 0; k < 7; ++k) dev_free(G3->s64[k]);
  for (int k = 0; k < 4; ++k) dev_free(G3->s32[k]);
  for (int k = 0; k < 3; ++k) {
    dev_free(G3->gh[k]);
    dev_free(G3->gl[k]);
  }
  for (int k = 0; k < 2; ++k) {
    dev_free(g->pade32[k].d_whi);
    dev_free(g->pade32[k].d_wlo);
    g->pade32[k].d_whi = g->pade32[k].d_wlo = nullptr;
  }
  delete G3;
  g->g3 = nullptr;
}

int state_arrays3d(ms_grid* g, double** f64, float** hi, float** lo, size_t* n) {
  Grid3D* G3 = g->g3;
  for (int c = 0; c < 6; ++c) {
    f64[c] = G3->f64[c];
    hi[c] = G3->hi[c];
    lo[c] = G3->lo[c];
    n[c] = G3->sh[c].size();
  }
  return 6;
}

ms_status step3d(ms_grid* g) { return g->desc.precision == MS_FP64 ? step3d64(g) : step3d32(g); }

ms_status set_fields3d(ms_grid* g, const double* const* comps, int host) {
  for (int c = 0; c < 6; ++c)
    if (!comps[c]) return fail3(MS_EINVAL, "NULL component");
  Grid3D* G3 = g->g3;
  for (int c = 0; c < 6; ++c) {
    const size_t n = G3->sh[c].size();
    if (host) {
      double* tmp = G3->s64[0];
      MS3_CUDA(cudaMemcpyAsync(tmp, comps[c], n * sizeof(double), cudaMemcpyHostToDevice, g->stream));
      MS3_TRY(store3(g, c, tmp));
    } else {
      MS3_TRY(store3(g, c, comps[c]));
    }
  }
  if (host) MS3_CUDA(cudaStreamSynchronize(g->stream));
  return MS_OK;
}

ms_status get_fields3d(ms_grid* g, double* const* comps, int host) {
  for (int c = 0; c < 6; ++c)
    if (!comps[c]) return fail3(MS_EINVAL, "NULL component");
  Grid3D* G3 = g->g3;
  for (int c = 0; c < 6; ++c) {
    const size_t n = G3->sh[c].size();
    if (g->desc.precision == MS_FP64) {
      MS3_CUDA(cudaMemcpyAsync(comps[c], G3->f64[c], n * sizeof(double),
                               host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, g->stream));
    } else if (host) {
      const double* v = view3(g, c, G3->s64[0]);
      MS3_CUDA(cudaMemcpyAsync(comps[c], v, n * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
      MS3_CUDA(cudaStreamSynchronize(g->stream));  // s64[0] is reused by the next component
    } else {
      view3(g, c, comps[c]);
    }
  }
  MS3_CUDA(cudaGetLastError());
  if (host) MS3_CUDA(cudaStreamSynchronize(g->stream));
  return MS_OK;
}

// FP64 components for the diagnostics.  An FP64 grid gives its state; an FP32_REFINED grid joins
// its float-float state into FP64 copies, and on the first call builds what the FP64 kernels need
// (FP64 Pade tables, the FP64 sweep count, FP64 scratch), kept until the grid is destroyed.
ms_status diag_view3d(ms_grid* g, double** f) {
  Grid3D* G3 = g->g3;
  if (g->desc.precision == MS_FP64) {
    for (int c = 0; c < 6; ++c) f[c] = G3->f64[c];
    return MS_OK;
  }
  std::string err;
  for (int kind = 0; kind < 2; ++kind) {
    PadeTable& t = g->pade[kind];
    if (t.d_w) continue;
    const int M = (kind == HALF_TO_NODE) ? g->N - 1 : g->N;
    if (build_pade_table(M, g->desc.closure, kind, 1e-18, &t, &err) != 0) return fail3(MS_EINVAL, err);
    MS3_TRY(alloc3(&t.d_w, t.w.size()));
    if (cudaMemcpy(t.d_w, t.w.data(), t.w.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail3(MS_ECUDA, "copy of Pade tables failed");
  }
  if (!g->p1_sweeps) MS3_TRY(ms_solver_sweeps(3, g->desc.r, MS_FP64, 1e-17, &g->p1_sweeps));
  for (int k = 0; k < 7; ++k)
    if (!G3->s64[k]) MS3_TRY(alloc3(&G3->s64[k], G3->nmax));
  for (int c = 0; c < 6; ++c) {
    const size_t n = G3->sh[c].size();
    if (!G3->dview[c]) MS3_TRY(alloc3(&G3->dview[c], n));
    k_join3<<<(unsigned)((n + 255) / 256), 256, 0, g->stream>>>(G3->hi[c], G3->lo[c], G3->dview[c], n);
    f[c] = G3->dview[c];
  }
  return MS_OK;
}

// Discrete energy of a 3D grid: W = h^3 [Z^-1 sum E.E + Z (sum H.H - h_tau sum H*.H)], H* the Step 2
// increment that the current E gives (P1^{-1} of the H right-hand side), computed in FP64 with the
// step's own filter, Pade and sweep kernels but not added to H.
ms_status energy3d(ms_grid* g, double* W) {
  Grid3D* G3 = g->g3;
  double* f[6];
  MS3_TRY(diag_view3d(g, f));
  double** G = G3->s64;  // G[0..2]: filtered E
  double* R = G3->s64[3];
  const double* X = G3->s64[6];  // the last sweep's iterate
  const double s_eh = g->kappa2 / (g->Z * g->h);
  int nl = 0;
  for (int c = 0; c < 3; ++c) {
    filter3d64(g, c, f[c], G[c]);
    const size_t n = G3->sh[c].size();
    launch_dot(f[c], f[c], n, g->d_partial, reduce_blocks(n), g->d_result, 0, c > 0, g->stream);
  }
  for (int hc = 0; hc < 3; ++hc) {
    const int p1 = (hc + 1) % 3, p2 = (hc + 2) % 3;
    pade3d64(g, p1, p2, 3 + hc, G[p2], R, -s_eh, 0);
    pade3d64(g, p2, p1, 3 + hc, G[p1], R, s_eh, 1);
    solve3d64(g, 3 + hc, R, nullptr, 0.0, &nl);
    const size_t n = G3->sh[3 + hc].size();
    const double* Hc = f[3 + hc];
    launch_dot(Hc, Hc, n, g->d_partial, reduce_blocks(n), g->d_result, 1, hc > 0, g->stream);
    launch_dot(X, Hc, n, g->d_partial, reduce_blocks(n), g->d_result, 2, hc > 0, g->stream);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail3(MS_ECUDA, std::string("3D energy: ") + cudaGetErrorString(e));
  double r[3];
  MS3_CUDA(cudaMemcpyAsync(r, g->d_result, sizeof r, cudaMemcpyDeviceToHost, g->stream));
  MS3_CUDA(cudaStreamSynchronize(g->stream));
  *W = g->h * g->h * g->h * (r[0] / g->Z + g->Z * (r[1] - g->ht * r[2]));
  return MS_OK;
}

// Pade divergence of H on the N^3 cell centres of a 3D grid (in FP64): div_h H = sum_a delta_a H_a,
// each a node -> half-node derivative along its own axis; *norm = sqrt(h^3 sum div^2).
ms_status divergence3d(ms_grid* g, double* norm) {
  Grid3D* G3 = g->g3;
  double* f[6];
  MS3_TRY(diag_view3d(g, f));
  const int N = g->N;
  Shape3 sc;  // cell centres: N points on every axis, no walls
  for (int a = 0; a < 3; ++a) {
    sc.n[a] = N;
    sc.bc[a] = NEU;
  }
  double* div = G3->s64[0];
  const PadeTable& t = g->pade[NODE_TO_HALF];
  const dim3 grd = grid3(sc, kBlk);
  const double sc_h = 1.0 / g->h;
  k_pade3d64<0><<<grd, kBlk, 0, g->stream>>>(f[3], div, sc, G3->sh[3], t.d_w, t.rows, t.n_in, t.left, t.K, t.B,
                                              t.all_explicit, 0, sc_h, 0);
  k_pade3d64<1><<<grd, kBlk, 0, g->stream>>>(f[4], div, sc, G3->sh[4], t.d_w, t.rows, t.n_in, t.left, t.K, t.B,
                                              t.all_explicit, 0, sc_h, 1);
  k_pade3d64<2><<<grd, kBlk, 0, g->stream>>>(f[5], div, sc, G3->sh[5], t.d_w, t.rows, t.n_in, t.left, t.K, t.B,
                                              t.all_explicit, 0, sc_h, 1);
  const size_t n = sc.size();
  launch_dot(div, div, n, g->d_partial, reduce_blocks(n), g->d_result, 0, 0, g->stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail3(MS_ECUDA, std::string("3D divergence: ") + cudaGetErrorString(e));
  double r;
  MS3_CUDA(cudaMemcpyAsync(&r, g->d_result, sizeof r, cudaMemcpyDeviceToHost, g->stream));
  MS3_CUDA(cudaStreamSynchronize(g->stream));
  *norm = std::sqrt(g->h * g->h * g->h * r);
  return MS_OK;
}

}  // namespace ms

using namespace ms;

extern "C" {

ms_status ms_init_modes3(ms_grid* g, const ms_mode3* modes, int nmodes) {
  if (!g || !g->g3) return fail3(MS_EINVAL, "ms_init_modes3 needs a 3D grid");
  MS3_TRY(check_modes3(modes, nmodes));
  double* tmp = g->g3->s64[1];
  for (int c = 0; c < 6; ++c) {
    MS3_TRY(exact3(g, modes, nmodes, 0.0, 0.5 * g->ht, c, tmp));
    MS3_TRY(store3(g, c, tmp));
  }
  g->step = 0;
  if (g->d_step) MS3_CUDA(cudaMemcpy(g->d_step, &g->step, sizeof(long), cudaMemcpyHostToDevice));
  MS3_CUDA(cudaStreamSynchronize(g->stream));
  return MS_OK;
}

ms_status ms_init_driven3(ms_grid* g, const ms_source3* src, int nsrc) {
  if (!g || !g->g3) return fail3(MS_EUNSUPPORTED, "ms_init_driven3 needs a 3D grid");
  MS3_TRY(check_sources3(src, nsrc, true));
  double* tmp = g->g3->s64[1];
  for (int c = 0; c < 6; ++c) {
    MS3_TRY(exact_driven3(g, src, nsrc, 0.0, 0.5 * g->ht, c, tmp));
    MS3_TRY(store3(g, c, tmp));
  }
  g->step = 0;
  if (g->d_step) MS3_CUDA(cudaMemcpy(g->d_step, &g->step, sizeof(long), cudaMemcpyHostToDevice));
  MS3_CUDA(cudaStreamSynchronize(g->stream));
  return MS_OK;
}

ms_status ms_error_vs_exact3(ms_grid* g, const ms_mode3* modes, int nmodes, double* l2_abs, double* l2_rel,
                             double* max_abs, double* sum_abs) {
  if (!g || !g->g3) return fail3(MS_EINVAL, "ms_error_vs_exact3 needs a 3D grid");
  MS3_TRY(check_modes3(modes, nmodes));
  Grid3D* G3 = g->g3;
  const double tE = g->step * g->ht, tH = (g->step + 0.5) * g->ht;
  for (int c = 0; c < 6; ++c) {
    const size_t n = G3->sh[c].size();
    MS3_TRY(exact3(g, modes, nmodes, tE, tH, c, G3->s64[1]));
    const double* v = view3(g, c, G3->s64[0]);
    launch_err_reduce(v, G3->s64[1], n, g->d_partial, reduce_blocks(n), g->d_result, c > 0, g->stream);
  }
  double r[4];
  MS3_CUDA(cudaMemcpyAsync(r, g->d_result, sizeof r, cudaMemcpyDeviceToHost, g->stream));
  MS3_CUDA(cudaStreamSynchronize(g->stream));
  const double h3 = g->h * g->h * g->h;
  if (l2_abs) *l2_abs = std::sqrt(h3 * r[0]);
  if (l2_rel) *l2_rel = r[1] > 0.0 ? std::sqrt(r[0] / r[1]) : 0.0;
  if (max_abs) *max_abs = r[2];
  if (sum_abs) *sum_abs = r[3];
  return MS_OK;
}

}  // extern "C"
