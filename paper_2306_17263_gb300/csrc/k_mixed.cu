// MS_FP32_REFINED: the step of Sec. 3.4 in FP32 arithmetic with accuracy won back by
// exact coefficients, float-float intermediates where the scheme cancels, and refinement.
//
// Scaling.  Every operator is applied in an integer-coefficient form so that FP32 only adds
// rounding noise, never a coherent error in a coefficient:
//   G~ = 12 G = (12 beta) u + L u                  (filter of Eq. "eq:ell", L = h^2 Delta_h)
//   y  = A^{-1} (D1~ G~)                           (Pade of App. A.1, D1~ the plain difference)
//   6 P~ x = b,  6 P~ = 6 c1 h^2 - 6 Lx - 6 Ly - Lx Ly   (P1 of Def. "def:operatorsP" times 6 h^2)
// Coefficients that are not exact in FP32 (12 beta, 6 c1 h^2, the entries of A^{-1}, the final
// scale) are carried as hi + lo pairs.  The P1 solve is a Richardson iteration whose fixed
// point is set by the residual alone, so the approximate relaxation factor changes only the
// rate.  With these scalings the increments are
//   E += (12 Z / r) x_E,   H_x += (12 / (r Z)) x_Hx,   H_y += (12 / (r Z)) x_Hy.
//
// Cancellation.  The Pade derivative of a resolved field is a difference of nearly equal
// values (|D1 G| ~ theta |G|, theta = pi k h), so an FP32 rounding of G at the level of |G|
// would be amplified by 1/theta in every step.  The filter therefore returns G~ as an unevaluated
// float-float pair (p, q) computed from the float-float state, the first differences are taken
// as (p_{m+1} - p_m) + (q_{m+1} - q_m), and only then is the well-conditioned A^{-1} band applied.
// The state itself is a float-float pair updated with error-free transformations (Knuth
// two-sum, FMA two-product).
#include <cmath>
#include <string>

#include "k_fp64.cuh"
#include "k_mixed.cuh"

namespace ms {

namespace {
thread_local std::string g_mixed_err;

struct Split {
  float hi, lo;
};
Split split(double v) {
  Split s;
  s.hi = (float)v;
  s.lo = (float)(v - (double)s.hi);
  return s;
}
}  // namespace

const char* mixed_last_error() { return g_mixed_err.c_str(); }

// ---------------------------------------------------------------------------------------
// G~ = (12 beta) u + L u as a float-float pair (p, q) from the state pair (hi, lo); zero on
// Dirichlet boundary points.  L is summed as differences to the centre (exact for close values).
__global__ void k_filter32ff(const float* __restrict__ hi, const float* __restrict__ lo, float* __restrict__ P,
                             float* __restrict__ Q, int nx, int ny, int bcx, int bcy, float cb_hi, float cb_lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const size_t p = (size_t)j * nx + i;
  if (!interior(bcx, i, nx) || !interior(bcy, j, ny)) {
    P[p] = 0.0f;
    Q[p] = 0.0f;
    return;
  }
  const int im = clampi(i - 1, nx), ip = clampi(i + 1, nx), jm = clampi(j - 1, ny), jp = clampi(j + 1, ny);
  const size_t pw = (size_t)j * nx + im, pe = (size_t)j * nx + ip, ps = (size_t)jm * nx + i, pn = (size_t)jp * nx + i;
  const float ch = hi[p], cl = lo[p];
  const float lh = ((hi[pw] - ch) + (hi[pe] - ch)) + ((hi[ps] - ch) + (hi[pn] - ch));
  const float ll = ((lo[pw] - cl) + (lo[pe] - cl)) + ((lo[ps] - cl) + (lo[pn] - cl));
  const float m = __fmul_rn(cb_hi, ch);
  const float e = fmaf(cb_hi, ch, -m);  // m + e == cb_hi * ch exactly
  P[p] = m;
  Q[p] = e + (fmaf(cb_lo, ch, cb_hi * cl) + (lh + ll));
}

// Pade derivative from first differences: out (+)= sign * sum_m A^{-1}(i, m) d_m with
// d_m = (P_{m+1} - P_m) + (Q_{m+1} - Q_m) along the line, A^{-1} split into (whi, wlo).
template <int AXIS>
__global__ void k_pade32d(const float* __restrict__ P, const float* __restrict__ Q, float* __restrict__ out,
                          int n_lines, int M, int in_ld, int out_len, int out_ld, int out_off, int line_lo,
                          int line_hi, const float* __restrict__ whi, const float* __restrict__ wlo, int K, int B,
                          int all_explicit, float sign, int accumulate) {
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
  float v = 0.0f;
  if (i >= 0 && i < M && line >= line_lo && line < line_hi) {
    const float* wh = pade_row_ptr(whi, i, M, K, B, all_explicit);
    const float* wl = pade_row_ptr(wlo, i, M, K, B, all_explicit);
    const int m0 = i - K;
    const size_t stride = (AXIS == 0) ? 1 : (size_t)in_ld;
    const size_t base = (AXIS == 0) ? (size_t)line * in_ld : (size_t)line;
    float a = 0.0f, b = 0.0f;
    for (int t = 0; t < 2 * K + 2; ++t) {
      const int m = m0 + t;
      if (m < 0 || m >= M) continue;
      const size_t k0 = base + (size_t)m * stride, k1 = k0 + stride;
      const float d = (P[k1] - P[k0]) + (Q[k1] - Q[k0]);
      a = fmaf(wh[t], d, a);
      b = fmaf(wl[t], d, b);
    }
    v = sign * (a + b);
  }
  if (accumulate) out[po] += v;
  else out[po] = v;
}

// (hi, lo) += (S_hi + S_lo) x with error-free transformations.  The _rn intrinsics keep the
// compiler from contracting these steps into FMAs, which would break the error accounting.
__device__ __forceinline__ void ff_add_scaled(float& hi, float& lo, float x, float s_hi, float s_lo) {
  const float p = __fmul_rn(s_hi, x);
  float e = fmaf(s_hi, x, -p);  // p + e == s_hi * x exactly
  e = fmaf(s_lo, x, e);
  const float s = __fadd_rn(hi, p);  // two-sum of hi and p
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float l = __fadd_rn(lo, __fadd_rn(err, e));
  const float h2 = __fadd_rn(s, l);  // renormalise (fast two-sum, |s| >= |l|)
  lo = __fsub_rn(l, __fsub_rn(h2, s));
  hi = h2;
}

// Richardson sweep on 6 P~ x = b:  x' = x + omega (b - 6 P~ x).
// Two details keep the FP32 iteration free of coherent error:
//  - the residual is computed accurately: the dominant diagonal product 6 c1 h^2 x is formed
//    as an exact two-product, so b - 6 P~ x carries no rounding at the level of |b|;
//  - the last sweep does not round x + omega r to FP32 (a correction below half an ulp of x
//    would be lost, and since the iterates approach the solution from one side for most
//    modes, the loss is a systematic shrink of every increment); instead x and omega r are
//    added to the float-float state separately.
// first != 0: x is taken as 0.  st_hi != nullptr marks the last sweep (state update, no xout).
__global__ void k_p1_sweep32(const float* __restrict__ b, const float* __restrict__ xin, float* __restrict__ xout,
                             int nx, int ny, int bcx, int bcy, float d_hi, float d_lo, float omega, int first,
                             float* __restrict__ st_hi, float* __restrict__ st_lo, float s_hi, float s_lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const size_t p = (size_t)j * nx + i;
  if (!interior(bcx, i, nx) || !interior(bcy, j, ny)) {
    if (!st_hi) xout[p] = 0.0f;
    return;
  }
  float x, corr;
  if (first) {
    x = 0.0f;
    corr = omega * b[p];
  } else {
    const int im = clampi(i - 1, nx), ip = clampi(i + 1, nx), jm = clampi(j - 1, ny), jp = clampi(j + 1, ny);
    const float* r0 = xin + (size_t)jm * nx;
    const float* r1 = xin + (size_t)j * nx;
    const float* r2 = xin + (size_t)jp * nx;
    const float c = r1[i];
    const float lx = (r1[im] - c) + (r1[ip] - c);
    const float ly = (r0[i] - c) + (r2[i] - c);
    const float lxm = (r0[im] - r0[i]) + (r0[ip] - r0[i]);
    const float lxp = (r2[im] - r2[i]) + (r2[ip] - r2[i]);
    const float lxly = (lxm - lx) + (lxp - lx);
    const float rest = -6.0f * (lx + ly) - lxly;
    const float ph = __fmul_rn(d_hi, c);
    const float pl = fmaf(d_lo, c, fmaf(d_hi, c, -ph));  // ph + pl = (d_hi + d_lo) c to ~2^-48
    const float res = __fsub_rn(__fsub_rn(b[p], ph), pl) - rest;
    x = c;
    corr = omega * res;
  }
  if (st_hi) {
    float h = st_hi[p], l = st_lo[p];
    ff_add_scaled(h, l, x, s_hi, s_lo);
    ff_add_scaled(h, l, corr, s_hi, s_lo);
    st_hi[p] = h;
    st_lo[p] = l;
  } else {
    xout[p] = x + corr;
  }
}

static inline dim3 grid2(int nx, int ny, dim3 blk) { return dim3((nx + blk.x - 1) / blk.x, (ny + blk.y - 1) / blk.y); }

static void pade32(ms_grid* g, int kind, int axis, const float* P, const float* Q, float* out, int n_lines, int in_ld,
                   int out_len, int out_ld, int out_off, int line_lo, int line_hi, float sign, int acc) {
  const PadeTable& t = g->pade32[kind];
  dim3 blk(32, 8);
  if (axis == 0)
    k_pade32d<0><<<grid2(out_len, n_lines, blk), blk, 0, g->stream>>>(P, Q, out, n_lines, t.M, in_ld, out_len, out_ld,
                                                                       out_off, line_lo, line_hi, t.d_whi, t.d_wlo,
                                                                       t.K, t.B, t.all_explicit, sign, acc);
  else
    k_pade32d<1><<<grid2(n_lines, out_len, blk), blk, 0, g->stream>>>(P, Q, out, n_lines, t.M, in_ld, out_len, out_ld,
                                                                       out_off, line_lo, line_hi, t.d_whi, t.d_wlo,
                                                                       t.K, t.B, t.all_explicit, sign, acc);
}

static void filter32(ms_grid* g, int f, float* P, float* Q) {
  const Shape& s = g->sh[f];
  const Split cb = split(12.0 * g->beta);
  dim3 blk(32, 8);
  k_filter32ff<<<grid2(s.nx, s.ny, blk), blk, 0, g->stream>>>(g->hi[f], g->lo[f], P, Q, s.nx, s.ny, s.bcx, s.bcy,
                                                               cb.hi, cb.lo);
  prof_mark(g, KK_FILTER32, 16.0 * (double)s.size());
}

// Solve 6 P~ x = b and add S x to the state (hi, lo) of field f.
static void solve32(ms_grid* g, int f, const float* b, double S, int* nl) {
  const Shape& s = g->sh[f];
  const double c1h2 = g->c1 * g->h * g->h;
  const Split d = split(6.0 * c1h2);
  const float omega = (float)(2.0 / (12.0 * c1h2 + 32.0));
  const Split sc = split(S);
  float* buf[2] = {g->s32[5], g->s32[6]};
  const float* xin = nullptr;
  dim3 blk(32, 8);
  const int n = g->p1_sweeps32;
  for (int k = 0; k < n; ++k) {
    const bool last = (k == n - 1);
    float* xo = buf[k & 1];
    k_p1_sweep32<<<grid2(s.nx, s.ny, blk), blk, 0, g->stream>>>(b, xin, xo, s.nx, s.ny, s.bcx, s.bcy, d.hi, d.lo, omega,
                                                                 k == 0, last ? g->hi[f] : nullptr,
                                                                 last ? g->lo[f] : nullptr, sc.hi, sc.lo);
    // reads b (and x unless first); writes x, or reads and writes the state pair on the last sweep
    prof_mark(g, KK_P1SWEEP32, 4.0 * (double)s.size() * ((k == 0 ? 1 : 2) + (last ? 4 : 1)));
    xin = xo;
  }
  *nl += n;
}

ms_status step_mixed(ms_grid* g, int* nl) {
  const int N = g->N;
  const double Nd = N;
  // Step 1: b = A^{-1} D1 G~_y (along x) - A^{-1} D1 G~_x (along y) on the E_z interior
  float *Px = g->s32[0], *Qx = g->s32[1], *Py = g->s32[2], *Qy = g->s32[3], *b = g->s32[4];
  filter32(g, HX, Px, Qx);
  filter32(g, HY, Py, Qy);
  pade32(g, HALF_TO_NODE, 0, Py, Qy, b, N + 1, N, N + 1, N + 1, 1, 1, N, 1.0f, 0);
  prof_mark(g, KK_PADE32, 4.0 * (2.0 * (Nd - 1) * Nd + (Nd + 1) * (Nd + 1)));
  pade32(g, HALF_TO_NODE, 1, Px, Qx, b, N + 1, N + 1, N + 1, N + 1, 1, 1, N, -1.0f, 1);
  prof_mark(g, KK_PADE32, 4.0 * (2.0 * (Nd - 1) * Nd + 2.0 * (Nd + 1) * (Nd + 1)));
  *nl += 4;
  solve32(g, EZ, b, 12.0 * g->Z / g->desc.r, nl);
  // Step 2: b_x = -A^{-1} D1 G~_E (along y), b_y = +A^{-1} D1 G~_E (along x)
  float *PE = g->s32[0], *QE = g->s32[1], *bx = g->s32[2], *by = g->s32[3];
  filter32(g, EZ, PE, QE);
  pade32(g, NODE_TO_HALF, 1, PE, QE, bx, N + 1, N + 1, N, N + 1, 0, 1, N, -1.0f, 0);
  prof_mark(g, KK_PADE32, 4.0 * (2.0 * (Nd - 1) * (Nd + 1) + Nd * (Nd + 1)));
  pade32(g, NODE_TO_HALF, 0, PE, QE, by, N + 1, N + 1, N, N, 0, 1, N, 1.0f, 0);
  prof_mark(g, KK_PADE32, 4.0 * (2.0 * (Nd - 1) * (Nd + 1) + Nd * (Nd + 1)));
  *nl += 3;
  solve32(g, HX, bx, 12.0 / (g->desc.r * g->Z), nl);
  solve32(g, HY, by, 12.0 / (g->desc.r * g->Z), nl);
  return MS_OK;
}

ms_status mixed_setup(ms_grid* g) {
  std::string err;
  for (int kind = 0; kind < 2; ++kind) {
    const int M = (kind == HALF_TO_NODE) ? g->N - 1 : g->N;
    PadeTable& t = g->pade32[kind];
    if (build_pade_table(M, g->desc.closure, kind, 1e-12, &t, &err, /*of_differences=*/true) != 0) {
      g_mixed_err = err;
      return MS_EINVAL;
    }
    std::vector<float> whi(t.w.size()), wlo(t.w.size());
    for (size_t k = 0; k < t.w.size(); ++k) {
      Split s = split(t.w[k]);
      whi[k] = s.hi;
      wlo[k] = s.lo;
    }
    if (cudaMalloc(&t.d_whi, whi.size() * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&t.d_wlo, wlo.size() * sizeof(float)) != cudaSuccess) {
      g_mixed_err = "cudaMalloc of FP32 Pade tables failed";
      return MS_ENOMEM;
    }
    if (cudaMemcpy(t.d_whi, whi.data(), whi.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t.d_wlo, wlo.data(), wlo.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      g_mixed_err = "copy of FP32 Pade tables failed";
      return MS_ECUDA;
    }
  }
  // Richardson sweeps to 1e-10 (below the FP32 rounding noise, which is not coherent)
  const double c1h2 = g->c1 * g->h * g->h;
  const double rho = (16.0 / 3.0) / (2.0 * c1h2 + 16.0 / 3.0);
  int s = (int)std::ceil(std::log(1e-10) / std::log(rho));
  g->p1_sweeps32 = s < 1 ? 1 : (s > 64 ? 64 : s);
  const size_t nmax = (size_t)(g->N + 1) * (g->N + 1);
  for (int k = 0; k < 8; ++k) {
    if (cudaMalloc(&g->s32[k], nmax * sizeof(float) + 256) != cudaSuccess) {
      g_mixed_err = "cudaMalloc of FP32 scratch failed";
      return MS_ENOMEM;
    }
    cudaMemset(g->s32[k], 0, nmax * sizeof(float));
  }
  return MS_OK;
}

void mixed_teardown(ms_grid* g) {
  for (int k = 0; k < 2; ++k) {
    cudaFree(g->pade32[k].d_whi);
    cudaFree(g->pade32[k].d_wlo);
    g->pade32[k].d_whi = g->pade32[k].d_wlo = nullptr;
  }
}

}  // namespace ms
