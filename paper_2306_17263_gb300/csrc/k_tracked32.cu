// Tracked-Delta-E variant of the step in MS_FP32_REFINED (MS_SCHEME_C4_DE): Sec. 3.4 as printed.
// Delta E_z is carried as float-float state DE, advanced after Step 1 by the modified Helmholtz
// equation of Eq. "eq:mhe" (J = 0),
//   DE^{n+1} = DE^n + kappa^2 (E^{n+1} - E^n) - Z (24 / h_tau) curl_h H^{n+1/2},
// and Step 2 filters E with it as in Eq. "eq:helm2": G~_E = 12 G_E = 12 beta E + h^2 DE.
//
// The update is the small difference of two large terms: kappa^2 (E^{n+1} - E^n) and the curl term
// agree to about omega h_tau / 24 (1.8e-3 at 2048^2), so both are formed in float-float.  The
// increment is the float-float difference of the state after and before the E solve; the curl is
// the Pade derivative of the unfiltered H (App. A.1) taken on exact first differences (two-sum of
// the hi parts plus the difference of the lo parts) through a band whose central taps are summed
// in float-float (exact two-products) and whose far taps, below 1.2e-4 of the centre, in FP32.
// Step 2 then runs the tile curl of the FP32 step on G~_E with its filter switched off.
#include <cmath>

#include "k_fp64.cuh"
#include "k_tiled.cuh"
#include "k_tracked32.cuh"

namespace ms {
namespace {

// (sh, sl) += (w + wl)(a + c): exact product of the hi parts, the lo parts in the error term.
__device__ __forceinline__ void ff_fma_acc_f(float& sh, float& sl, float w, float wl, float a, float c) {
  const float prod = __fmul_rn(w, a);
  float e = fmaf(w, a, -prod);
  e = fmaf(w, c, e);
  e = fmaf(wl, a, e);
  const float s = __fadd_rn(sh, prod);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(prod, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// a - b of two float-float values as an unnormalised pair (exact two-sum of the hi parts).
__device__ __forceinline__ void ff_diff(float ah, float al, float bh, float bl, float& dh, float& dl) {
  const float s = __fsub_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(-bh, bb));
  dh = s;
  dl = __fadd_rn(err, __fsub_rn(al, bl));
}

// Renormalise (h, l) so that |l| <= ulp(h) / 2.
__device__ __forceinline__ void ff_norm(float& h, float& l) {
  const float s = __fadd_rn(h, l);
  const float bb = __fsub_rn(s, h);
  l = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(l, bb));
  h = s;
}

// Forward Pade band in float-float: y_r = sum_t W(r, t) delta_{r - K + t} on the first differences
// of a float-float field along the lines of one axis.  Line l of the source is
// u[l * ul + m * ua] (m = 0 .. M), outputs r = 0 .. M-1 go to y[l * yl + (r + 1) * ya].
struct BandF {
  const float* uh;
  const float* ul_;
  float* yh;
  float* yl_;
  int ua, ul, ya, yl;  // strides along / across for the source and the output
  int nlines;
  const float* whi;
  const float* wlo;
  int M, K, B, all_explicit;
};

// Tiles: AXIS 0 (lines are rows, contiguous): 8 lines x 128 outputs, a warp per line; AXIS 1 (lines
// are columns): 32 lines x 32 outputs, lanes across the lines.  The differences a tile reads (its
// outputs widened by the band's reach, zero past the line) are staged once in shared memory.
constexpr int BF_THREADS = 256;
constexpr int BF_KMAX = kTiledKMax;
template <int AXIS>
struct BandFTile {
  static constexpr int LINES = AXIS == 0 ? 8 : 32;
  static constexpr int OUTS = AXIS == 0 ? 128 : 32;
  static constexpr int WIN = OUTS + 2 * BF_KMAX + 2;
};

template <int AXIS>
__global__ void __launch_bounds__(BF_THREADS) k_bandF32(BandF p) {
  using T = BandFTile<AXIS>;
  __shared__ float dh_s[T::LINES][T::WIN + 1];
  __shared__ float dl_s[T::LINES][T::WIN + 1];
  __shared__ float wh_s[2 * BF_KMAX + 2], wl_s[2 * BF_KMAX + 2];
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * T::OUTS;  // first output row of the tile
  const int l0 = blockIdx.y * T::LINES;
  const int base = r0 - p.K;            // difference index of slot 0
  const int win = T::OUTS + 2 * p.K + 2;
  // stage the exact differences delta_m, m in [base, base + win), of every line of the tile
  for (int e = tid; e < T::LINES * win; e += BF_THREADS) {
    int ll, q;
    if (AXIS == 0) {
      ll = e / win;
      q = e - ll * win;
    } else {
      q = e / T::LINES;
      ll = e - q * T::LINES;
    }
    const int m = base + q, l = l0 + ll;
    float dh = 0.0f, dl = 0.0f;
    if (m >= 0 && m < p.M && l < p.nlines) {
      const size_t o = (size_t)l * p.ul + (size_t)m * p.ua;
      ff_diff(p.uh[o + p.ua], p.ul_[o + p.ua], p.uh[o], p.ul_[o], dh, dl);
    }
    dh_s[ll][q] = dh;
    dl_s[ll][q] = dl;
  }
  // the interior row of the table (taps d = m - r = -K .. K+1 at index d + K)
  const int rs = 2 * p.K + 2;
  if (!p.all_explicit && tid < rs) {
    wh_s[tid] = p.whi[(size_t)(2 * p.B) * rs + tid];
    wl_s[tid] = p.wlo[(size_t)(2 * p.B) * rs + tid];
  }
  __syncthreads();
  constexpr int PER = T::OUTS * T::LINES / BF_THREADS;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    int ll, ro;
    if (AXIS == 0) {
      ll = tid >> 5;
      ro = (tid & 31) + 32 * k;
    } else {
      ll = tid & 31;
      ro = (tid >> 5) + 8 * k;
    }
    const int r = r0 + ro, l = l0 + ll;
    if (r >= p.M || l >= p.nlines) continue;
    const float* ah = &dh_s[ll][r - base];  // ah[d] = delta_{r + d}
    const float* al = &dl_s[ll][r - base];
    float sh = 0.0f, sl = 0.0f;
    if (!p.all_explicit && r >= p.B && r < p.M - p.B && r >= p.K && r + p.K + 1 < p.M) {
      // interior row: taps |d| >= 3 (below 1.2e-4 of the centre tap) summed in FP32, farthest
      // first, then joined to the float-float sum of the five central taps
      float small = 0.0f;
#pragma unroll
      for (int d = BF_KMAX + 1; d >= -BF_KMAX; --d) {
        if (d >= -2 && d <= 2) continue;
        if (d > p.K + 1 || d < -p.K) continue;
        small = fmaf(wh_s[d + p.K], ah[d], small);
      }
#pragma unroll
      for (int d = 2; d >= -2; --d) ff_fma_acc_f(sh, sl, wh_s[d + p.K], wl_s[d + p.K], ah[d], al[d]);
      sl = __fadd_rn(sl, small);
    } else {
      const float* wh = pade_row_ptr(p.whi, r, p.M, p.K, p.B, p.all_explicit);
      const float* wl = pade_row_ptr(p.wlo, r, p.M, p.K, p.B, p.all_explicit);
      for (int t = 2 * p.K + 1; t >= 0; --t) {
        const int d = t - p.K;
        if (r + d < 0 || r + d >= p.M) continue;
        ff_fma_acc_f(sh, sl, wh[t], wl[t], ah[d], al[d]);
      }
    }
    ff_norm(sh, sl);
    const size_t yo = (size_t)l * p.yl + (size_t)(r + 1) * p.ya;
    p.yh[yo] = sh;
    p.yl_[yo] = sl;
  }
}

// DE (+)= kappa^2 (E - E_old) - cz (y_x - y_y) in float-float (cz = 24 Z / (h_tau h): y is the Pade
// band on plain differences, the derivative being y / h), then G~ = 12 beta E + h^2 DE, on the
// E_z nodes; 0 on the walls.
__global__ void k_de_combine32(const float* __restrict__ eh, const float* __restrict__ el,
                               const float* __restrict__ oh, const float* __restrict__ ol,
                               const float* __restrict__ xh, const float* __restrict__ xl,
                               const float* __restrict__ yh, const float* __restrict__ yl, float* __restrict__ dh,
                               float* __restrict__ dl, float* __restrict__ gh, float* __restrict__ gl, int n,
                               float k2_hi, float k2_lo, float cz_hi, float cz_lo, float cb_hi, float cb_lo,
                               float h2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const size_t p = (size_t)j * n + i;
  if (i == 0 || j == 0 || i == n - 1 || j == n - 1) {
    dh[p] = dl[p] = gh[p] = gl[p] = 0.0f;
    return;
  }
  const float ehv = eh[p], elv = el[p];
  float ih, il, ch, cl;
  ff_diff(ehv, elv, oh[p], ol[p], ih, il);   // E^{n+1} - E^n
  ff_diff(xh[p], xl[p], yh[p], yl[p], ch, cl);  // y_x - y_y
  // the two products, each as (hi, error)
  const float ph = __fmul_rn(k2_hi, ih);
  float pl = fmaf(k2_hi, ih, -ph);
  pl = fmaf(k2_hi, il, pl);
  pl = fmaf(k2_lo, ih, pl);
  const float qh = __fmul_rn(cz_hi, ch);
  float ql = fmaf(cz_hi, ch, -qh);
  ql = fmaf(cz_hi, cl, ql);
  ql = fmaf(cz_lo, ch, ql);
  float th, tl;
  ff_diff(ph, pl, qh, ql, th, tl);  // the increment of DE (the two terms nearly cancel)
  // DE + increment
  float sh, sl;
  ff_diff(dh[p], dl[p], -th, -tl, sh, sl);
  ff_norm(sh, sl);
  dh[p] = sh;
  dl[p] = sl;
  // G~ = 12 beta E + h^2 DE
  const float pr = __fmul_rn(cb_hi, ehv);
  float e = fmaf(cb_hi, ehv, -pr);
  e = fmaf(cb_hi, elv, e);
  e = fmaf(cb_lo, ehv, e);
  e = fmaf(h2, sh, e);
  float g_hi = pr, g_lo = e;
  ff_norm(g_hi, g_lo);
  gh[p] = g_hi;
  gl[p] = g_lo;
}

struct Split2 {
  float hi, lo;
};
Split2 split2(double v) {
  Split2 s;
  s.hi = (float)v;
  s.lo = (float)(v - (double)s.hi);
  return s;
}

}  // namespace

ms_status tracked32_setup(ms_grid* g) {
  const size_t n = g->sh[EZ].size();
  float** planes[] = {&g->de_hi, &g->de_lo, &g->t32[0], &g->t32[1], &g->t32[2], &g->t32[3],
                      &g->t32[4], &g->t32[5], &g->t32[6], &g->t32[7]};
  for (float** q : planes) {
    if (dev_malloc(q, n * sizeof(float) + 256) != cudaSuccess) return MS_ENOMEM;
    if (cudaMemsetAsync(*q, 0, n * sizeof(float) + 256, g->stream) != cudaSuccess) return MS_ECUDA;
  }
  return MS_OK;
}

void tracked32_teardown(ms_grid* g) {
  dev_free(g->de_hi);
  dev_free(g->de_lo);
  g->de_hi = g->de_lo = nullptr;
  for (int k = 0; k < 8; ++k) {
    dev_free(g->t32[k]);
    g->t32[k] = nullptr;
  }
}

void tracked32_set_de(ms_grid* g, const double* de) {
  launch_split(de, g->de_hi, g->de_lo, g->sh[EZ].size(), g->stream);
}

ms_status step_mixed_tracked(ms_grid* g, int* nl) {
  const int N = g->N;
  const double N1 = N + 1.0, Nd = N;
  const double ne = N1 * N1, nh = Nd * N1;
  const MixedConsts k = mixed_consts(g);
  const size_t nE = g->sh[EZ].size();
  // Step 1 as in the FP32 step, keeping E^n for the increment
  if (cudaMemcpyAsync(g->t32[0], g->hi[EZ], nE * sizeof(float), cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess ||
      cudaMemcpyAsync(g->t32[1], g->lo[EZ], nE * sizeof(float), cudaMemcpyDeviceToDevice, g->stream) != cudaSuccess)
    return MS_ECUDA;
  prof_mark(g, KK_TRACKED32, 16.0 * ne);
  float* bE = g->s32[4];
  tiled_curl(g, 0, k.cb_hi, k.cb_lo, bE, nullptr);
  prof_mark(g, KK_CURL32, 8.0 * 2.0 * nh);
  const int fe[1] = {EZ};
  const float* be[1] = {bE};
  tiled_solve(g, 1, fe, be, k.S, k.d_hi, k.d_lo, k.omega, k.sE_hi, k.sE_lo);
  prof_mark(g, KK_SOLVE32, 16.0 * ne);
  // the unfiltered Pade curl of H in float-float: y_x = W delta_x H_y, y_y = W delta_y H_x
  const PadeTable& t = g->pade32[HALF_TO_NODE];
  BandF bx;
  bx.uh = g->hi[HY];
  bx.ul_ = g->lo[HY];
  bx.yh = g->t32[2];
  bx.yl_ = g->t32[3];
  bx.ua = 1;
  bx.ul = g->sh[HY].nx;  // H_y rows: N half-node values, N + 1 rows
  bx.ya = 1;
  bx.yl = N + 1;
  bx.nlines = N + 1;
  bx.whi = t.d_whi;
  bx.wlo = t.d_wlo;
  bx.M = t.M;
  bx.K = t.K;
  bx.B = t.B;
  bx.all_explicit = t.all_explicit;
  BandF by = bx;
  by.uh = g->hi[HX];
  by.ul_ = g->lo[HX];
  by.yh = g->t32[4];
  by.yl_ = g->t32[5];
  by.ua = g->sh[HX].nx;  // H_x columns: N + 1 columns of N half-node values
  by.ul = 1;
  by.ya = N + 1;
  by.yl = 1;
  {
    using T0 = BandFTile<0>;
    using T1 = BandFTile<1>;
    const dim3 g0((t.M + T0::OUTS - 1) / T0::OUTS, (N + 1 + T0::LINES - 1) / T0::LINES);
    const dim3 g1((t.M + T1::OUTS - 1) / T1::OUTS, (N + 1 + T1::LINES - 1) / T1::LINES);
    k_bandF32<0><<<g0, BF_THREADS, 0, g->stream>>>(bx);
    prof_mark(g, KK_TRACKED32, 8.0 * (nh + ne));
    k_bandF32<1><<<g1, BF_THREADS, 0, g->stream>>>(by);
    prof_mark(g, KK_TRACKED32, 8.0 * (nh + ne));
  }
  // DE update and G~_E
  {
    const double ht = g->ht, h = g->h;
    const Split2 k2 = split2(g->kappa2), cz = split2(24.0 * g->Z / (ht * h));
    const dim3 blk(32, 8), grd((N + 1 + 31) / 32, (N + 1 + 7) / 8);
    k_de_combine32<<<grd, blk, 0, g->stream>>>(g->hi[EZ], g->lo[EZ], g->t32[0], g->t32[1], g->t32[2], g->t32[3],
                                               g->t32[4], g->t32[5], g->de_hi, g->de_lo, g->t32[6], g->t32[7], N + 1,
                                               k2.hi, k2.lo, cz.hi, cz.lo, k.cb_hi, k.cb_lo, (float)(h * h));
    prof_mark(g, KK_TRACKED32, 4.0 * 12.0 * ne);
  }
  // Step 2 on G~_E with the filter off, then both H solves
  float* bxp = g->s32[2];
  float* byp = g->s32[3];
  tiled_curl_unfiltered(g, g->t32[6], g->t32[7], bxp, byp);
  prof_mark(g, KK_CURL32, 8.0 * ne);
  const int fh[2] = {HX, HY};
  const float* bh[2] = {bxp, byp};
  tiled_solve(g, 2, fh, bh, k.S, k.d_hi, k.d_lo, k.omega, k.sH_hi, k.sH_lo);
  prof_mark(g, KK_SOLVE32, 16.0 * 2.0 * nh);
  *nl += 9;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MS_OK : MS_ECUDA;
}

}  // namespace ms
