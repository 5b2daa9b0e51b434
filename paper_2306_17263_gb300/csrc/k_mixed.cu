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
// would be amplified by 1/theta in every step.  The kernels therefore take the first
// differences of the float-float state, (hi_{m+1} - hi_m) + (lo_{m+1} - lo_m), filter the
// differences (the filter commutes with D1~), and only then apply the well-conditioned A^{-1}
// band.  The Richardson residual forms the dominant diagonal product exactly (FMA), and
// the last correction is added to the state separately so the iteration cannot stall into a
// coherent bias.  The state is a float-float pair updated with error-free transformations.
//
// Kernels (k_tiled.cu): one right-hand-side tile kernel and one solve-and-update tile kernel
// per half-step, i.e. four launches per time step.
#include <cmath>
#include <string>

#include "k_fp64.cuh"
#include "k_mixed.cuh"
#include "k_tiled.cuh"

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

MixedConsts mixed_consts(const ms_grid* g) {
  const double c1h2 = g->c1 * g->h * g->h;
  const Split cb = split(12.0 * g->beta);
  const Split d = split(6.0 * c1h2);
  const Split sE = split(12.0 * g->Z / g->desc.r);
  const Split sH = split(12.0 / (g->desc.r * g->Z));
  MixedConsts k;
  k.cb_hi = cb.hi;
  k.cb_lo = cb.lo;
  k.d_hi = d.hi;
  k.d_lo = d.lo;
  k.omega = (float)(2.0 / (12.0 * c1h2 + 32.0));
  k.sE_hi = sE.hi;
  k.sE_lo = sE.lo;
  k.sH_hi = sH.hi;
  k.sH_lo = sH.lo;
  k.S = g->p1_sweeps32;
  return k;
}

ms_status step_mixed(ms_grid* g, int* nl) {
  const double N1 = g->N + 1.0, Nd = g->N;
  const double ne = N1 * N1, nh = Nd * N1;  // points of E_z and of each H component
  const MixedConsts k = mixed_consts(g);
  // Step 1: b = A^{-1} D1 G~_y (along x) - A^{-1} D1 G~_x (along y) on E_z, then the E solve
  float* bE = g->s32[4];
  tiled_curl(g, 0, k.cb_hi, k.cb_lo, bE, nullptr);
  // recorded bytes: the state each launch must touch (8 B per point per float-float read or
  // write), the algorithmic bytes of a step being 48 B per cell (each component read and written
  // once); the right-hand-side planes b are intermediates and are not counted
  prof_mark(g, KK_CURL32, 8.0 * 2.0 * nh);                   // H_x, H_y (hi, lo) read
  // sources in the units of b: 6 h^2 P1 x = b with E += (12 Z / r) x, so b = (h^3 r^2 / (2 Z)) R
  const double hr2 = g->h * g->h * g->h * g->desc.r * g->desc.r;
  if (g->nsrc) {  // H += (12 / (r Z)) x, so b = (h^3 r^2 Z / 2) R on the H side
    launch_src_time(g, hr2 / (2.0 * g->Z), hr2 * g->Z / 2.0);
    prof_mark(g, KK_SRC, 0.0);
    *nl += 1;
    if (g->d_walldata) {
      launch_wall_data(g);
      prof_mark(g, KK_SRC, 8.0 * 12.0 * N1);
      *nl += 1;
    }
    launch_src_e32(g, bE, hr2 / (2.0 * g->Z));
    prof_mark(g, KK_SRC, 8.0 * ne);
    *nl += 1;
  }
  const int fe[1] = {EZ};
  const float* be[1] = {bE};
  tiled_solve(g, 1, fe, be, k.S, k.d_hi, k.d_lo, k.omega, k.sE_hi, k.sE_lo);
  prof_mark(g, KK_SOLVE32, 16.0 * ne);                       // E (hi, lo) read and written
  // Step 2: b_x = -A^{-1} D1 G~_E (along y), b_y = +A^{-1} D1 G~_E (along x), then both H solves
  float* bx = g->s32[2];
  float* by = g->s32[3];
  tiled_curl(g, 1, k.cb_hi, k.cb_lo, bx, by);
  prof_mark(g, KK_CURL32, 8.0 * ne);                         // E (hi, lo) read
  if (g->nsrc) {
    launch_src_h32(g, bx, by, hr2 * g->Z / 2.0);
    prof_mark(g, KK_SRC, 16.0 * nh);
    *nl += 1;
  }
  const int fh[2] = {HX, HY};
  const float* bh[2] = {bx, by};
  tiled_solve(g, 2, fh, bh, k.S, k.d_hi, k.d_lo, k.omega, k.sH_hi, k.sH_lo);
  prof_mark(g, KK_SOLVE32, 16.0 * 2.0 * nh);                 // H_x, H_y (hi, lo) read and written
  if (g->nsrc) {
    launch_tick(g);
    prof_mark(g, KK_SRC, 0.0);
    *nl += 1;
  }
  *nl += 4;
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
    // the explicit rows of the tile kernels hold half-widths up to kTiledKMax
    if (t.K > kTiledKMax) {
      g_mixed_err = "FP32 Pade band half-width outside the range the tile kernels hold";
      return MS_EUNSUPPORTED;
    }
    std::vector<float> whi(t.w.size()), wlo(t.w.size());
    for (size_t k = 0; k < t.w.size(); ++k) {
      Split s = split(t.w[k]);
      whi[k] = s.hi;
      wlo[k] = s.lo;
    }
    if (dev_malloc(&t.d_whi, whi.size() * sizeof(float)) != cudaSuccess ||
        dev_malloc(&t.d_wlo, wlo.size() * sizeof(float)) != cudaSuccess) {
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
  const ms_status sw = ms_solver_sweeps(2, g->desc.r, MS_FP32_REFINED, 1e-10, &g->p1_sweeps32);
  if (sw != MS_OK) {
    g_mixed_err = "too many Richardson sweeps for the FP32 tile solve";
    return sw;
  }
  if (tiled_configure() != 0) {
    g_mixed_err = "cannot configure shared memory of the tile kernels";
    return MS_ECUDA;
  }
  // right-hand-side planes of the tile kernels: s32[4] (E_z), s32[2] (H_x), s32[3] (H_y)
  const size_t nmax = (size_t)(g->N + 1) * (g->N + 1);
  for (int k = 2; k < 5; ++k) {
    if (dev_malloc(&g->s32[k], nmax * sizeof(float) + 256) != cudaSuccess) {
      g_mixed_err = "cudaMalloc of FP32 scratch failed";
      return MS_ENOMEM;
    }
    cudaMemset(g->s32[k], 0, nmax * sizeof(float));
  }
  return MS_OK;
}

void mixed_teardown(ms_grid* g) {
  for (int k = 0; k < 2; ++k) {
    dev_free(g->pade32[k].d_whi);
    dev_free(g->pade32[k].d_wlo);
    g->pade32[k].d_whi = g->pade32[k].d_wlo = nullptr;
  }
}

}  // namespace ms
