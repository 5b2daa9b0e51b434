// Tiled kernels of the FP32_REFINED step: two launches per half-step.
//
//   k_curl_tile  : right-hand side b of one half-step on a 64 x 64 output tile.  For every
//                  Pade line through the tile it forms the first differences of the source
//                  state in float-float, delta_m = (hi_{m+1} - hi_m) + (lo_{m+1} - lo_m), filters
//                  them, d = 12 beta delta + L delta (the filter of Eq. "eq:ell" commutes with the
//                  difference: D1 (12 beta + L) u = (12 beta + L') D1 u with the ghost rules below),
//                  and applies A^{-1} (App. A.1, Eq. "eq:lhs"): rows near a wall as explicit rows
//                  of its band, interior rows as the two first-order recurrences A factors into.
//                  Step 1: b = A^{-1} D1 G~_y (along x) - A^{-1} D1 G~_x (along y) on E_z;
//                  Step 2: b_x = -A^{-1} D1 G~_E (along y), b_y = +A^{-1} D1 G~_E (along x).
//   k_solve_tile : S Richardson sweeps of 6 h^2 P1 (Def. "def:operatorsP") on the tile plus an
//                  (S-1)-cell halo in shared memory, then the float-float state update of the
//                  paper's E += h_tau E* / H += h_tau H* with the exact-product residual and
//                  the split last correction (see k_mixed.cu).
//
// Ghost rules of the difference field along a Pade line: a source that is Neumann along the
// line (H_y along x, H_x along y; even ghost u(-1) = u(0), Cor. "cor:ghost_cor") has zero
// differences beyond the ends; a source that is Dirichlet along the line (E_z, zero at the
// wall, filter zero there) has even differences (delta_{-1} = delta_0, delta_M = delta_{M-1}).
// Across the line every source is Dirichlet with stored zeros.
//
// Launch order: both kernels launch the boundary ring of tiles first (those take the general
// paths and run about twice as long), so they do not form the tail of the launch.
//
// Instruction budget: both kernels are bound by issue, not by DRAM, so loops have constant
// strides and 32-bit offsets, tiles away from the walls take block-uniform paths without any
// boundary test, and interior rows of A^{-1} (the same Toeplitz row for every grid,
// 24 (-rho) rho^|d| / (1 - rho^2), rho = -11 + sqrt(120)) cost two FMAs per output and
// recurrence instead of one per tap.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "k_fp64.cuh"
#include "k_tiled.cuh"

namespace ms {
namespace {

constexpr int TB = 64;               // output tile edge
constexpr int KMAX = kTiledKMax;     // largest band half-width of the explicit end rows
constexpr int NT = 512;              // threads per block
constexpr int NW = NT / 32;          // warps per block
constexpr int SEG = 8;               // outputs per segment of A^{-1} along a line (one per thread)
static_assert(TB / SEG == NW / 2, "two warps per 64 lines, one segment per thread");
constexpr int KR = 6;                // warm-up length of the interior recurrences
constexpr int DL = TB + 2 * KMAX + 2;  // filtered differences held per line
constexpr int DLP = DL | 1;            // odd row pitch: conflict-free across lanes
constexpr int XL = DL + 2;             // raw differences per line (one more on each side)
constexpr int XLP = XL | 1;
constexpr int XROWS = TB + 2;          // lines of raw differences (one more on each side)
constexpr int YSP = TB + 1;
constexpr int RS = 64;                     // solve region edge (output tile + 2 x halo)
constexpr int RSP = RS + 1;
constexpr int MAXR = (RS + NW / 2 - 1) / (NW / 2);  // rows of a sweep strip, at most
constexpr int PF = 4;                                // state rows fetched ahead in the last sweep

// interior A^{-1} as two first-order recurrences: rho, 1 / (1 - rho), and the scale (1 - rho)^2
// split hi + lo (rho is the FP32 root, so the scale gives the recurrences a DC gain of exactly 1)
__constant__ float c_rec[4];

// Programmatic dependent launch.  A tile kernel lets the next kernel of the stream start launching
// as soon as every one of its own blocks has started (pdl_trigger), and reads no global memory
// before every kernel it depends on has completed and its writes are visible (pdl_wait).  Blocks
// that wait hold only slots the earlier grids no longer need (all their blocks are resident by
// then), and launch latency at kernel boundaries overlaps the previous kernel's tail.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

struct PhaseArgs {
  const float* hi;
  const float* lo;
  int snx;           // row length of the source array
  int axis;          // 0: lines along x, 1: lines along y
  int M;             // differences (= outputs) per line
  int ghost_even;    // 1: source Dirichlet along the line
  int n_across;      // source lines
  const float* whi;  // A^{-1} band table (hi, lo), layout of PadeTable
  const float* wlo;
  int Kt, Bt, all_explicit;
  float cb_hi, cb_lo;  // 12 beta
};

// Interior rows of A^{-1} d for the segment of SEG outputs starting at row rf (drow[j] = d_{rf+j}).
// A = (1/24) tridiag(1, 22, 1) factors as (1 - rho E^-1)(1 - rho E) / (1 - rho)^2 (rho^2 + 22 rho
// + 1 = 0, so (1 - rho)^2 = -24 rho), and A^{-1} d is a forward recurrence z_i = d_i + rho z_{i-1},
// a backward one y_i = z_i + rho y_{i+1}, and the scale (1 - rho)^2.  Each recurrence starts
// KR + 1 rows outside the segment from the steady state of the value there (d / (1 - rho),
// z / (1 - rho)): its error reaches the segment damped by |rho|^(KR+1) ~ 4e-10, times the change
// of d over those rows.  Every product enters through one FMA, so no tap is dropped against a
// larger partial sum.  SKIP: rows inside the line whose row of A^{-1} is not the interior one
// (r < B or r >= M - B) are left to the explicit rows; rows past the line are emitted (unused).
template <bool SKIP, typename Emit>
__device__ __forceinline__ void interior_rows(const float* drow, int rf, int M, int B, Emit emit) {
  const float rho = c_rec[0], inv1mr = c_rec[1];
  float zs[SEG + KR];
  float z = drow[-KR - 1] * inv1mr;
#pragma unroll
  for (int q = -KR; q < SEG + KR; ++q) {
    z = fmaf(rho, z, drow[q]);
    if (q >= 0) zs[q] = z;
  }
  float y = z * inv1mr;
#pragma unroll
  for (int q = SEG + KR - 1; q >= 0; --q) {
    y = fmaf(rho, y, zs[q]);
    if (q < SEG) {
      const int r = rf + q;
      if (!SKIP || r < 0 || r >= M || (r >= B && r < M - B)) emit(q, fmaf(c_rec[2], y, c_rec[3] * y));
    }
  }
}

// Explicit row r of the band table (dc[j] = d_{r+j}): the tap loop unrolled to the largest
// half-width the tile holds, taps beyond the table's K predicated off; taps past the line read the
// zero differences stored there, so the sums are those of the taps inside the line.  Rows past
// the line give 0.
__device__ __forceinline__ float explicit_row(const PhaseArgs& p, const float* dc, int r) {
  if (r < 0 || r >= p.M) return 0.0f;
  const float* wh = pade_row_ptr(p.whi, r, p.M, p.Kt, p.Bt, p.all_explicit) + p.Kt;  // wh[d]: d_{r+d}
  const float* wl = pade_row_ptr(p.wlo, r, p.M, p.Kt, p.Bt, p.all_explicit) + p.Kt;
  float acc = 0.0f, lo = 0.0f;
#pragma unroll
  for (int dist = KMAX + 1; dist >= 1; --dist) {
    if (dist <= p.Kt + 1) {
      const float dm = dc[dist];
      acc = fmaf(__ldg(wh + dist), dm, acc);
      lo = fmaf(__ldg(wl + dist), dm, lo);
    }
    if (dist <= p.Kt) {
      const float dm = dc[-dist];
      acc = fmaf(__ldg(wh - dist), dm, acc);
      lo = fmaf(__ldg(wl - dist), dm, lo);
    }
  }
  lo = fmaf(__ldg(wl), dc[0], lo);
  return fmaf(__ldg(wh), dc[0], acc + lo);
}

// One Pade phase on the tile: y(a, r) for lines c = c0 + a (a < TB) and outputs r = r0 + o
// (o < TB), handed to out(a, o, y).  Caller synchronises before reusing dlt / dd.
// FILTER false: d = delta (the source is already filtered, as G~_E of the tracked-Delta-E step).
template <bool FILTER, typename Out>
__device__ __forceinline__ void pade_phase(const PhaseArgs& p, int c0, int r0, float* dlt, float* dd, Out out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int mb = r0 - KMAX - 1;  // along index of raw-difference column 0
  // the whole strip lies inside the lines and needs no ghost: no per-element tests
  const bool inside = (mb >= 0) && (mb + XL <= p.M) && (c0 >= 1) && (c0 + TB + 1 <= p.n_across);
  // 1) raw differences delta on lines c0-1 .. c0+TB, along m in [mb, mb + XL)
  if (inside) {
    // block-uniform path: fixed trip counts, constant offsets, every load of a thread in flight
    // before its first use
    if (p.axis == 0) {
      const size_t base = (size_t)(c0 - 1) * p.snx + mb + lane;
      const float* hb = p.hi + base;
      const float* lb = p.lo + base;
      float* db = dlt + lane;
#pragma unroll 2
      for (int a = warp; a < XROWS; a += NW) {
        const float* hr = hb + (size_t)a * p.snx;
        const float* lr = lb + (size_t)a * p.snx;
#pragma unroll
        for (int cc = 0; cc < (XL + 31) / 32; ++cc)
          if (32 * cc + 32 <= XL || lane + 32 * cc < XL)
            db[a * XLP + 32 * cc] = (hr[32 * cc + 1] - hr[32 * cc]) + (lr[32 * cc + 1] - lr[32 * cc]);
      }
    } else {
      // lines a = lane, lane + 32 (lanes along x); warp w walks rows q = QW w .. QW w + QW - 1,
      // carrying each source row in registers to the next difference (every row loaded once);
      // the two last lines with lanes along m
      constexpr int QW = (XL + NW - 1) / NW;
      const int q0 = QW * warp;
      const size_t sn = (size_t)p.snx;
      const size_t base = (size_t)(mb + q0) * sn + (c0 - 1) + lane;
      const float* hr = p.hi + base;
      const float* lr = p.lo + base;
      float h0 = hr[0], h1 = hr[32], l0 = lr[0], l1 = lr[32];
#pragma unroll
      for (int t = 0; t < QW; ++t) {
        if (q0 + t < XL) {  // warp-uniform
          hr += sn;
          lr += sn;
          const float nh0 = hr[0], nh1 = hr[32], nl0 = lr[0], nl1 = lr[32];
          dlt[lane * XLP + q0 + t] = (nh0 - h0) + (nl0 - l0);
          dlt[(lane + 32) * XLP + q0 + t] = (nh1 - h1) + (nl1 - l1);
          h0 = nh0;
          h1 = nh1;
          l0 = nl0;
          l1 = nl1;
        }
      }
      for (int idx = threadIdx.x; idx < (XROWS - 64) * XL; idx += NT) {
        const int e = idx / XL, q = idx - e * XL;
        const size_t g0 = (size_t)(mb + q) * sn + (c0 - 1) + 64 + e;
        dlt[(64 + e) * XLP + q] = (p.hi[g0 + sn] - p.hi[g0]) + (p.lo[g0 + sn] - p.lo[g0]);
      }
    }
  } else if (p.axis == 0) {
    // strip at a line end or with lines past the array: the ghost rule per element, zero lines
    // past the array; rows unrolled by two and chunks unrolled so the loads are in flight together
#pragma unroll 2
    for (int a = warp; a < XROWS; a += NW) {
      const int c = c0 - 1 + a;
      const bool line_ok = c >= 0 && c < p.n_across;
      const float* hr = p.hi + (size_t)(line_ok ? c : 0) * p.snx;
      const float* lr = p.lo + (size_t)(line_ok ? c : 0) * p.snx;
#pragma unroll
      for (int cc = 0; cc < (XL + 31) / 32; ++cc) {
        const int q = lane + 32 * cc;
        if (32 * cc + 32 <= XL || q < XL) {
          const int m = mb + q;
          float v = 0.0f;
          if (line_ok) {
            int mm = m;
            bool zero = false;
            if (m < 0 || m >= p.M) {
              if (!p.ghost_even || m < -1 || m > p.M) zero = true;
              else mm = (m < 0) ? 0 : p.M - 1;
            }
            if (!zero) v = (hr[mm + 1] - hr[mm]) + (lr[mm + 1] - lr[mm]);
          }
          dlt[a * XLP + q] = v;
        }
      }
    }
  } else {
    // same for lines along y: lanes across the lines (zero past the array, load index clamped
    // into it), warp along the rows with the ghost rule per row; rows unrolled by two
    const int ca = c0 - 1 + lane, cb = c0 + 31 + lane;
    const bool va = ca >= 0 && ca < p.n_across, vb = cb >= 0 && cb < p.n_across;
    const int ka = va ? ca : 0, kb = vb ? cb : 0;
    const size_t sn = (size_t)p.snx;
#pragma unroll 2
    for (int q = warp; q < XL; q += NW) {
      int m = mb + q;
      bool zero = false;
      if (m < 0 || m >= p.M) {
        if (!p.ghost_even || m < -1 || m > p.M) zero = true;
        else m = (m < 0) ? 0 : p.M - 1;
      }
      const size_t row0 = (size_t)(zero ? 0 : m) * sn;
      const float* h0 = p.hi + row0;
      const float* l0 = p.lo + row0;
      float v0 = 0.0f, v1 = 0.0f;
      if (!zero) {
        v0 = (h0[sn + ka] - h0[ka]) + (l0[sn + ka] - l0[ka]);
        v1 = (h0[sn + kb] - h0[kb]) + (l0[sn + kb] - l0[kb]);
      }
      dlt[lane * XLP + q] = va ? v0 : 0.0f;
      dlt[(lane + 32) * XLP + q] = vb ? v1 : 0.0f;
    }
    for (int idx = threadIdx.x; idx < (XROWS - 64) * XL; idx += NT) {  // the last two lines
      const int e = idx / XL, q = idx - e * XL;
      const int c = c0 + 63 + e;
      int m = mb + q;
      bool zero = !(c >= 0 && c < p.n_across);
      if (!zero && (m < 0 || m >= p.M)) {
        if (!p.ghost_even || m < -1 || m > p.M) zero = true;
        else m = (m < 0) ? 0 : p.M - 1;
      }
      float v = 0.0f;
      if (!zero) {
        const size_t g0 = (size_t)m * sn + c;
        v = (p.hi[g0 + sn] - p.hi[g0]) + (p.lo[g0 + sn] - p.lo[g0]);
      }
      dlt[(64 + e) * XLP + q] = v;
    }
  }
  __syncthreads();
  // 2) filtered differences d = 12 beta delta + L delta on lines c0 .. c0+TB-1, m in [mb+1, mb+1+DL);
  //    the 12 beta delta term dominates (beta = 1 + 2/r^2), so L delta is summed plainly
  if (inside) {
    // warp w filters lines 4w .. 4w+3, walking down them: the differences above and below a line
    // are the centres of its neighbour lines, carried in registers (three shared loads per element)
    constexpr int LPW = TB / NW;  // lines per warp
    constexpr int NCC = (DL + 31) / 32;
    const int a0 = LPW * warp;
    float up[NCC], mid[NCC];
#pragma unroll
    for (int cc = 0; cc < NCC; ++cc) {
      const bool ok = 32 * cc + 32 <= DL || lane + 32 * cc < DL;
      const float* r0 = dlt + a0 * XLP + 1 + lane + 32 * cc;  // line a0 - 1 of the filter
      up[cc] = ok ? r0[0] : 0.0f;
      mid[cc] = ok ? r0[XLP] : 0.0f;
    }
#pragma unroll
    for (int it = 0; it < LPW; ++it) {
      const int a = a0 + it;
      const float* r1 = dlt + (a + 1) * XLP + 1 + lane;
      float* o = dd + a * DLP + lane;
#pragma unroll
      for (int cc = 0; cc < NCC; ++cc) {
        if (32 * cc + 32 <= DL || lane + 32 * cc < DL) {
          const int q = 32 * cc;
          const float x = mid[cc];
          const float dn = r1[q + XLP];
          if (FILTER) {
            const float lap = fmaf(-4.0f, x, (r1[q - 1] + r1[q + 1]) + (up[cc] + dn));
            o[q] = fmaf(p.cb_hi, x, fmaf(p.cb_lo, x, lap));
          } else {
            o[q] = x;
          }
          up[cc] = x;
          mid[cc] = dn;
        }
      }
    }
  } else
  for (int a = warp; a < TB; a += NW) {
    const int c = c0 + a;
    const bool line_ok = inside || (c >= 1 && c <= p.n_across - 2);
    const float* r1 = dlt + (a + 1) * XLP + 1;
    for (int q = lane; q < DL; q += 32) {
      const int m = mb + 1 + q;
      float v = 0.0f;
      if (line_ok && (inside || (m >= 0 && m < p.M))) {
        const float x = r1[q];
        if (FILTER) {
          const float lap = ((r1[q - 1] - x) + (r1[q + 1] - x)) + ((r1[q - XLP] - x) + (r1[q + XLP] - x));
          v = fmaf(p.cb_hi, x, fmaf(p.cb_lo, x, lap));
        } else {
          v = x;
        }
      }
      dd[a * DLP + q] = v;
    }
  }
  __syncthreads();
  // 3) A^{-1} d: lane -> line, warp -> (line half, segment of SEG outputs).  Rows whose row of
  //    A^{-1} is the interior one come from the recurrences; the explicit rows near the ends of
  //    the line are dealt out over the line's TB / SEG threads.
  const int a = lane + 32 * (warp & 1);
  const int s = warp >> 1;
  const int rf = r0 + s * SEG;  // first output of this segment
  const float* drow = dd + a * DLP + (rf - (mb + 1));  // drow[j] = d_{rf + j}
  auto emit = [&](int q, float v) { out(a, s * SEG + q, v); };
  if (!p.all_explicit && r0 >= p.Bt && r0 + TB - 1 < p.M - p.Bt) {  // block-uniform: no end row
    interior_rows<false>(drow, rf, p.M, p.Bt, emit);
  } else {
    if (!p.all_explicit) interior_rows<true>(drow, rf, p.M, p.Bt, emit);
    // explicit rows of the tile: [max(r0, 0), min(B, r0 + TB)) and [max(M - B, r0), min(M, r0 + TB));
    // every row of the tile when the table is all explicit (rows past the line give 0)
    int s1, n1, s2, n2;
    if (p.all_explicit) {
      s1 = r0; n1 = TB; s2 = 0; n2 = 0;
    } else {
      s1 = max(r0, 0);
      n1 = max(0, min(p.Bt, r0 + TB) - s1);
      s2 = max(p.M - p.Bt, r0);
      n2 = max(0, min(p.M, r0 + TB) - s2);
    }
    const float* dline = dd + a * DLP - (mb + 1);  // dline[m] = d_m
    for (int t = s; t < n1 + n2; t += TB / SEG) {
      const int r = t < n1 ? s1 + t : s2 + (t - n1);
      out(a, r - r0, explicit_row(p, dline + r, r));
    }
  }
}

}  // namespace

struct CurlArgs {
  PhaseArgs ph[2];
  float* b0;  // Step 1: b on E_z;  Step 2: b_x on H_x
  float* b1;  // Step 2: b_y on H_y
  int N;
  int ntiles;  // tiles per row of the cavity (batched launches)
};

namespace {

// The TB x TB tile ys (row jj, column ii at ys[jj * YSP + ii]) to dst[jj * ld + ii], negated if
// NEG, for a tile whose entries all lie inside the array and off the walls: no tests, strides only.
template <bool NEG>
__device__ __forceinline__ void store_tile(float* dst, size_t ld, const float* ys) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* d = dst + (size_t)warp * ld + lane;
  const float* y = ys + warp * YSP + lane;
  const size_t st = (size_t)NW * ld;
#pragma unroll
  for (int k = 0; k < TB / NW; ++k) {
    const float v0 = y[k * NW * YSP], v1 = y[k * NW * YSP + 32];
    d[0] = NEG ? -v0 : v0;
    d[32] = NEG ? -v1 : v1;
    d += st;
  }
}

// STEP 0: right-hand side of Step 1 on E_z; STEP 1: right-hand sides of Step 2 on H_x, H_y;
// the tile with origin (i0, j0).
template <int STEP, bool FILTER = true>
__device__ __forceinline__ void curl_body(const CurlArgs& A, int i0, int j0) {
  extern __shared__ float sm[];
  float* dlt = sm;
  float* dd = dlt + XROWS * XLP;
  float* ys = dd + TB * DLP;
  const int N = A.N;
  // every output of the tile is off the walls and inside its array (all three layouts)
  const bool interior = i0 >= 1 && j0 >= 1 && i0 + TB <= N && j0 + TB <= N;
  if (STEP == 0) {
    // x-Pade of H_y: line = row j (c0 = j0), output node i = r + 1 (r0 = i0 - 1)
    pade_phase<FILTER>(A.ph[0], j0, i0 - 1, dlt, dd, [&](int a, int o, float v) { ys[a * YSP + o] = v; });
    __syncthreads();
    // y-Pade of H_x: line = column i (c0 = i0), output node j = r + 1 (r0 = j0 - 1)
    pade_phase<FILTER>(A.ph[1], i0, j0 - 1, dlt, dd, [&](int a, int o, float v) { ys[o * YSP + a] -= v; });
    __syncthreads();
    if (interior) {
      store_tile<false>(A.b0 + (size_t)j0 * (N + 1) + i0, (size_t)(N + 1), ys);
      return;
    }
    for (int jj = threadIdx.x >> 5; jj < TB; jj += NW) {
      const int j = j0 + jj;
      if (j > N) break;
      for (int ii = threadIdx.x & 31; ii < TB; ii += 32) {
        const int i = i0 + ii;
        if (i > N) break;
        const bool in = (i >= 1 && i <= N - 1 && j >= 1 && j <= N - 1);
        A.b0[(size_t)j * (N + 1) + i] = in ? ys[jj * YSP + ii] : 0.0f;
      }
    }
  } else {
    // y-Pade of E for H_x: line = column i (c0 = i0), output half-row jh = r (r0 = j0)
    pade_phase<FILTER>(A.ph[0], i0, j0, dlt, dd, [&](int a, int o, float v) { ys[o * YSP + a] = v; });
    __syncthreads();
    if (interior) store_tile<true>(A.b0 + (size_t)j0 * (N + 1) + i0, (size_t)(N + 1), ys);
    else
    for (int jj = threadIdx.x >> 5; jj < TB; jj += NW) {
      const int jh = j0 + jj;
      if (jh >= N) break;
      for (int ii = threadIdx.x & 31; ii < TB; ii += 32) {
        const int i = i0 + ii;
        if (i > N) break;
        A.b0[(size_t)jh * (N + 1) + i] = (i >= 1 && i <= N - 1) ? -ys[jj * YSP + ii] : 0.0f;
      }
    }
    __syncthreads();
    // x-Pade of E for H_y: line = row j (c0 = j0), output half-column ih = r (r0 = i0)
    pade_phase<FILTER>(A.ph[1], j0, i0, dlt, dd, [&](int a, int o, float v) { ys[a * YSP + o] = v; });
    __syncthreads();
    if (interior) {
      store_tile<false>(A.b1 + (size_t)j0 * N + i0, (size_t)N, ys);
      return;
    }
    for (int jj = threadIdx.x >> 5; jj < TB; jj += NW) {
      const int j = j0 + jj;
      if (j > N) break;
      for (int ii = threadIdx.x & 31; ii < TB; ii += 32) {
        const int ih = i0 + ii;
        if (ih >= N) break;
        A.b1[(size_t)j * N + ih] = (j >= 1 && j <= N - 1) ? ys[jj * YSP + ii] : 0.0f;
      }
    }
  }
}

// Launch order of the tiles of an nt x nt grid: the boundary ring first, then the interior.  Ring
// tiles take the general paths (line ends, ghost lines, explicit Pade rows) and run about twice as
// long as interior tiles; started first, they no longer form the tail of the launch.
__host__ __device__ __forceinline__ void ring_first_tile(int b, int nt, int* tx, int* ty) {
  const int ring = nt > 1 ? 4 * (nt - 1) : 1;
  if (b >= ring) {  // interior tiles, row by row
    const int k = b - ring, w = nt - 2;
    *tx = 1 + k % w;
    *ty = 1 + k / w;
  } else if (b < nt) {  // first row
    *tx = b;
    *ty = 0;
  } else if (b < 2 * nt) {  // last row
    *tx = b - nt;
    *ty = nt - 1;
  } else {  // first and last columns, rows 1 .. nt-2
    const int k = b - 2 * nt;
    *tx = (k & 1) ? nt - 1 : 0;
    *ty = 1 + (k >> 1);
  }
}

template <int STEP, bool FILTER = true>
__global__ void __launch_bounds__(NT, 3) k_curl_tile(CurlArgs A) {
  pdl_trigger();
  pdl_wait();
  int tx, ty;
  ring_first_tile(blockIdx.y * gridDim.x + blockIdx.x, gridDim.x, &tx, &ty);
  curl_body<STEP, FILTER>(A, tx * TB, ty * TB);
}

// Words of a small argument struct copied from global to shared memory by the first warp.
template <typename T>
__device__ __forceinline__ void copy_args(T* dst, const T* src) {
  static_assert(sizeof(T) % 4 == 0, "argument structs are made of 4-byte words");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int k = threadIdx.x; k < (int)(sizeof(T) / 4); k += NT) d[k] = s[k];
  __syncthreads();
}

// Batched form: item w is tile work[2w+1] of cavity work[2w]; block b takes items b, b + gridDim.x,
// ... (one item per block when the grid covers the list, persistent blocks when it does not).
template <int STEP>
__global__ void __launch_bounds__(NT, 3) k_curl_batch(const CurlArgs* __restrict__ args, const int* __restrict__ work,
                                                      int nwork) {
  __shared__ CurlArgs sA;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int cav = work[2 * w], t = work[2 * w + 1];
    copy_args(&sA, args + cav);
    const int nt = sA.ntiles;
    curl_body<STEP>(sA, (t % nt) * TB, (t / nt) * TB);
    __syncthreads();  // sA and the tile buffers are rewritten by the next item
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
struct SolveArgs {
  const float* b[2];
  float* hi[2];
  float* lo[2];
  int nx[2], ny[2], bcx[2], bcy[2];
  int S;
  float d_hi, d_lo, omega, s_hi, s_lo;
  int ntiles;  // tiles per row of the cavity (batched launches)
};

namespace {

// (hi, lo) += (S_hi + S_lo) x with error-free transformations (see k_mixed.cu).
__device__ __forceinline__ void ff_add_scaled_t(float& hi, float& lo, float x, float s_hi, float s_lo) {
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

// (hi, lo) += (s_hi + s_lo)(x + c) for the last Richardson iterate x and its correction c (|c| is
// below |x| by the contraction factor except where both are negligible): x + c = s + t by Fast2Sum,
// then one two-product s_hi s and one two-sum into the pair, with s_lo s and s_hi t folded into the
// product's error term.  x and c are never rounded into one float, so the correction's low bits
// reach the state (rounding them away would shrink every increment coherently).
__device__ __forceinline__ void ff_add_scaled2_t(float& hi, float& lo, float x, float c, float s_hi, float s_lo) {
  const float s = __fadd_rn(x, c);
  const float t = __fsub_rn(c, __fsub_rn(s, x));
  const float p = __fmul_rn(s_hi, s);
  float e = fmaf(s_hi, s, -p);
  e = fmaf(s_lo, s, e);
  e = fmaf(s_hi, t, e);
  const float u = __fadd_rn(hi, p);
  const float bb = __fsub_rn(u, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(u, bb)), __fsub_rn(p, bb));
  const float l = __fadd_rn(lo, __fadd_rn(err, e));
  const float h2 = __fadd_rn(u, l);
  lo = __fsub_rn(l, __fsub_rn(h2, u));
  hi = h2;
}

// Residual b - d x - rest of 6 h^2 P1 x = b (d the diagonal, rest the stencil Laplacians): the
// product (d_hi + d_lo) x enters exactly, through two FMAs (b - d_hi x, then - d_lo x), each
// rounded once at the size of b - d x.
__device__ __forceinline__ float p1_resid(float b, float x, float d_hi, float d_lo, float rest) {
  return fmaf(-d_lo, x, fmaf(-d_hi, x, b)) - rest;
}

// Fill the even ghosts of the Neumann axes from the edge values (only tiles at such an edge).
__device__ __forceinline__ void fill_ghosts(float* x, int gx0, int gy0, int nx, int ny, bool neu_x, bool neu_y) {
  if (neu_x) {
    const int lg0 = -1 - gx0, lg1 = nx - gx0;  // local columns of the ghosts gx = -1 and gx = nx
    for (int ly = threadIdx.x; ly < RS; ly += NT) {
      if (lg0 >= 0 && lg0 + 1 < RS) x[ly * RSP + lg0] = x[ly * RSP + lg0 + 1];
      if (lg1 >= 1 && lg1 < RS) x[ly * RSP + lg1] = x[ly * RSP + lg1 - 1];
    }
  }
  if (neu_y) {
    const int lg0 = -1 - gy0, lg1 = ny - gy0;
    for (int lx = threadIdx.x; lx < RS; lx += NT) {
      if (lg0 >= 0 && lg0 + 1 < RS) x[lg0 * RSP + lx] = x[(lg0 + 1) * RSP + lx];
      if (lg1 >= 1 && lg1 < RS) x[lg1 * RSP + lx] = x[(lg1 - 1) * RSP + lx];
    }
  }
}

// Sweeps 1 .. S-1 of one region (see solve_body); EDGE: the region touches a wall, so points
// off the unknowns are masked and Neumann ghosts refilled after every sweep.
// One column strip of one sweep: rows ly0 .. ly1-1 of column c, sliding down a window of rows
// ly-1, ly, ly+1.  The residual's dominant term d x enters exactly (p1_resid), so the stencil
// Laplacians around it are summed plainly (their rounding is ~1e-3 ulp of the residual).
// LAST: add the iterate and its correction to the state instead of writing the next iterate.
template <bool EDGE, bool LAST>
__device__ __forceinline__ void sweep_column(const SolveArgs& A, const float* bs, const float* xcol, float* xn, int c,
                                             int ly0, int ly1, int gx, int gy0, int nx, int ny, int bcy,
                                             bool col_unk, float* shi, float* slo) {
  float a0 = xcol[(ly0 - 1) * RSP];
  float b0 = xcol[ly0 * RSP];
  float lxa = fmaf(-2.0f, a0, xcol[(ly0 - 1) * RSP - 1] + xcol[(ly0 - 1) * RSP + 1]);
  float lxb = fmaf(-2.0f, b0, xcol[ly0 * RSP - 1] + xcol[ly0 * RSP + 1]);
  if constexpr (LAST) {
    const size_t gp = (size_t)(gy0 + ly0) * nx + gx;
    // the state of PF rows at a time is fetched before the first of them is updated
#pragma unroll
    for (int t0 = 0; t0 < MAXR; t0 += PF) {
      float ph_[PF], pl_[PF];
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int ly = ly0 + t0 + u;
        const bool unk =
            ly < ly1 && (!EDGE || (col_unk && gy0 + ly >= 0 && gy0 + ly < ny && interior(bcy, gy0 + ly, ny)));
        ph_[u] = unk ? shi[gp + (size_t)(t0 + u) * nx] : 0.0f;
        pl_[u] = unk ? slo[gp + (size_t)(t0 + u) * nx] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const int ly = ly0 + t0 + u;
        if (ly >= ly1) break;
        const float* row = xcol + (ly + 1) * RSP;
        const float cm = row[-1], c0v = row[0], cp = row[1];
        const float lxc = fmaf(-2.0f, c0v, cm + cp);
        const float x = b0;
        const float lyv = fmaf(-2.0f, x, a0 + c0v);
        const float lxly = fmaf(-2.0f, lxb, lxa + lxc);
        const float rest = fmaf(-6.0f, lxb + lyv, -lxly);
        const float res = p1_resid(bs[ly * RSP + c], x, A.d_hi, A.d_lo, rest);
        const float corr = A.omega * res;
        const bool unk = !EDGE || (col_unk && gy0 + ly >= 0 && gy0 + ly < ny && interior(bcy, gy0 + ly, ny));
        if (unk) {
          float h = ph_[u], l = pl_[u];
          ff_add_scaled2_t(h, l, x, corr, A.s_hi, A.s_lo);
          shi[gp + (size_t)(t0 + u) * nx] = h;
          slo[gp + (size_t)(t0 + u) * nx] = l;
        }
        a0 = b0;
        lxa = lxb;
        b0 = c0v;
        lxb = lxc;
      }
    }
  } else {
#pragma unroll 4
  for (int ly = ly0; ly < ly1; ++ly) {
    const float* row = xcol + (ly + 1) * RSP;
    const float cm = row[-1], c0v = row[0], cp = row[1];
    const float lxc = fmaf(-2.0f, c0v, cm + cp);
    const float x = b0;
    const float lyv = fmaf(-2.0f, x, a0 + c0v);
    const float lxly = fmaf(-2.0f, lxb, lxa + lxc);
    const float rest = fmaf(-6.0f, lxb + lyv, -lxly);
    const float res = p1_resid(bs[ly * RSP + c], x, A.d_hi, A.d_lo, rest);
    const float corr = A.omega * res;
    bool unk = true;
    if (EDGE) {
      const int gy = gy0 + ly;
      unk = col_unk && gy >= 0 && gy < ny && interior(bcy, gy, ny);
    }
    xn[ly * RSP + c] = unk ? x + corr : 0.0f;
    a0 = b0;
    lxa = lxb;
    b0 = c0v;
    lxb = lxc;
  }
  }
}

// Sweeps 1 .. S-1 of one region (see solve_body); EDGE: the region touches a wall, so points
// off the unknowns are masked and Neumann ghosts refilled after every sweep.
template <bool EDGE>
__device__ __forceinline__ void solve_sweeps(const SolveArgs& A, const float* bs, float* xa, float* xb, int gx0,
                                             int gy0, int nx, int ny, int bcx, int bcy, float* shi, float* slo,
                                             bool neu_x, bool neu_y) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = lane + 32 * (warp & 1);
  const int st = warp >> 1;
  const int gx = gx0 + c;
  const bool col_unk = !EDGE || (gx >= 0 && gx < nx && interior(bcx, gx, nx));
  float* xc = xa;
  float* xn = xb;
  for (int k = 1; k < A.S; ++k) {
    const bool last = (k == A.S - 1);
    const int rps = (RS - 2 * k + NW / 2 - 1) / (NW / 2);
    const int ly0 = k + st * rps, ly1 = min(ly0 + rps, RS - k);
    if (c >= k && c < RS - k && ly0 < ly1) {
      if (last)
        sweep_column<EDGE, true>(A, bs, xc + c, xn, c, ly0, ly1, gx, gy0, nx, ny, bcy, col_unk, shi, slo);
      else
        sweep_column<EDGE, false>(A, bs, xc + c, xn, c, ly0, ly1, gx, gy0, nx, ny, bcy, col_unk, shi, slo);
    }
    __syncthreads();
    if (EDGE && !last && (neu_x || neu_y)) {
      fill_ghosts(xn, gx0, gy0, nx, ny, neu_x, neu_y);
      __syncthreads();
    }
    float* t = xc;
    xc = xn;
    xn = t;
  }
}

// Interior regions (every point an unknown, no boundary rule anywhere): warp w owns rows
// FR w .. FR w + FR - 1 of the region and lane l the column pair 2l, 2l + 1.  b and the current
// iterate of a thread's own points stay in registers; shared memory holds each iterate once for the
// neighbours, in two planes with a zero pad row above and below and two pad columns on each side
// (the row pitch keeps every column pair 8-byte aligned for one 64-bit access).  Every sweep updates
// every region point: after sweep k the points within k of the region's edge are wrong (their outer
// neighbours are the pads), which never reaches the output tile since k <= S - 1 = H.  The
// arithmetic per point is that of sweep_column, operation for operation.
constexpr int FR = RS / NW;           // rows per thread
constexpr int XP2 = RS + 4;           // row pitch of the interior planes
constexpr int XPL = (RS + 2) * XP2;   // floats per interior plane
static_assert(FR * NW == RS && 2 * 32 == RS, "interior solve layout: 16 warps x FR rows, 32 lanes x 2 columns");

__device__ __forceinline__ int xi2(int ly, int lx) { return (ly + 1) * XP2 + lx + 2; }

// One sweep of an interior region.  LAST: add the iterate and its correction to the state at the
// output points (region rows and columns H .. RS-1-H) instead of writing the next iterate.
// MASK: the region touches a wall; bit 2k + j of um marks the thread's unknowns (inside the field
// and off its Dirichlet walls).  Every other point is held at 0 (Neumann ghosts are refilled by the
// caller), and only unknowns read or write the state.
template <bool LAST, bool MASK>
__device__ __forceinline__ void interior_sweep(const SolveArgs& A, const float* xc, float* xn, const float (&bv)[FR][2],
                                               float (&xv)[FR][2], int r0, int c, float* shi, float* slo, int gp,
                                               int nx, int H, unsigned um) {
  auto unk = [&](int k, int j) { return !MASK || ((um >> (2 * k + j)) & 1u); };
  // output rows (the same for every lane of the warp) and output columns of the thread
  float sh[FR][2], sl[FR][2];
  bool rowok[FR];
  const bool colok0 = c >= H && c < RS - H, colok1 = c + 1 >= H && c + 1 < RS - H;
  if constexpr (LAST) {  // the state of the output rows, fetched ahead of the arithmetic (the region
                         // lies inside the field, so both columns may be read)
#pragma unroll
    for (int k = 0; k < FR; ++k) {
      rowok[k] = r0 + k >= H && r0 + k < RS - H;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        sh[k][j] = rowok[k] && unk(k, j) ? shi[gp + k * nx + j] : 0.0f;
        sl[k][j] = rowok[k] && unk(k, j) ? slo[gp + k * nx + j] : 0.0f;
      }
    }
  }
  // rows r0-1 .. r0+FR of columns c-1 .. c+2: own rows' pair from registers, the rest from the plane
  float wl[FR + 2], w0[FR + 2], w1[FR + 2], wr[FR + 2];
  {
    const float2 t = *reinterpret_cast<const float2*>(xc + xi2(r0 - 1, c));
    const float2 u = *reinterpret_cast<const float2*>(xc + xi2(r0 + FR, c));
    w0[0] = t.x;
    w1[0] = t.y;
    w0[FR + 1] = u.x;
    w1[FR + 1] = u.y;
  }
#pragma unroll
  for (int q = 0; q < FR + 2; ++q) {
    wl[q] = xc[xi2(r0 - 1 + q, c - 1)];
    wr[q] = xc[xi2(r0 - 1 + q, c + 2)];
  }
#pragma unroll
  for (int k = 0; k < FR; ++k) {
    w0[k + 1] = xv[k][0];
    w1[k + 1] = xv[k][1];
  }
  float l0[FR + 2], l1[FR + 2];
#pragma unroll
  for (int q = 0; q < FR + 2; ++q) {
    l0[q] = fmaf(-2.0f, w0[q], wl[q] + w1[q]);
    l1[q] = fmaf(-2.0f, w1[q], w0[q] + wr[q]);
  }
#pragma unroll
  for (int k = 0; k < FR; ++k) {
    if constexpr (LAST) {  // rows outside the output tile (the same for every lane of the warp)
      if (!rowok[k]) continue;
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const float* w = j ? w1 : w0;
      const float* l = j ? l1 : l0;
      const float x = w[k + 1];
      const float lyv = fmaf(-2.0f, x, w[k] + w[k + 2]);
      const float lxly = fmaf(-2.0f, l[k + 1], l[k] + l[k + 2]);
      const float rest = fmaf(-6.0f, l[k + 1] + lyv, -lxly);
      const float res = p1_resid(bv[k][j], x, A.d_hi, A.d_lo, rest);
      const float corr = A.omega * res;
      if constexpr (LAST) {
        float h = sh[k][j], lo = sl[k][j];
        ff_add_scaled2_t(h, lo, x, corr, A.s_hi, A.s_lo);
        if ((j ? colok1 : colok0) && unk(k, j)) {
          shi[gp + k * nx + j] = h;
          slo[gp + k * nx + j] = lo;
        }
      } else {
        xv[k][j] = unk(k, j) ? x + corr : 0.0f;
      }
    }
  }
  if constexpr (!LAST) {
#pragma unroll
    for (int k = 0; k < FR; ++k) *reinterpret_cast<float2*>(xn + xi2(r0 + k, c)) = make_float2(xv[k][0], xv[k][1]);
  }
}

// Zero pads of both interior planes: rows -1 and RS, columns -2, -1, RS, RS+1.
__device__ __forceinline__ void zero_pads(float* xa, float* xb) {
  for (int t = threadIdx.x; t < 2 * XP2 + 4 * RS; t += NT) {
    int idx;
    if (t < XP2) {
      idx = t;
    } else if (t < 2 * XP2) {
      idx = (RS + 1) * XP2 + (t - XP2);
    } else {
      const int q = t - 2 * XP2, e = q & 3;
      idx = xi2(q >> 2, e < 2 ? e - 2 : RS + e - 2);
    }
    xa[idx] = 0.0f;
    xb[idx] = 0.0f;
  }
}

// Even ghosts of a Neumann axis in a region that reaches past that wall (2D fields have at most
// one Neumann axis): a ghost point (index -1 or n along the axis) takes the value its mirror (0 or
// n - 1) has in the plane just written, in the plane and in the owner's registers.
__device__ __forceinline__ void refill_ghosts(float* xp, float (&xv)[FR][2], int r0, int c, int gx, int gy, int nx,
                                              int ny, bool neu_x, bool neu_y) {
#pragma unroll
  for (int k = 0; k < FR; ++k)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int px = gx + j, py = gy + k;
      const int dx = neu_x ? (px == -1 ? 1 : (px == nx ? -1 : 0)) : 0;
      const int dy = neu_y ? (py == -1 ? 1 : (py == ny ? -1 : 0)) : 0;
      if (dx | dy) {
        const float v = xp[xi2(r0 + k + dy, c + j + dx)];
        xv[k][j] = v;
        xp[xi2(r0 + k, c + j)] = v;
      }
    }
}

// The whole solve of a region with origin (gx0, gy0) in the field (S >= 2).  MASK false: every
// point of the region is an unknown.  MASK true: the region touches a wall (see interior_sweep).
template <bool MASK>
__device__ __forceinline__ void solve_interior(const SolveArgs& A, const float* __restrict__ b, float* shi, float* slo,
                                               int nx, int ny, int bcx, int bcy, int gx0, int gy0) {
  extern __shared__ float sm[];
  float* xa = sm;
  float* xb = sm + XPL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = 2 * lane, r0 = FR * warp;
  const int gx = gx0 + c, gy = gy0 + r0;  // field coordinates of the thread's first point
  zero_pads(xa, xb);
  unsigned um = 0xffu;
  bool neu_x = false, neu_y = false;
  float bv[FR][2], xv[FR][2];
  if constexpr (MASK) {
    um = 0u;
#pragma unroll
    for (int k = 0; k < FR; ++k)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int px = gx + j, py = gy + k;
        if (px >= 0 && px < nx && py >= 0 && py < ny && interior(bcx, px, nx) && interior(bcy, py, ny))
          um |= 1u << (2 * k + j);
      }
    neu_x = bcx == NEU && (gx0 < 0 || gx0 + RS > nx);
    neu_y = bcy == NEU && (gy0 < 0 || gy0 + RS > ny);
#pragma unroll
    for (int k = 0; k < FR; ++k)
#pragma unroll
      for (int j = 0; j < 2; ++j)
        bv[k][j] = ((um >> (2 * k + j)) & 1u) ? b[(gy + k) * nx + gx + j] : 0.0f;
  } else {
    // 32-bit offsets from the region's first own point (planes hold fewer than 2^31 points)
    const float* bp = b + ((size_t)gy * nx + gx);
#pragma unroll
    for (int k = 0; k < FR; ++k) {
      bv[k][0] = bp[k * nx];
      bv[k][1] = bp[k * nx + 1];
    }
  }
#pragma unroll
  for (int k = 0; k < FR; ++k) {
    xv[k][0] = A.omega * bv[k][0];
    xv[k][1] = A.omega * bv[k][1];
    *reinterpret_cast<float2*>(xa + xi2(r0 + k, c)) = make_float2(xv[k][0], xv[k][1]);
  }
  __syncthreads();
  if (MASK && (neu_x || neu_y)) {
    refill_ghosts(xa, xv, r0, c, gx, gy, nx, ny, neu_x, neu_y);
    __syncthreads();
  }
  // the state from the region's first own point (MASK: from the field's origin, so offsets of
  // points off the field are never formed into addresses)
  float* const shb = MASK ? shi : shi + ((size_t)gy * nx + gx);
  float* const slb = MASK ? slo : slo + ((size_t)gy * nx + gx);
  const int gp = MASK ? gy * nx + gx : 0;
  const int H = A.S - 1;
  float* xc = xa;
  float* xn = xb;
  for (int k = 1; k < A.S - 1; ++k) {
    interior_sweep<false, MASK>(A, xc, xn, bv, xv, r0, c, shb, slb, gp, nx, H, um);
    __syncthreads();
    if (MASK && (neu_x || neu_y)) {
      refill_ghosts(xn, xv, r0, c, gx, gy, nx, ny, neu_x, neu_y);
      __syncthreads();
    }
    float* t = xc;
    xc = xn;
    xn = t;
  }
  interior_sweep<true, MASK>(A, xc, xn, bv, xv, r0, c, shb, slb, gp, nx, H, um);
}

// Region of RS x RS points = output tile (RS - 2H)^2 plus an H-cell halo, H = S - 1.  Warp w owns
// columns 32 (w & 1) .. +31 and row strip w >> 1 of every sweep, so no warp straddles strips.
__device__ __forceinline__ void solve_body(const SolveArgs& A, int f, int tbx, int tby) {
  extern __shared__ float sm[];
  float* bs = sm;
  float* xa = bs + RS * RSP;
  float* xb = xa + RS * RSP;
  const int nx = f ? A.nx[1] : A.nx[0], ny = f ? A.ny[1] : A.ny[0];
  const int bcx = f ? A.bcx[1] : A.bcx[0], bcy = f ? A.bcy[1] : A.bcy[0];
  float* const shi = f ? A.hi[1] : A.hi[0];
  float* const slo = f ? A.lo[1] : A.lo[0];
  const float* b = f ? A.b[1] : A.b[0];
  const int H = A.S - 1;
  const int TS = RS - 2 * H;
  const int tx0 = tbx * TS, ty0 = tby * TS;
  if (tx0 >= nx || ty0 >= ny) return;
  const int gx0 = tx0 - H, gy0 = ty0 - H;
  // interior tile: the region holds only unknowns, so no boundary tests and no ghosts
  const bool edge = !(gx0 >= 1 && gy0 >= 1 && gx0 + RS <= nx - 1 && gy0 + RS <= ny - 1);
  if (A.S >= 2) {
    if (edge) solve_interior<true>(A, b, shi, slo, nx, ny, bcx, bcy, gx0, gy0);
    else solve_interior<false>(A, b, shi, slo, nx, ny, bcx, bcy, gx0, gy0);
    return;
  }
  const bool neu_x = edge && bcx == NEU, neu_y = edge && bcy == NEU;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // b and the first iterate x1 = omega b (0 off the unknowns)
#pragma unroll
  for (int ly = warp; ly < RS; ly += NW) {
    const int gy = gy0 + ly;
    const bool row_ok = !edge || (gy >= 0 && gy < ny && interior(bcy, gy, ny));
    const float* brow = b + (size_t)(row_ok ? gy : 0) * nx;
#pragma unroll
    for (int cc = 0; cc < RS / 32; ++cc) {
      const int lx = lane + 32 * cc;
      const int gx = gx0 + lx;
      float v = 0.0f;
      if (row_ok && (!edge || (gx >= 0 && gx < nx && interior(bcx, gx, nx)))) v = brow[gx];
      bs[ly * RSP + lx] = v;
      xa[ly * RSP + lx] = A.omega * v;
    }
  }
  __syncthreads();
  if (neu_x || neu_y) {
    fill_ghosts(xa, gx0, gy0, nx, ny, neu_x, neu_y);
    __syncthreads();
  }
  if (edge) solve_sweeps<true>(A, bs, xa, xb, gx0, gy0, nx, ny, bcx, bcy, shi, slo, neu_x, neu_y);
  else solve_sweeps<false>(A, bs, xa, xb, gx0, gy0, nx, ny, bcx, bcy, shi, slo, false, false);
  if (A.S == 1) {  // the first iterate is also the last: x = 0, correction omega b
    for (int ly = warp; ly < RS; ly += NW) {
      const int gy = ty0 + ly;
#pragma unroll
      for (int cc = 0; cc < RS / 32; ++cc) {
        const int lx = lane + 32 * cc;
        const int gx2 = tx0 + lx;
        if (gx2 < nx && gy < ny && interior(bcx, gx2, nx) && interior(bcy, gy, ny)) {
          const size_t gp = (size_t)gy * nx + gx2;
          float h = shi[gp], l = slo[gp];
          ff_add_scaled_t(h, l, xa[ly * RSP + lx], A.s_hi, A.s_lo);
          shi[gp] = h;
          slo[gp] = l;
        }
      }
    }
  }
}

// Block b of the launch -> (field, tile): the boundary-ring tiles of every field first (they take
// the masked edge path and run longest), then the interior tiles of each field row by row.
__global__ void __launch_bounds__(NT, 2) k_solve_tile(SolveArgs A) {
  pdl_trigger();
  pdl_wait();
  const int nt = gridDim.x, nf = gridDim.z;
  const int b = blockIdx.x + nt * (blockIdx.y + nt * blockIdx.z);
  const int ring = nt > 1 ? 4 * (nt - 1) : 1;
  int f, k;
  if (b < nf * ring) {
    f = b / ring;
    k = b - f * ring;
  } else {
    const int c = b - nf * ring, ni = nt * nt - ring;  // ni > 0 here
    f = c / ni;
    k = ring + (c - f * ni);
  }
  int tx, ty;
  ring_first_tile(k, nt, &tx, &ty);
  solve_body(A, f, tx, ty);
}



// Batched form: item w solves tile work[3w+2] of field slot work[3w+1] of cavity work[3w]; blocks
// stride over the items as in k_curl_batch.
__global__ void __launch_bounds__(NT, 2) k_solve_batch(const SolveArgs* __restrict__ args, const int* __restrict__ work,
                                                       int nwork) {
  __shared__ SolveArgs sA;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int cav = work[3 * w], f = work[3 * w + 1], t = work[3 * w + 2];
    copy_args(&sA, args + cav);
    const int nt = sA.ntiles;
    solve_body(sA, f, t % nt, t / nt);
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side

static int g_curl_resident = 0, g_solve_resident = 0;  // resident blocks per batch kernel (tiled_configure)

static PhaseArgs phase(const ms_grid* g, int src, int axis, int kind, float cb_hi, float cb_lo) {
  const Shape& s = g->sh[src];
  const PadeTable& t = g->pade32[kind];
  PhaseArgs p;
  p.hi = g->hi[src];
  p.lo = g->lo[src];
  p.snx = s.nx;
  p.axis = axis;
  p.M = t.M;
  p.ghost_even = (axis == 0 ? s.bcx : s.bcy) == DIR;
  p.n_across = axis == 0 ? s.ny : s.nx;
  p.whi = t.d_whi;
  p.wlo = t.d_wlo;
  p.Kt = t.K;
  p.Bt = t.B;
  p.all_explicit = t.all_explicit;
  p.cb_hi = cb_hi;
  p.cb_lo = cb_lo;
  return p;
}

static CurlArgs make_curl(const ms_grid* g, int step, float cb_hi, float cb_lo, float* b0, float* b1) {
  CurlArgs A;
  A.N = g->N;
  A.b0 = b0;
  A.b1 = b1;
  // every output off the walls has both indices <= N - 1, so tiles cover 0 .. N-1 only; the
  // right-hand-side planes are zeroed at set-up and their wall entries are never written
  A.ntiles = (g->N + TB - 1) / TB;
  if (step == 0) {
    A.ph[0] = phase(g, HY, 0, HALF_TO_NODE, cb_hi, cb_lo);
    A.ph[1] = phase(g, HX, 1, HALF_TO_NODE, cb_hi, cb_lo);
  } else {
    A.ph[0] = phase(g, EZ, 1, NODE_TO_HALF, cb_hi, cb_lo);
    A.ph[1] = phase(g, EZ, 0, NODE_TO_HALF, cb_hi, cb_lo);
  }
  return A;
}

static SolveArgs make_solve(const ms_grid* g, int nfields, const int* fields, const float* const* b, int S, float d_hi,
                            float d_lo, float omega, float s_hi, float s_lo) {
  SolveArgs A;
  for (int k = 0; k < 2; ++k) {
    const int f = fields[k < nfields ? k : 0];
    const Shape& s = g->sh[f];
    A.b[k] = b[k < nfields ? k : 0];
    A.hi[k] = g->hi[f];
    A.lo[k] = g->lo[f];
    A.nx[k] = s.nx;
    A.ny[k] = s.ny;
    A.bcx[k] = s.bcx;
    A.bcy[k] = s.bcy;
  }
  A.S = S;
  A.d_hi = d_hi;
  A.d_lo = d_lo;
  A.omega = omega;
  A.s_hi = s_hi;
  A.s_lo = s_lo;
  const int TS = RS - 2 * (S - 1);
  A.ntiles = (g->N + 1 + TS - 1) / TS;
  return A;
}

size_t tiled_curl_smem() { return sizeof(float) * (size_t)(XROWS * XLP + TB * DLP + TB * YSP); }
size_t tiled_solve_smem() {
  static_assert(2 * XPL <= 3 * RS * RSP, "interior planes fit in the edge path's shared memory");
  return sizeof(float) * (size_t)(3 * RS * RSP);
}

int tiled_configure() {
  const int cs = (int)tiled_curl_smem(), ss = (int)tiled_solve_smem();
  if (cudaFuncSetAttribute(k_curl_tile<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs) != cudaSuccess ||
      cudaFuncSetAttribute(k_curl_tile<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs) != cudaSuccess ||
      cudaFuncSetAttribute(k_curl_tile<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs) != cudaSuccess ||
      cudaFuncSetAttribute(k_curl_batch<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs) != cudaSuccess ||
      cudaFuncSetAttribute(k_curl_batch<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs) != cudaSuccess ||
      cudaFuncSetAttribute(k_solve_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, ss) != cudaSuccess ||
      cudaFuncSetAttribute(k_solve_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, ss) != cudaSuccess)
    return -1;
  // blocks of the batch kernels resident on the device at once (persistent launches)
  int dev = 0, sms = 0, pc = 0, ps = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pc, k_curl_batch<0>, NT, cs) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_solve_batch, NT, ss) != cudaSuccess)
    return -1;
  g_curl_resident = sms * pc;
  g_solve_resident = sms * ps;
  // interior recurrences of A^{-1}: rho rounded to FP32, and the scale (1 - rho_f)^2 that makes
  // their DC gain exactly 1 with that rho_f, split hi + lo
  const float rho_f = (float)(-11.0L + std::sqrt(120.0L));
  const long double one_m = 1.0L - (long double)rho_f;
  const long double scale = one_m * one_m;
  float rec[4];
  rec[0] = rho_f;
  rec[1] = (float)(1.0L / one_m);
  rec[2] = (float)scale;
  rec[3] = (float)(scale - (long double)rec[2]);
  if (cudaMemcpyToSymbol(c_rec, rec, sizeof rec) != cudaSuccess)
    return -1;
  return 0;
}

// Launch with programmatic stream serialisation (the kernels above wait for their predecessors
// themselves); errors surface through cudaGetLastError as for <<<>>> launches.
template <typename Kern, typename Arg>
static void launch_pdl(Kern kernel, dim3 grid, size_t smem, cudaStream_t st, const Arg& arg) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, arg);
}

void tiled_curl(ms_grid* g, int step, float cb_hi, float cb_lo, float* b0, float* b1) {
  const CurlArgs A = make_curl(g, step, cb_hi, cb_lo, b0, b1);
  dim3 grid(A.ntiles, A.ntiles);
  if (step == 0) launch_pdl(k_curl_tile<0>, grid, tiled_curl_smem(), g->stream, A);
  else launch_pdl(k_curl_tile<1>, grid, tiled_curl_smem(), g->stream, A);
}

void tiled_curl_unfiltered(ms_grid* g, const float* hi, const float* lo, float* b0, float* b1) {
  CurlArgs A = make_curl(g, 1, 1.0f, 0.0f, b0, b1);
  for (int k = 0; k < 2; ++k) {
    A.ph[k].hi = hi;
    A.ph[k].lo = lo;
  }
  dim3 grid(A.ntiles, A.ntiles);
  launch_pdl(k_curl_tile<1, false>, grid, tiled_curl_smem(), g->stream, A);
}

void tiled_solve(ms_grid* g, int nfields, const int* fields, const float* const* b, int S, float d_hi, float d_lo,
                 float omega, float s_hi, float s_lo) {
  const SolveArgs A = make_solve(g, nfields, fields, b, S, d_hi, d_lo, omega, s_hi, s_lo);
  dim3 grid(A.ntiles, A.ntiles, nfields);
  launch_pdl(k_solve_tile, grid, tiled_solve_smem(), g->stream, A);
}

// ---------------------------------------------------------------------------------------
// Batched launches: one work list of (cavity, tile) entries covers every cavity.

int tiled_batch_build(ms_grid* const* cav, int count, int order, TiledBatch* tb, std::string* err) {
  std::vector<CurlArgs> curl(2 * (size_t)count);
  std::vector<SolveArgs> solve(2 * (size_t)count);
  // cavities in list order, or largest first (order 2)
  std::vector<int> seq(count);
  for (int c = 0; c < count; ++c) seq[c] = c;
  if (order == 2)
    std::stable_sort(seq.begin(), seq.end(), [&](int a, int b) { return cav[a]->N > cav[b]->N; });
  for (int c = 0; c < count; ++c) {
    ms_grid* g = cav[c];
    const MixedConsts k = mixed_consts(g);
    float* bE = g->s32[4];
    float* bx = g->s32[2];
    float* by = g->s32[3];
    curl[c] = make_curl(g, 0, k.cb_hi, k.cb_lo, bE, nullptr);
    curl[count + c] = make_curl(g, 1, k.cb_hi, k.cb_lo, bx, by);
    const int fe[1] = {EZ};
    const float* be[1] = {bE};
    const int fh[2] = {HX, HY};
    const float* bh[2] = {bx, by};
    solve[c] = make_solve(g, 1, fe, be, k.S, k.d_hi, k.d_lo, k.omega, k.sE_hi, k.sE_lo);
    solve[count + c] = make_solve(g, 2, fh, bh, k.S, k.d_hi, k.d_lo, k.omega, k.sH_hi, k.sH_lo);
  }
  // work lists; order 1 puts the tiles of every cavity's boundary ring (the general, slower paths)
  // ahead of all interior tiles
  std::vector<int> wc, we, wh;
  for (int pass = 0; pass < (order == 1 ? 2 : 1); ++pass)
    for (int c : seq) {
      const int ntc = curl[c].ntiles, nts = solve[c].ntiles;
      auto take = [&](int t, int nt) {
        if (order != 1) return true;
        const int tx = t % nt, ty = t / nt;
        const bool ring = tx == 0 || ty == 0 || tx == nt - 1 || ty == nt - 1;
        return ring == (pass == 0);
      };
      for (int t = 0; t < ntc * ntc; ++t) {
        if (!take(t, ntc)) continue;
        wc.push_back(c);
        wc.push_back(t);
      }
      for (int t = 0; t < nts * nts; ++t) {
        if (!take(t, nts)) continue;
        we.insert(we.end(), {c, 0, t});
        wh.insert(wh.end(), {c, 0, t});
        wh.insert(wh.end(), {c, 1, t});
      }
    }
  tb->n_curl = (int)(wc.size() / 2);
  tb->n_solveE = (int)(we.size() / 3);
  tb->n_solveH = (int)(wh.size() / 3);
  tb->off_curl = 0;
  tb->off_solveE = wc.size();
  tb->off_solveH = wc.size() + we.size();
  std::vector<int> work(wc);
  work.insert(work.end(), we.begin(), we.end());
  work.insert(work.end(), wh.begin(), wh.end());
  if (dev_malloc(&tb->d_curl, curl.size() * sizeof(CurlArgs)) != cudaSuccess ||
      dev_malloc(&tb->d_solve, solve.size() * sizeof(SolveArgs)) != cudaSuccess ||
      dev_malloc(&tb->d_work, work.size() * sizeof(int)) != cudaSuccess) {
    *err = "cudaMalloc of the batch work lists failed";
    return -1;
  }
  if (cudaMemcpy(tb->d_curl, curl.data(), curl.size() * sizeof(CurlArgs), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(tb->d_solve, solve.data(), solve.size() * sizeof(SolveArgs), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(tb->d_work, work.data(), work.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
    *err = "copy of the batch work lists failed";
    return -1;
  }
  tb->count = count;
  return 0;
}

void tiled_batch_step(const TiledBatch& tb, cudaStream_t st, int persistent) {
  const size_t cs = tiled_curl_smem(), ss = tiled_solve_smem();
  auto blocks = [&](int n, int resident) { return (persistent && resident > 0 && resident < n) ? resident : n; };
  k_curl_batch<0><<<blocks(tb.n_curl, g_curl_resident), NT, cs, st>>>(tb.d_curl, tb.d_work + tb.off_curl, tb.n_curl);
  k_solve_batch<<<blocks(tb.n_solveE, g_solve_resident), NT, ss, st>>>(tb.d_solve, tb.d_work + tb.off_solveE,
                                                                      tb.n_solveE);
  k_curl_batch<1><<<blocks(tb.n_curl, g_curl_resident), NT, cs, st>>>(tb.d_curl + tb.count, tb.d_work + tb.off_curl,
                                                                     tb.n_curl);
  k_solve_batch<<<blocks(tb.n_solveH, g_solve_resident), NT, ss, st>>>(tb.d_solve + tb.count,
                                                                      tb.d_work + tb.off_solveH, tb.n_solveH);
}

void tiled_batch_free(TiledBatch* tb) {
  dev_free(tb->d_curl);
  dev_free(tb->d_solve);
  dev_free(tb->d_work);
  *tb = TiledBatch{};
}

}  // namespace ms
