// Reverse (adjoint) pass of the FP32_REFINED step in FP32 arithmetic with a float-float adjoint
// state.
//
// The FP32_REFINED forward step, in the units of its tile kernels (k_tiled.cu, k_mixed.cu), is
//   S1: E   += sE P~_E^{-1} (Y_x F~ H_y - Y_y F~ H_x),
//   S2: H_x += sH P~_Hx^{-1} (-Y_y F~ E),   H_y += sH P~_Hy^{-1} (Y_x F~ E),
// with P~ = 6 h^2 P1 (Def. "def:operatorsP"), F~ = 12 beta + L the filter of Eq. "eq:ell" on the
// source grid, Y = W D the Pade derivative of App. A.1 as a band W of A^{-1} applied to the first
// differences D of a line, sE = 12 Z / r, sH = 12 / (r Z).  F~ and P~ are symmetric on the unknowns
// (Dirichlet zeros, even Neumann ghosts), so the transposed step M^T = S1^T S2^T is
//   S2^T: l_E  += sH F~_E (-Y_y^T P~^{-1} l_Hx + Y_x^T P~^{-1} l_Hy),
//   S1^T: l_Hy += sE F~_Hy Y_x^T P~_E^{-1} l_E,   l_Hx += -sE F~_Hx Y_y^T P~_E^{-1} l_E,
// with Y^T = D^T W^T: (Y^T u)_j = v_{j-1} - v_j, v = W^T u, v_{-1} = v_M = 0.
//
// Precision.  D^T takes the difference of two nearly equal values of a smooth v, which would
// amplify an FP32 rounding of v by 1 / (pi k h).  So every quantity before that difference is
// carried with more than FP32 accuracy: the adjoint state l is a float-float pair; the solve
// u = P~^{-1} l iterates in FP32 against a residual with l's low part and an exact two-product of
// the diagonal term, and returns the last iterate x and its correction c as a pair (u = x + c to
// about 31 bits, far below the correction's own size); v = W^T u is accumulated in float-float
// (exact two-products of the hi parts, the lo parts of W and u folded into the error term); only
// the difference of v is rounded to FP32.  The filter and the sH / sE scaling act on that
// difference, a well-conditioned FP32 value, and the result is added to l with error-free
// transformations.  The step is the exact transpose of the FP32_REFINED forward operator (same
// truncated band tables) up to this rounding.
#include <string>

#include "k_fp64.cuh"
#include "k_mixed.cuh"
#include "k_tiled.cuh"

namespace ms {

struct Adj32 {
  float* lh[3] = {};  // adjoint state (l_E, l_Hx, l_Hy), hi parts
  float* ll[3] = {};  // lo parts
  float* ux[2] = {};  // solve results: last iterate ...
  float* uc[2] = {};  // ... and its correction
  float* vh[2] = {};  // W^T u, float-float, in the target field's layout
  float* vl[2] = {};
  float* sw[2] = {};  // sweep iterates
  Graph g1, gk;
};

namespace {

const dim3 kBlk2(32, 8, 1);

ms_status a32fail(ms_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

void free_graph32(Graph* gr) {
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  if (gr->graph) cudaGraphDestroy(gr->graph);
  *gr = Graph{};
}

dim3 grid2(int nx, int ny) { return dim3((nx + kBlk2.x - 1) / kBlk2.x, (ny + kBlk2.y - 1) / kBlk2.y); }

// Richardson sweep on 6 h^2 P1 x = b with b = (b_hi, b_lo) (see the tile solve): FIRST reads the
// first iterate as omega b_hi; LAST writes the iterate and its correction separately.
template <bool FIRST, bool LAST>
__global__ void k_sweepT32(const float* __restrict__ bh, const float* __restrict__ bl, const float* __restrict__ xin,
                           float* __restrict__ xout, float* __restrict__ cout, int nx, int ny, int bcx, int bcy,
                           float d_hi, float d_lo, float omega) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const size_t p = (size_t)j * nx + i;
  if (!interior(bcx, i, nx) || !interior(bcy, j, ny)) {
    xout[p] = 0.0f;
    if (LAST) cout[p] = 0.0f;
    return;
  }
  const int im = clampi(i - 1, nx), ip = clampi(i + 1, nx), jm = clampi(j - 1, ny), jp = clampi(j + 1, ny);
  // iterate on the 3 x 3 neighbourhood (Dirichlet neighbours are stored zeros, Neumann ones clamp)
  auto X = [&](int jj, int ii) {
    const size_t q = (size_t)jj * nx + ii;
    return FIRST ? omega * bh[q] : xin[q];
  };
  const float x = X(j, i);
  const float lx = fmaf(-2.0f, x, X(j, im) + X(j, ip));
  const float ly = fmaf(-2.0f, x, X(jm, i) + X(jp, i));
  const float lxm = fmaf(-2.0f, X(jm, i), X(jm, im) + X(jm, ip));
  const float lxp = fmaf(-2.0f, X(jp, i), X(jp, im) + X(jp, ip));
  const float lxly = fmaf(-2.0f, lx, lxm + lxp);
  const float rest = fmaf(-6.0f, lx + ly, -lxly);
  const float ph = __fmul_rn(d_hi, x);
  const float pl = fmaf(d_lo, x, fmaf(d_hi, x, -ph));
  const float res = __fsub_rn(__fsub_rn(__fadd_rn(__fsub_rn(bh[p], ph), bl[p]), pl), rest);
  const float corr = omega * res;
  if (LAST) {
    xout[p] = x;
    cout[p] = corr;
  } else {
    xout[p] = x + corr;
  }
}

// v = W^T u along lines of one axis, in float-float.  Line l (lines [line_lo, line_hi)) holds the
// M outputs r of the forward band at u[(r + uoff) * ustride_along + l * ustride_across]; v_m
// (m = 0..M-1) and v_M = 0 go to v[m * vstride_along + l * vstride_across].
struct BandT {
  const float* ux;
  const float* uc;
  float* vh;
  float* vl;
  int ua, uc_, uoff;  // u strides along / across the line, offset of output 0 along the line
  int va, vc;         // v strides along / across
  int line_lo, line_hi;
  const float* whi;
  const float* wlo;
  int M, K, B, all_explicit;
};

// One term of the float-float sum: (sh, sl) += (w + wl)(a + c), exact product of the hi parts.
__device__ __forceinline__ void ff_fma_acc(float& sh, float& sl, float w, float wl, float a, float c) {
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

// Tiles of the transposed band: AXIS 0 (lines are rows): 8 lines x 128 outputs per block, a warp
// per line and four outputs per lane 32 apart; AXIS 1 (lines are columns): 32 lines x 32 outputs,
// lanes across the lines.  The inputs a tile reads (its outputs widened by the band's reach, zero
// past the line) are staged once in shared memory with coalesced loads; outputs whose window lies
// in the interior rows of the table read the one interior row.
constexpr int BT_THREADS = 256;
constexpr int BT_KMAX = kTiledKMax;
template <int AXIS>
struct BandTile {
  static constexpr int LINES = AXIS == 0 ? 8 : 32;
  static constexpr int OUTS = AXIS == 0 ? 128 : 32;
  static constexpr int WIN = OUTS + 2 * BT_KMAX + 2;  // staged inputs per line
};

template <int AXIS>
__global__ void __launch_bounds__(BT_THREADS) k_bandT32(BandT p) {
  using T = BandTile<AXIS>;
  __shared__ float sx[T::LINES][T::WIN + 1];
  __shared__ float sc[T::LINES][T::WIN + 1];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.x * T::OUTS;               // first output of the tile
  const int l0 = p.line_lo + blockIdx.y * T::LINES;  // first line of the tile
  const int base = m0 - p.K - 1;                     // input index of slot 0
  const int win = T::OUTS + 2 * p.K + 2;
  // stage u on [base, base + win) of every line of the tile
  if (AXIS == 0) {
    for (int e = tid; e < T::LINES * win; e += BT_THREADS) {
      const int ll = e / win, q = e - ll * win, r = base + q, l = l0 + ll;
      float a = 0.0f, c = 0.0f;
      if (r >= 0 && r < p.M && l < p.line_hi) {
        const size_t uo = (size_t)(r + p.uoff) * p.ua + (size_t)l * p.uc_;
        a = p.ux[uo];
        c = p.uc[uo];
      }
      sx[ll][q] = a;
      sc[ll][q] = c;
    }
  } else {
    for (int e = tid; e < T::LINES * win; e += BT_THREADS) {
      const int q = e / T::LINES, ll = e - q * T::LINES, r = base + q, l = l0 + ll;
      float a = 0.0f, c = 0.0f;
      if (r >= 0 && r < p.M && l < p.line_hi) {
        const size_t uo = (size_t)(r + p.uoff) * p.ua + (size_t)l * p.uc_;
        a = p.ux[uo];
        c = p.uc[uo];
      }
      sx[ll][q] = a;
      sc[ll][q] = c;
    }
  }
  // the interior row of the table (taps d = m - r = -K .. K+1 at index d + K)
  __shared__ float wh_s[2 * BT_KMAX + 2], wl_s[2 * BT_KMAX + 2];
  const int rs = 2 * p.K + 2;
  if (!p.all_explicit && tid < rs) {
    wh_s[tid] = p.whi[(size_t)(2 * p.B) * rs + tid];
    wl_s[tid] = p.wlo[(size_t)(2 * p.B) * rs + tid];
  }
  __syncthreads();
  constexpr int PER = T::OUTS * T::LINES / BT_THREADS;  // outputs per thread
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    int ll, mo;
    if (AXIS == 0) {
      ll = tid >> 5;
      mo = (tid & 31) + 32 * k;
    } else {
      ll = tid & 31;
      mo = (tid >> 5) + 8 * k;
    }
    const int m = m0 + mo, l = l0 + ll;
    if (m > p.M || l >= p.line_hi) continue;
    const size_t vo = (size_t)m * p.va + (size_t)l * p.vc;
    if (m == p.M) {
      p.vh[vo] = 0.0f;
      p.vl[vo] = 0.0f;
      continue;
    }
    float sh = 0.0f, sl = 0.0f;
    const int r0 = max(0, m - p.K - 1), r1 = min(p.M - 1, m + p.K);
    if (!p.all_explicit && r0 >= p.B && r1 < p.M - p.B) {
      // interior row: taps |m - r| >= 3 are below 1.2e-4 of the centre tap (|rho|^3), so their sum
      // (below 2e-4 of |v|) is accumulated in plain FP32 (error ~1e-11 |v|, including the dropped
      // lo parts); the five central taps go through the float-float sum
      const float* ax = &sx[ll][m - base];  // ax[-d] = u_{m-d}
      const float* ac = &sc[ll][m - base];
      float small = 0.0f;
#pragma unroll
      for (int d = BT_KMAX + 1; d >= -BT_KMAX; --d) {  // farthest taps first
        if (d >= -2 && d <= 2) continue;
        if (d > p.K + 1 || d < -p.K) continue;
        small = fmaf(wh_s[d + p.K], ax[-d], small);
      }
#pragma unroll
      for (int d = 2; d >= -2; --d) ff_fma_acc(sh, sl, wh_s[d + p.K], wl_s[d + p.K], ax[-d], ac[-d]);
      sl = __fadd_rn(sl, small);
    } else {
      for (int r = r0; r <= r1; ++r) {
        const int t = m - r + p.K;  // tap of input m in row r
        const float* wh = pade_row_ptr(p.whi, r, p.M, p.K, p.B, p.all_explicit);
        const float* wl = pade_row_ptr(p.wlo, r, p.M, p.K, p.B, p.all_explicit);
        ff_fma_acc(sh, sl, wh[t], wl[t], sx[ll][r - base], sc[ll][r - base]);
      }
    }
    const float h2 = __fadd_rn(sh, sl);
    p.vh[vo] = h2;
    p.vl[vo] = __fsub_rn(sl, __fsub_rn(h2, sh));
  }
}

// l (hi, lo) += (s_hi + s_lo)(12 beta y + L y) at the unknowns of a field, with
//   y = sx (v^x_{i-1} - v^x_i) + sy (v^y_{j-1} - v^y_j)  (v_{-1} = 0; sx, sy in {-1, 0, 1}),
// the differences taken of float-float values; L the 5-point h^2 Delta_h with Dirichlet zeros and
// even Neumann ghosts.  A 32 x 8 tile of y with a one-point halo is formed in shared memory (0 off
// the unknowns), then filtered and added to l with error-free transformations.
constexpr int FT_X = 32, FT_Y = 8;
__global__ void __launch_bounds__(FT_X * FT_Y) k_combine_filterT32(const float* __restrict__ vxh, const float* __restrict__ vxl,
                                                                   const float* __restrict__ vyh, const float* __restrict__ vyl,
                                                                   float* __restrict__ lh, float* __restrict__ ll, int nx,
                                                                   int ny, int bcx, int bcy, float sx, float sy, float cb_hi,
                                                                   float cb_lo, float s_hi, float s_lo) {
  __shared__ float ys[FT_Y + 2][FT_X + 2];
  const int i0 = blockIdx.x * FT_X - 1, j0 = blockIdx.y * FT_Y - 1;
  for (int e = threadIdx.y * FT_X + threadIdx.x; e < (FT_X + 2) * (FT_Y + 2); e += FT_X * FT_Y) {
    const int a = e / (FT_X + 2), b = e - a * (FT_X + 2);
    // ghost positions take the clamped point (even ghosts of a Neumann axis; a Dirichlet axis has
    // its stored zero wall there, whose y is 0 below)
    const int i = clampi(i0 + b, nx), j = clampi(j0 + a, ny);
    float v = 0.0f;
    if (interior(bcx, i, nx) && interior(bcy, j, ny)) {
      const size_t p = (size_t)j * nx + i;
      if (sx != 0.0f) {
        const float h0 = i > 0 ? vxh[p - 1] : 0.0f, l0 = i > 0 ? vxl[p - 1] : 0.0f;
        v = sx * (__fsub_rn(h0, vxh[p]) + __fsub_rn(l0, vxl[p]));
      }
      if (sy != 0.0f) {
        const float h0 = j > 0 ? vyh[p - nx] : 0.0f, l0 = j > 0 ? vyl[p - nx] : 0.0f;
        v = fmaf(sy, __fsub_rn(h0, vyh[p]) + __fsub_rn(l0, vyl[p]), v);
      }
    }
    ys[a][b] = v;
  }
  __syncthreads();
  const int i = blockIdx.x * FT_X + threadIdx.x, j = blockIdx.y * FT_Y + threadIdx.y;
  if (i >= nx || j >= ny || !interior(bcx, i, nx) || !interior(bcy, j, ny)) return;
  const int a = threadIdx.y + 1, b = threadIdx.x + 1;
  const float c = ys[a][b];
  const float lap = fmaf(-4.0f, c, (ys[a][b - 1] + ys[a][b + 1]) + (ys[a - 1][b] + ys[a + 1][b]));
  const float f = fmaf(cb_hi, c, fmaf(cb_lo, c, lap));
  const size_t p = (size_t)j * nx + i;
  float h = lh[p], l = ll[p];
  const float prod = __fmul_rn(s_hi, f);
  float e = fmaf(s_hi, f, -prod);
  e = fmaf(s_lo, f, e);
  const float s2 = __fadd_rn(h, prod);
  const float bb = __fsub_rn(s2, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s2, bb)), __fsub_rn(prod, bb));
  const float l2 = __fadd_rn(l, __fadd_rn(err, e));
  const float h2 = __fadd_rn(s2, l2);
  ll[p] = __fsub_rn(l2, __fsub_rn(h2, s2));
  lh[p] = h2;
}

// u = P~^{-1} l for field f: pair (ux[slot], uc[slot]).
void solveT32(ms_grid* g, int f, int slot, const MixedConsts& k) {
  Adj32* A = g->adj32;
  const Shape& s = g->sh[f];
  const dim3 grd = grid2(s.nx, s.ny);
  const float* bh = A->lh[f];
  const float* bl = A->ll[f];
  // sweeps k = 1 .. S-1 (x_1 = omega b is read inside the first); the last writes the pair
  const int L = k.S - 1;
  const float* xin = nullptr;
  for (int q = 0; q < L; ++q) {
    const bool first = q == 0, last = q == L - 1;
    float* xo = last ? A->ux[slot] : A->sw[q & 1];
    float* co = A->uc[slot];
    if (first && last)
      k_sweepT32<true, true><<<grd, kBlk2, 0, g->stream>>>(bh, bl, xin, xo, co, s.nx, s.ny, s.bcx, s.bcy, k.d_hi, k.d_lo,
                                                          k.omega);
    else if (first)
      k_sweepT32<true, false><<<grd, kBlk2, 0, g->stream>>>(bh, bl, xin, xo, co, s.nx, s.ny, s.bcx, s.bcy, k.d_hi,
                                                           k.d_lo, k.omega);
    else if (last)
      k_sweepT32<false, true><<<grd, kBlk2, 0, g->stream>>>(bh, bl, xin, xo, co, s.nx, s.ny, s.bcx, s.bcy, k.d_hi,
                                                           k.d_lo, k.omega);
    else
      k_sweepT32<false, false><<<grd, kBlk2, 0, g->stream>>>(bh, bl, xin, xo, co, s.nx, s.ny, s.bcx, s.bcy, k.d_hi,
                                                            k.d_lo, k.omega);
    xin = xo;
  }
}

// v = W^T u (one transposed band) into pair slot vs.  axis 0: lines are rows (along x), axis 1:
// columns.  u: pair slot us of field fu; the target field ft gives v's layout; uoff: offset of the
// band's output 0 in u along the line; lines [1, n - 1) of the target.
void bandT32(ms_grid* g, int axis, int kind, int us, int fu, int ft, int uoff, int vs) {
  Adj32* A = g->adj32;
  const PadeTable& t = g->pade32[kind];
  const Shape& su = g->sh[fu];
  const Shape& st = g->sh[ft];
  BandT p;
  p.ux = A->ux[us];
  p.uc = A->uc[us];
  p.vh = A->vh[vs];
  p.vl = A->vl[vs];
  p.uoff = uoff;
  if (axis == 0) {
    p.ua = 1;
    p.uc_ = su.nx;
    p.va = 1;
    p.vc = st.nx;
    p.line_lo = 1;
    p.line_hi = st.ny - 1;
  } else {
    p.ua = su.nx;
    p.uc_ = 1;
    p.va = st.nx;
    p.vc = 1;
    p.line_lo = 1;
    p.line_hi = st.nx - 1;
  }
  p.whi = t.d_whi;
  p.wlo = t.d_wlo;
  p.M = t.M;
  p.K = t.K;
  p.B = t.B;
  p.all_explicit = t.all_explicit;
  const int nl = p.line_hi - p.line_lo;
  if (axis == 0) {
    using T = BandTile<0>;
    k_bandT32<0><<<dim3((t.M + 1 + T::OUTS - 1) / T::OUTS, (nl + T::LINES - 1) / T::LINES), BT_THREADS, 0,
                   g->stream>>>(p);
  } else {
    using T = BandTile<1>;
    k_bandT32<1><<<dim3((t.M + 1 + T::OUTS - 1) / T::OUTS, (nl + T::LINES - 1) / T::LINES), BT_THREADS, 0,
                   g->stream>>>(p);
  }
}

// l_f += s F~ (sx Y^T along x + sy Y^T along y) from the v pairs vx, vy (slots, -1: none).
void combine_filterT32(ms_grid* g, int f, int vx, float sx, int vy, float sy, const MixedConsts& k, float s_hi,
                       float s_lo) {
  Adj32* A = g->adj32;
  const Shape& s = g->sh[f];
  const dim3 blk(FT_X, FT_Y, 1), grd((s.nx + FT_X - 1) / FT_X, (s.ny + FT_Y - 1) / FT_Y);
  k_combine_filterT32<<<grd, blk, 0, g->stream>>>(
      vx >= 0 ? A->vh[vx] : nullptr, vx >= 0 ? A->vl[vx] : nullptr, vy >= 0 ? A->vh[vy] : nullptr,
      vy >= 0 ? A->vl[vy] : nullptr, A->lh[f], A->ll[f], s.nx, s.ny, s.bcx, s.bcy, sx, sy, k.cb_hi, k.cb_lo, s_hi,
      s_lo);
}

// One transposed step on the float-float adjoint state.
void adjoint_step32(ms_grid* g) {
  const MixedConsts k = mixed_consts(g);
  // S2^T: u_H = P~^{-1} l_H; y_E = Y_x^T u_Hy - Y_y^T u_Hx (node-to-half bands); l_E += sH F~ y_E
  solveT32(g, HX, 0, k);
  solveT32(g, HY, 1, k);
  bandT32(g, 1, NODE_TO_HALF, 0, HX, EZ, 0, 0);  // columns of H_x -> columns of E
  bandT32(g, 0, NODE_TO_HALF, 1, HY, EZ, 0, 1);  // rows of H_y -> rows of E
  combine_filterT32(g, EZ, 1, 1.0f, 0, -1.0f, k, k.sH_hi, k.sH_lo);
  // S1^T: u_E = P~^{-1} l_E; y_Hy = Y_x^T u_E, y_Hx = -Y_y^T u_E (half-to-node bands, output r at
  // node r + 1); l_H += sE F~ y_H
  solveT32(g, EZ, 0, k);
  bandT32(g, 0, HALF_TO_NODE, 0, EZ, HY, 1, 1);  // rows of E -> rows of H_y
  bandT32(g, 1, HALF_TO_NODE, 0, EZ, HX, 1, 0);  // columns of E -> columns of H_x
  combine_filterT32(g, HY, 1, 1.0f, -1, 0.0f, k, k.sE_hi, k.sE_lo);
  combine_filterT32(g, HX, -1, 0.0f, 0, -1.0f, k, k.sE_hi, k.sE_lo);
}

ms_status capture32(ms_grid* g, Graph* gr, int steps) {
  if (gr->exec) return MS_OK;
  if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return a32fail(MS_ECUDA, "cudaStreamBeginCapture failed");
  for (int q = 0; q < steps; ++q) adjoint_step32(g);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
  if (e != cudaSuccess) return a32fail(MS_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&gr->exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return a32fail(MS_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  gr->graph = graph;
  gr->steps = steps;
  return MS_OK;
}

}  // namespace

ms_status adjoint32_setup(ms_grid* g) {
  if (g->adj32) return MS_OK;
  Adj32* A = new Adj32();
  g->adj32 = A;
  const size_t n = (size_t)(g->N + 1) * (g->N + 1);
  float** planes[] = {&A->lh[0], &A->lh[1], &A->lh[2], &A->ll[0], &A->ll[1], &A->ll[2], &A->ux[0], &A->ux[1],
                      &A->uc[0], &A->uc[1], &A->vh[0], &A->vh[1], &A->vl[0], &A->vl[1], &A->sw[0], &A->sw[1]};
  for (float** p : planes) {
    if (dev_malloc((void**)p, n * sizeof(float) + 256) != cudaSuccess) {
      adjoint32_teardown(g);
      return a32fail(MS_ENOMEM, "cudaMalloc of the FP32 adjoint planes failed");
    }
    if (cudaMemsetAsync(*p, 0, n * sizeof(float) + 256, g->stream) != cudaSuccess) {
      adjoint32_teardown(g);
      return a32fail(MS_ECUDA, "clearing the FP32 adjoint planes failed");
    }
  }
  return MS_OK;
}

void adjoint32_teardown(ms_grid* g) {
  Adj32* A = g->adj32;
  if (!A) return;
  free_graph32(&A->g1);
  free_graph32(&A->gk);
  float* all[] = {A->lh[0], A->lh[1], A->lh[2], A->ll[0], A->ll[1], A->ll[2], A->ux[0], A->ux[1], A->uc[0],
                  A->uc[1], A->vh[0], A->vh[1], A->vl[0], A->vl[1], A->sw[0], A->sw[1]};
  for (float* p : all) dev_free(p);
  delete A;
  g->adj32 = nullptr;
}

// The adjoint state from / to FP64 arrays (device), three fields.
void adjoint32_load(ms_grid* g, const double* const* l) {
  for (int f = 0; f < 3; ++f) launch_split(l[f], g->adj32->lh[f], g->adj32->ll[f], g->sh[f].size(), g->stream);
}
void adjoint32_store(ms_grid* g, double* const* l) {
  for (int f = 0; f < 3; ++f) launch_join(g->adj32->lh[f], g->adj32->ll[f], l[f], g->sh[f].size(), g->stream);
}

// (M^T)^nsteps on the float-float adjoint state, replaying captured chunks of 16 steps.
ms_status adjoint32_steps(ms_grid* g, long nsteps) {
  Adj32* A = g->adj32;
  const int chunk = 16;
  if (nsteps >= chunk) {
    ms_status s = capture32(g, &A->gk, chunk);
    if (s != MS_OK) return s;
  }
  if (nsteps % chunk) {
    ms_status s = capture32(g, &A->g1, 1);
    if (s != MS_OK) return s;
  }
  long left = nsteps;
  for (; left >= chunk; left -= chunk)
    if (cudaGraphLaunch(A->gk.exec, g->stream) != cudaSuccess) return a32fail(MS_ECUDA, "cudaGraphLaunch failed");
  for (; left > 0; --left)
    if (cudaGraphLaunch(A->g1.exec, g->stream) != cudaSuccess) return a32fail(MS_ECUDA, "cudaGraphLaunch failed");
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return a32fail(MS_ECUDA, std::string("FP32 adjoint steps: ") + cudaGetErrorString(e));
  return MS_OK;
}

}  // namespace ms
