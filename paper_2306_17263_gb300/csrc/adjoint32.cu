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
  float* y[2] = {};   // Y^T u before the filter (FP32)
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

__global__ void k_bandT32(BandT p) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int l = p.line_lo + blockIdx.y * blockDim.y + threadIdx.y;
  if (m > p.M || l >= p.line_hi) return;
  const size_t vo = (size_t)m * p.va + (size_t)l * p.vc;
  if (m == p.M) {
    p.vh[vo] = 0.0f;
    p.vl[vo] = 0.0f;
    return;
  }
  float sh = 0.0f, sl = 0.0f;
  const int r0 = max(0, m - p.K - 1), r1 = min(p.M - 1, m + p.K);
  for (int r = r0; r <= r1; ++r) {
    const int t = m - r + p.K;  // tap of input m in row r
    const float* wh = pade_row_ptr(p.whi, r, p.M, p.K, p.B, p.all_explicit);
    const float* wl = pade_row_ptr(p.wlo, r, p.M, p.K, p.B, p.all_explicit);
    const size_t uo = (size_t)(r + p.uoff) * p.ua + (size_t)l * p.uc_;
    const float a = p.ux[uo], c = p.uc[uo], w = wh[t];
    const float prod = __fmul_rn(w, a);
    float e = fmaf(w, a, -prod);
    e = fmaf(w, c, e);
    e = fmaf(wl[t], a, e);
    const float s = __fadd_rn(sh, prod);
    const float bb = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(prod, bb));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
  }
  const float h2 = __fadd_rn(sh, sl);
  p.vh[vo] = h2;
  p.vl[vo] = __fsub_rn(sl, __fsub_rn(h2, sh));
}

// y = sx (v^x_{i-1} - v^x_i) + sy (v^y_{j-1} - v^y_j) at the unknowns of a field (v_{-1} = 0),
// differences of float-float values; 0 elsewhere.  sx, sy in {-1, 0, 1}.
__global__ void k_combineT32(const float* __restrict__ vxh, const float* __restrict__ vxl, const float* __restrict__ vyh,
                             const float* __restrict__ vyl, float* __restrict__ y, int nx, int ny, int bcx, int bcy,
                             float sx, float sy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const size_t p = (size_t)j * nx + i;
  if (!interior(bcx, i, nx) || !interior(bcy, j, ny)) {
    y[p] = 0.0f;
    return;
  }
  float v = 0.0f;
  if (sx != 0.0f) {
    const float h0 = i > 0 ? vxh[p - 1] : 0.0f, l0 = i > 0 ? vxl[p - 1] : 0.0f;
    v = sx * (__fsub_rn(h0, vxh[p]) + __fsub_rn(l0, vxl[p]));
  }
  if (sy != 0.0f) {
    const float h0 = j > 0 ? vyh[p - nx] : 0.0f, l0 = j > 0 ? vyl[p - nx] : 0.0f;
    v = fmaf(sy, __fsub_rn(h0, vyh[p]) + __fsub_rn(l0, vyl[p]), v);
  }
  y[p] = v;
}

// (l_hi, l_lo) += (s_hi + s_lo) (12 beta y + L y) at the unknowns (L the 5-point h^2 Delta_h with
// Dirichlet zeros and even Neumann ghosts), with error-free transformations.
__global__ void k_filter_accT32(const float* __restrict__ y, float* __restrict__ lh, float* __restrict__ ll, int nx,
                                int ny, int bcx, int bcy, float cb_hi, float cb_lo, float s_hi, float s_lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  if (!interior(bcx, i, nx) || !interior(bcy, j, ny)) return;
  const size_t p = (size_t)j * nx + i;
  const int im = clampi(i - 1, nx), ip = clampi(i + 1, nx), jm = clampi(j - 1, ny), jp = clampi(j + 1, ny);
  const float c = y[p];
  const float lap = fmaf(-4.0f, c, (y[(size_t)j * nx + im] + y[(size_t)j * nx + ip]) +
                                       (y[(size_t)jm * nx + i] + y[(size_t)jp * nx + i]));
  const float f = fmaf(cb_hi, c, fmaf(cb_lo, c, lap));
  float h = lh[p], l = ll[p];
  const float prod = __fmul_rn(s_hi, f);
  float e = fmaf(s_hi, f, -prod);
  e = fmaf(s_lo, f, e);
  const float s = __fadd_rn(h, prod);
  const float bb = __fsub_rn(s, h);
  const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(prod, bb));
  const float l2 = __fadd_rn(l, __fadd_rn(err, e));
  const float h2 = __fadd_rn(s, l2);
  ll[p] = __fsub_rn(l2, __fsub_rn(h2, s));
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
  const dim3 blk(64, 4, 1);
  const dim3 grd((t.M + 1 + blk.x - 1) / blk.x, (p.line_hi - p.line_lo + blk.y - 1) / blk.y);
  k_bandT32<<<grd, blk, 0, g->stream>>>(p);
}

void combineT32(ms_grid* g, int ft, int vx, float sx, int vy, float sy, int yslot) {
  Adj32* A = g->adj32;
  const Shape& s = g->sh[ft];
  k_combineT32<<<grid2(s.nx, s.ny), kBlk2, 0, g->stream>>>(
      vx >= 0 ? A->vh[vx] : nullptr, vx >= 0 ? A->vl[vx] : nullptr, vy >= 0 ? A->vh[vy] : nullptr,
      vy >= 0 ? A->vl[vy] : nullptr, A->y[yslot], s.nx, s.ny, s.bcx, s.bcy, sx, sy);
}

void filter_accT32(ms_grid* g, int f, int yslot, const MixedConsts& k, float s_hi, float s_lo) {
  Adj32* A = g->adj32;
  const Shape& s = g->sh[f];
  k_filter_accT32<<<grid2(s.nx, s.ny), kBlk2, 0, g->stream>>>(A->y[yslot], A->lh[f], A->ll[f], s.nx, s.ny, s.bcx,
                                                               s.bcy, k.cb_hi, k.cb_lo, s_hi, s_lo);
}

// One transposed step on the float-float adjoint state.
void adjoint_step32(ms_grid* g) {
  const MixedConsts k = mixed_consts(g);
  // S2^T: u_H = P~^{-1} l_H; y_E = Y_x^T u_Hy - Y_y^T u_Hx (node-to-half bands); l_E += sH F~ y_E
  solveT32(g, HX, 0, k);
  solveT32(g, HY, 1, k);
  bandT32(g, 1, NODE_TO_HALF, 0, HX, EZ, 0, 0);  // columns of H_x -> columns of E
  bandT32(g, 0, NODE_TO_HALF, 1, HY, EZ, 0, 1);  // rows of H_y -> rows of E
  combineT32(g, EZ, 1, 1.0f, 0, -1.0f, 0);
  filter_accT32(g, EZ, 0, k, k.sH_hi, k.sH_lo);
  // S1^T: u_E = P~^{-1} l_E; y_Hy = Y_x^T u_E, y_Hx = -Y_y^T u_E (half-to-node bands, output r at
  // node r + 1); l_H += sE F~ y_H
  solveT32(g, EZ, 0, k);
  bandT32(g, 0, HALF_TO_NODE, 0, EZ, HY, 1, 1);  // rows of E -> rows of H_y
  bandT32(g, 1, HALF_TO_NODE, 0, EZ, HX, 1, 0);  // columns of E -> columns of H_x
  combineT32(g, HY, 1, 1.0f, -1, 0.0f, 1);
  combineT32(g, HX, -1, 0.0f, 0, -1.0f, 0);
  filter_accT32(g, HY, 1, k, k.sE_hi, k.sE_lo);
  filter_accT32(g, HX, 0, k, k.sE_hi, k.sE_lo);
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
                      &A->uc[0], &A->uc[1], &A->vh[0], &A->vh[1], &A->vl[0], &A->vl[1], &A->y[0],  &A->y[1],
                      &A->sw[0], &A->sw[1]};
  for (float** p : planes) {
    if (cudaMalloc((void**)p, n * sizeof(float) + 256) != cudaSuccess) {
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
                  A->uc[1], A->vh[0], A->vh[1], A->vl[0], A->vl[1], A->y[0],  A->y[1],  A->sw[0], A->sw[1]};
  for (float* p : all) cudaFree(p);
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
