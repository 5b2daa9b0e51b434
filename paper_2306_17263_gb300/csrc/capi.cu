// C ABI of include/maxwell4.h: grid life cycle, the time step (Sec. 3.4 Step 1 / Step 2),
// graph-captured time loop, diagnostics and operator-level entry points.
#include <array>
#include <cctype>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "grid3d.cuh"
#include "k_fp64.cuh"
#include "k_mixed.cuh"
#include "k_src3.cuh"
#include "k_tiled.cuh"
#include "k_tracked32.cuh"

using namespace ms;

namespace {

thread_local std::string g_last_error;

ms_status fail(ms_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define MS_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(MS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define MS_TRY(expr)              \
  do {                            \
    ms_status s_ = (expr);        \
    if (s_ != MS_OK) return s_;   \
  } while (0)

ms_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return MS_OK;
}

template <typename T>
ms_status dalloc(T** p, size_t n) {
  cudaError_t e = dev_malloc((void**)p, n * sizeof(T) + 256);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(MS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  return MS_OK;
}

double omega_of(double c1h2) { return 2.0 / (2.0 * c1h2 + 16.0 / 3.0); }

// ---------------------------------------------------------------------------------------
// FP64 operator building blocks on arbitrary device arrays.

// R = kappa^2 Z (delta_x G_y - delta_y G_x) on E_z (Step 1, third row of curl_h).
void curl_he64(ms_grid* g, const double* Gx, const double* Gy, double* R, int* nl) {
  const int N = g->N;
  const double s = g->kappa2 * g->Z / g->h;
  // delta_x G_y: rows j = 1..N-1 of H_y (N half-node values) -> E_z columns 1..N-1
  launch_pade64(0, Gy, R, N + 1, N, N + 1, N + 1, 1, 1, N, g->pade[HALF_TO_NODE], s, 0, g->stream);
  prof_mark(g, KK_PADE64, 8.0 * ((double)(N - 1) * N + (double)(N + 1) * (N + 1)));
  // delta_y G_x: columns i = 1..N-1 of H_x (N half-node values) -> E_z rows 1..N-1
  launch_pade64(1, Gx, R, N + 1, N + 1, N + 1, N + 1, 1, 1, N, g->pade[HALF_TO_NODE], -s, 1, g->stream);
  prof_mark(g, KK_PADE64, 8.0 * ((double)(N - 1) * N + 2.0 * (N + 1) * (N + 1)));
  *nl += 2;
}

// (R_x, R_y) = (kappa^2/Z) (-delta_y G_E, delta_x G_E) (Step 2).
void curl_eh64(ms_grid* g, const double* GE, double* Rx, double* Ry, int* nl) {
  const int N = g->N;
  const double s = g->kappa2 / (g->Z * g->h);
  // delta_y G_E: columns i = 1..N-1 of E_z (N+1 node values) -> H_x rows 0..N-1
  launch_pade64(1, GE, Rx, N + 1, N + 1, N, N + 1, 0, 1, N, g->pade[NODE_TO_HALF], -s, 0, g->stream);
  prof_mark(g, KK_PADE64, 8.0 * ((double)(N - 1) * (N + 1) + (double)N * (N + 1)));
  // delta_x G_E: rows j = 1..N-1 of E_z -> H_y columns 0..N-1
  launch_pade64(0, GE, Ry, N + 1, N + 1, N, N, 0, 1, N, g->pade[NODE_TO_HALF], s, 0, g->stream);
  prof_mark(g, KK_PADE64, 8.0 * ((double)(N - 1) * (N + 1) + (double)N * (N + 1)));
  *nl += 2;
}

}  // namespace

namespace ms {
// x = P1^{-1} b by Richardson sweeps; the last sweep writes `out` and, if upd != nullptr,
// adds upd_scale * x to upd (the state update E += h_tau E*).
void p1_solve64(ms_grid* g, int f, const double* b, double* out, double* upd, double upd_scale, int* nl) {
  const Shape& s = g->sh[f];
  const double c1h2 = g->c1 * g->h * g->h, om = omega_of(c1h2), h2 = g->h * g->h;
  const int S = g->p1_sweeps;
  double* buf[2] = {g->s64[3], g->s64[4]};
  const double* xin = nullptr;
  for (int k = 0; k < S; ++k) {
    const bool last = (k == S - 1);
    double* xo = last ? out : buf[k & 1];
    launch_p1_sweep64(b, xin, xo, s, c1h2, om, h2, k == 0, last ? upd : nullptr, upd_scale, g->stream);
    prof_mark(g, KK_P1SWEEP64, 8.0 * (double)s.size() * ((k == 0 ? 2 : 3) + (last && upd ? 2 : 0)));
    xin = xo;
  }
  *nl += S;
}
}  // namespace ms

namespace {

// H* = P1^{-1} R_H(E) for a given E (Step 2 without the update) into hxs, hys.
void h_increment64(ms_grid* g, const double* ez, double* hxs, double* hys, double* hx_upd, double* hy_upd, int* nl,
                   bool with_sources = false) {
  double* GE = g->s64[0];
  double* Rx = g->s64[1];
  double* Ry = g->s64[2];
  launch_filter64(ez, GE, g->sh[EZ], g->beta, g->stream);
  prof_mark(g, KK_FILTER64, 16.0 * (double)g->sh[EZ].size());
  *nl += 1;
  if (with_sources && g->src_wall) {  // G_E on the boundary nodes from d_t J
    launch_wall_ge64(g, GE);
    prof_mark(g, KK_SRC, 8.0 * 4.0 * g->N);
    *nl += 1;
  }
  curl_eh64(g, GE, Rx, Ry, nl);
  if (with_sources && g->nsrc) {
    launch_src_h64(g, Rx, Ry);
    prof_mark(g, KK_SRC, 8.0 * 2.0 * (double)g->sh[HX].size());
    *nl += 1;
  }
  if (with_sources && g->src_wall) {  // the ghost part of P1 with the wall data of H*
    launch_wall_hsolve64(g, Rx, Ry);
    prof_mark(g, KK_SRC, 8.0 * 8.0 * g->N);
    *nl += 1;
  }
  p1_solve64(g, HX, Rx, hxs, hx_upd, g->ht, nl);
  p1_solve64(g, HY, Ry, hys, hy_upd, g->ht, nl);
}

// The step as printed in Sec. 3.4 (MS_SCHEME_C4_DE): Step 1 as in step64, then DE advanced by
// Eq. "eq:mhe" with the unfiltered Pade curl of H, and Step 2 with G_E = beta E + (h^2/12) DE.
ms_status step64_tracked(ms_grid* g) {
  int nl = 0;
  double *ez = g->f64[EZ], *hx = g->f64[HX], *hy = g->f64[HY];
  double* Gx = g->s64[0];
  double* Gy = g->s64[1];
  double* R = g->s64[2];
  launch_filter64(hx, Gx, g->sh[HX], g->beta, g->stream);
  prof_mark(g, KK_FILTER64, 16.0 * (double)g->sh[HX].size());
  launch_filter64(hy, Gy, g->sh[HY], g->beta, g->stream);
  prof_mark(g, KK_FILTER64, 16.0 * (double)g->sh[HY].size());
  nl += 2;
  curl_he64(g, Gx, Gy, R, &nl);
  p1_solve64(g, EZ, R, g->s64[5], ez, g->ht, &nl);  // E* in s64[5], E += h_tau E*
  curl_he64(g, hx, hy, g->s64[0], &nl);              // kappa^2 Z curl_h H (unfiltered)
  double* GE = g->s64[1];
  launch_de_update64(g->de64, g->s64[5], g->s64[0], ez, GE, g->N, g->ht, g->kappa2, g->beta, g->h, g->stream);
  prof_mark(g, KK_FILTER64, 8.0 * 6.0 * (double)g->sh[EZ].size());
  nl += 1;
  double* Rx = g->s64[0];
  double* Ry = g->s64[2];
  curl_eh64(g, GE, Rx, Ry, &nl);
  p1_solve64(g, HX, Rx, g->s64[5], hx, g->ht, &nl);
  p1_solve64(g, HY, Ry, g->s64[5], hy, g->ht, &nl);
  g->launches_per_step = nl;
  return check_launch("fp64 tracked step");
}

ms_status step64(ms_grid* g) {
  int nl = 0;
  double *ez = g->f64[EZ], *hx = g->f64[HX], *hy = g->f64[HY];
  if (g->desc.scheme == MS_SCHEME_YEE2) {
    const double ne = (double)g->sh[EZ].size(), nh = (double)g->sh[HX].size();
    launch_yee_e64(ez, hx, hy, g->N, g->desc.r * g->Z, g->stream);
    prof_mark(g, KK_YEE64, 8.0 * (2 * ne + 2 * nh));
    launch_yee_h64(ez, hx, hy, g->N, g->desc.r / g->Z, g->stream);
    prof_mark(g, KK_YEE64, 8.0 * (ne + 4 * nh));
    g->launches_per_step = 2;
    return check_launch("yee step");
  }
  if (g->desc.scheme == MS_SCHEME_NC4) {
    const double ne = (double)g->sh[EZ].size(), nh = (double)g->sh[HX].size();
    launch_nc_e64(ez, hx, hy, g->N, g->ht * g->Z, g->stream);
    prof_mark(g, KK_NC64, 8.0 * (2 * ne + 2 * nh));
    launch_nc_h64(ez, hx, hy, g->N, g->ht / g->Z, g->stream);
    prof_mark(g, KK_NC64, 8.0 * (ne + 4 * nh));
    g->launches_per_step = 2;
    return check_launch("nc step");
  }
  if (g->desc.scheme == MS_SCHEME_C4_DE) return step64_tracked(g);
  // Step 1: G = (beta + (h^2/12) Delta_h) H, R = kappa^2 Z curl_h G, P1 E* = R, E += h_tau E*
  double* Gx = g->s64[0];
  double* Gy = g->s64[1];
  double* R = g->s64[2];
  launch_filter64(hx, Gx, g->sh[HX], g->beta, g->stream);
  prof_mark(g, KK_FILTER64, 16.0 * (double)g->sh[HX].size());
  launch_filter64(hy, Gy, g->sh[HY], g->beta, g->stream);
  prof_mark(g, KK_FILTER64, 16.0 * (double)g->sh[HY].size());
  nl += 2;
  if (g->src_wall) {  // the inhomogeneous ghosts of H^{n+1/2} in the filter
    launch_wall_hfilter64(g, Gx, Gy);
    prof_mark(g, KK_SRC, 8.0 * 8.0 * g->N);
    nl += 1;
  }
  curl_he64(g, Gx, Gy, R, &nl);
  if (g->nsrc) {
    launch_src_time(g, 1.0, 1.0);
    prof_mark(g, KK_SRC, 0.0);
    launch_src_e64(g, R);
    prof_mark(g, KK_SRC, 16.0 * (double)g->sh[EZ].size());
    nl += 2;
  }
  // the solve's result lands in s64[5]; the last sweep also performs E += h_tau E*
  p1_solve64(g, EZ, R, g->s64[5], ez, g->ht, &nl);
  // Step 2 on E^{n+1}
  h_increment64(g, ez, g->s64[5], g->s64[5], hx, hy, &nl, true);
  if (g->nsrc) {
    launch_tick(g);
    prof_mark(g, KK_SRC, 0.0);
    nl += 1;
  }
  g->launches_per_step = nl;
  return check_launch("fp64 step");
}

ms_status step_any(ms_grid* g) {
  if (g->g3) return step3d(g);
  if (g->desc.precision == MS_FP64) return step64(g);
  int nl = 0;
  if (g->de_hi) {
    const ms_status s = step_mixed_tracked(g, &nl);
    if (s != MS_OK) return fail(s, "tracked Delta E step failed");
    g->launches_per_step = nl;
    return check_launch("tracked mixed step");
  }
  ms_status s = step_mixed(g, &nl);
  if (s != MS_OK) return fail(s, mixed_last_error());
  g->launches_per_step = nl;
  return check_launch("mixed step");
}

ms_status capture(ms_grid* g, Graph* gr, int steps) {
  if (gr->exec) return MS_OK;
  MS_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
  ms_status st = MS_OK;
  for (int k = 0; k < steps && st == MS_OK; ++k) st = step_any(g);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
  if (st != MS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(MS_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&gr->exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(MS_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  gr->graph = graph;
  gr->steps = steps;
  return MS_OK;
}

void free_graph(Graph* gr) {
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  if (gr->graph) cudaGraphDestroy(gr->graph);
  *gr = Graph{};
}

ms_status ensure_partial(ms_grid* g, size_t n) {
  int b = reduce_blocks(n);
  if (b <= g->partial_cap) return MS_OK;
  if (g->d_partial) dev_free(g->d_partial);
  MS_TRY(dalloc(&g->d_partial, (size_t)b * 4));
  g->partial_cap = b;
  return MS_OK;
}

// 1D tables of the separable cavity modes on the three grids (Eq. "eq:data").
// Per field: [tab_x (nm x nx)] [tab_y (nm x ny)] [coef (nm)].
ms_status exact_fields64(ms_grid* g, const ms_mode* modes, int nm, double tE, double tH, double* out[3],
                         const double* wover = nullptr) {
  const int N = g->N;
  const double pi = M_PI;
  std::vector<double> host;
  size_t offs[3][3];
  for (int f = 0; f < 3; ++f) {
    const Shape& s = g->sh[f];
    offs[f][0] = host.size();
    host.resize(host.size() + (size_t)nm * s.nx);
    offs[f][1] = host.size();
    host.resize(host.size() + (size_t)nm * s.ny);
    offs[f][2] = host.size();
    host.resize(host.size() + nm);
  }
  // sin(pi k i / N) and cos(pi k (2i+1) / (2N)) with exact integer argument reduction
  auto sin_node = [&](int k, int i) {
    if (i == 0 || i == N) return 0.0;
    long q = ((long)k * i) % (2L * N);
    return std::sin(pi * (double)q / N);
  };
  auto cos_half = [&](int k, int i) {
    long q = ((long)k * (2L * i + 1)) % (4L * N);
    return std::cos(pi * (double)q / (2.0 * N));
  };
  for (int m = 0; m < nm; ++m) {
    const int kx = modes[m].m, ky = modes[m].n;
    const double A = modes[m].amp, w = wover ? wover[m] : pi * std::sqrt((double)kx * kx + (double)ky * ky);
    // E_z
    for (int i = 0; i <= N; ++i) host[offs[EZ][0] + (size_t)m * (N + 1) + i] = sin_node(kx, i);
    for (int j = 0; j <= N; ++j) host[offs[EZ][1] + (size_t)m * (N + 1) + j] = sin_node(ky, j);
    host[offs[EZ][2] + m] = A * std::cos(w * tE);
    // H_x at (x_i, y_{j+1/2})
    for (int i = 0; i <= N; ++i) host[offs[HX][0] + (size_t)m * (N + 1) + i] = sin_node(kx, i);
    for (int j = 0; j < N; ++j) host[offs[HX][1] + (size_t)m * N + j] = cos_half(ky, j);
    host[offs[HX][2] + m] = -A * std::sin(w * tH) / (w * g->Z) * pi * ky;
    // H_y at (x_{i+1/2}, y_j)
    for (int i = 0; i < N; ++i) host[offs[HY][0] + (size_t)m * N + i] = cos_half(kx, i);
    for (int j = 0; j <= N; ++j) host[offs[HY][1] + (size_t)m * (N + 1) + j] = sin_node(ky, j);
    host[offs[HY][2] + m] = A * std::sin(w * tH) / (w * g->Z) * pi * kx;
  }
  if (host.size() > g->modetab_cap) {
    if (g->d_modetab) dev_free(g->d_modetab);
    g->d_modetab = nullptr;
    g->modetab_cap = 0;
    MS_TRY(dalloc(&g->d_modetab, host.size()));
    g->modetab_cap = host.size();
  }
  MS_CUDA(cudaMemcpyAsync(g->d_modetab, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  for (int f = 0; f < 3; ++f)
    launch_mode_field(out[f], g->sh[f], g->d_modetab + offs[f][0], g->d_modetab + offs[f][1],
                      g->d_modetab + offs[f][2], nm, g->stream);
  MS_TRY(check_launch("mode field"));
  MS_CUDA(cudaStreamSynchronize(g->stream));  // the host table is released on return
  return MS_OK;
}

// FP64 view of the state: the FP64 arrays themselves, or hi+lo joined into dst scratch.
ms_status state64(ms_grid* g, double* dst[3], const double* view[3]) {
  for (int f = 0; f < 3; ++f) {
    if (g->desc.precision == MS_FP64) {
      view[f] = g->f64[f];
    } else {
      launch_join(g->hi[f], g->lo[f], dst[f], g->sh[f].size(), g->stream);
      view[f] = dst[f];
    }
  }
  return check_launch("join");
}

ms_status store_state(ms_grid* g, const double* const* src) {
  for (int f = 0; f < 3; ++f) {
    const size_t n = g->sh[f].size();
    if (g->desc.precision == MS_FP64) {
      if (src[f] != g->f64[f])
        MS_CUDA(cudaMemcpyAsync(g->f64[f], src[f], n * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
      launch_zero_dirichlet64(g->f64[f], g->sh[f], g->stream);
    } else {
      // zero the Dirichlet entries in a scratch copy, then split
      double* tmp = g->s64[0];
      MS_CUDA(cudaMemcpyAsync(tmp, src[f], n * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
      launch_zero_dirichlet64(tmp, g->sh[f], g->stream);
      launch_split(tmp, g->hi[f], g->lo[f], n, g->stream);
    }
  }
  return check_launch("store state");
}

bool valid_grid(ms_grid* g) { return g != nullptr && g->N > 0; }

// The device copy of the step index read by the source kernels (sources only).
ms_status sync_step(ms_grid* g) {
  if (g->d_step) MS_CUDA(cudaMemcpyAsync(g->d_step, &g->step, sizeof(long), cudaMemcpyHostToDevice, g->stream));
  return MS_OK;
}

ms_status check_sources(ms_grid* g, const ms_source* src, int nsrc, bool need_off_resonance) {
  if (nsrc < 0 || nsrc > 64 || (nsrc > 0 && !src)) return fail(MS_EINVAL, "invalid sources (0 <= nsrc <= 64)");
  for (int q = 0; q < nsrc; ++q) {
    if (src[q].m < 1 || src[q].n < 1) return fail(MS_EINVAL, "source indices must be >= 1");
    if (!std::isfinite(src[q].amp) || !std::isfinite(src[q].omega)) return fail(MS_EINVAL, "non-finite source");
    const double w2 = M_PI * M_PI * ((double)src[q].m * src[q].m + (double)src[q].n * src[q].n);
    if (need_off_resonance && std::fabs(src[q].omega * src[q].omega - w2) <= 1e-12 * w2)
      return fail(MS_EINVAL, "the driven solution needs omega^2 != pi^2 (m^2 + n^2)");
    if (need_off_resonance && src[q].omega == 0.0) return fail(MS_EINVAL, "the driven solution needs omega != 0");
  }
  (void)g;
  return MS_OK;
}

// The driven solution as a mode superposition with its own frequencies (ms_init_driven).
void driven_modes(ms_grid* g, const ms_source* src, int nsrc, std::vector<ms_mode>* modes, std::vector<double>* w) {
  modes->resize(nsrc);
  w->resize(nsrc);
  for (int q = 0; q < nsrc; ++q) {
    const double om = src[q].omega;
    const double w2 = M_PI * M_PI * ((double)src[q].m * src[q].m + (double)src[q].n * src[q].n);
    (*modes)[q] = ms_mode{src[q].m, src[q].n, g->Z * src[q].amp * om / (om * om - w2)};
    (*w)[q] = om;
  }
}

}  // namespace

namespace ms {

void set_last_error(const char* msg) { g_last_error = msg; }

void prof_mark(ms_grid* g, int kind, double bytes) {
  Prof& p = g->prof;
  if (!p.on) return;
  if (p.next >= p.pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    p.pool.push_back(e);
  }
  cudaEventRecord(p.pool[p.next++], g->stream);
  p.kinds.push_back(kind);
  p.bytes.push_back(bytes);
}

const char* kernel_kind_name(int k) {
  static const char* names[KK_COUNT] = {"filter64", "pade64", "p1sweep64", "yee64", "curl32", "solve32",
                                        "filter3d64", "pade3d64", "sweep3d64", "filt3d32", "band3d32",
                                        "sweep3d32", "nc64", "source", "term3d32", "tsgemm", "tspack", "tracked32"};
  return (k >= 0 && k < KK_COUNT) ? names[k] : "";
}

}  // namespace ms

namespace {
std::atomic<int> g_fail_alloc{0};    // the allocation that fails, counted from 1; 0: none armed
std::atomic<long> g_live_allocs{0};  // device allocations held by the library
}  // namespace

namespace ms {

cudaError_t dev_malloc(void** p, size_t bytes) {
  int n = g_fail_alloc.load();
  while (n > 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
  }
  if (n == 1) {  // the armed allocation: fail as an out-of-memory device would, allocating nothing
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_live_allocs.fetch_add(1);
  else *p = nullptr;
  return e;
}

void dev_free(void* p) {
  if (!p) return;
  if (cudaFree(p) == cudaSuccess) g_live_allocs.fetch_sub(1);
}

}  // namespace ms

// =======================================================================================
extern "C" {

const char* ms_last_error(void) { return g_last_error.c_str(); }

ms_status ms_debug_fail_alloc(int n) {
  if (n < 0) return fail(MS_EINVAL, "n must be >= 0");
  g_fail_alloc.store(n);
  return MS_OK;
}

long ms_debug_live_allocs(void) { return g_live_allocs.load(); }

ms_status ms_stability_limit(int dim, double* rmax) {
  if (!rmax) return fail(MS_EINVAL, "rmax is NULL");
  if (dim != 2 && dim != 3) return fail(MS_EINVAL, "dim must be 2 or 3");
  *rmax = dim == 2 ? stability_limit_2d() : stability_limit_3d();
  return MS_OK;
}

// Largest Richardson sweep count the solve kernels of a precision hold.
static int max_sweeps(int dim, int precision) {
  if (precision == MS_FP64) return 64;
  return dim == 2 ? kTiledMaxSweeps : kMaxSweeps3d32;
}

ms_status ms_solver_sweeps(int dim, double r, int precision, double tol, int* sweeps) {
  if (!sweeps) return fail(MS_EINVAL, "sweeps is NULL");
  *sweeps = 0;
  if (dim != 2 && dim != 3) return fail(MS_EINVAL, "dim must be 2 or 3");
  if (precision != MS_FP64 && precision != MS_FP32_REFINED) return fail(MS_EINVAL, "unknown precision");
  if (!(r > 0.0) || !std::isfinite(r)) return fail(MS_EINVAL, "r must be positive");
  if (!(tol > 0.0 && tol < 1.0)) return fail(MS_EINVAL, "tol must be in (0, 1)");
  const double rmax = dim == 2 ? stability_limit_2d() : stability_limit_3d();
  if (r >= rmax) return fail(MS_ECFL, "r is at or above the stability limit");
  // Richardson on h^2 P1, spectrum in [c1 h^2, c1 h^2 + 16/3] (App. A.2) in 2D and 3D, from x = 0:
  // contraction (16/3) / (2 c1 h^2 + 16/3) per sweep; h^2 c1 = (24 / r^2)(1 + 2 / r^2) for any h
  const double c1h2 = (24.0 / (r * r)) * (1.0 + 2.0 / (r * r));
  const double rho = (16.0 / 3.0) / (2.0 * c1h2 + 16.0 / 3.0);
  const double s = std::ceil(std::log(tol) / std::log(rho));
  const int cap = max_sweeps(dim, precision);
  if (!(s <= cap)) {
    char buf[200];
    snprintf(buf, sizeof buf,
             "reaching tol = %.3g needs %.0f Richardson sweeps; the %s solve holds at most %d", tol, s,
             precision == MS_FP64 ? "FP64" : "FP32_REFINED", cap);
    return fail(MS_ENOTCONV, buf);
  }
  *sweeps = s < 1 ? 1 : (int)s;
  return MS_OK;
}

// shared64 != nullptr: the grid uses these six FP64 diagnostic planes (at least (n+1)^2 each,
// owned by a batch) instead of allocating its own.
static ms_status create_grid_impl(const ms_grid_desc* d, double* const* shared64, ms_grid** out);

ms_status ms_create_grid(const ms_grid_desc* d, ms_grid** out) {
  g_last_error.clear();
  return create_grid_impl(d, nullptr, out);
}

static ms_status create_grid_impl(const ms_grid_desc* d, double* const* shared64, ms_grid** out) {
  if (!out) return fail(MS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d) return fail(MS_EINVAL, "desc is NULL");
  if (d->dim == 3 && !shared64) return create_grid3d(d, out);
  if (d->dim != 2) return fail(MS_EINVAL, "dim must be 2 or 3 (batches: 2)");
  if (d->n < 4 || d->n > 32768) return fail(MS_EINVAL, "n must be in [4, 32768]");
  if (!(d->z_imp > 0.0) || !std::isfinite(d->z_imp)) return fail(MS_EINVAL, "z_imp must be positive");
  if (!(d->r > 0.0) || !std::isfinite(d->r)) return fail(MS_EINVAL, "r must be positive");
  if (d->precision != MS_FP64 && d->precision != MS_FP32_REFINED) return fail(MS_EINVAL, "unknown precision");
  if (d->closure != MS_CLOSURE_PAPER && d->closure != MS_CLOSURE_REFLECT) return fail(MS_EINVAL, "unknown closure");
  if (d->scheme != MS_SCHEME_C4 && d->scheme != MS_SCHEME_YEE2 && d->scheme != MS_SCHEME_NC4 &&
      d->scheme != MS_SCHEME_C4_DE)
    return fail(MS_EINVAL, "unknown scheme");
  if ((d->scheme == MS_SCHEME_YEE2 || d->scheme == MS_SCHEME_NC4) && d->precision != MS_FP64)
    return fail(MS_EUNSUPPORTED, "the Yee and NC comparators run in FP64 only");
  if (d->scheme == MS_SCHEME_C4_DE && shared64)
    return fail(MS_EUNSUPPORTED, "batches run the compact scheme MS_SCHEME_C4");
  const bool compact = d->scheme == MS_SCHEME_C4 || d->scheme == MS_SCHEME_C4_DE;
  if (compact) {
    const double rmax = stability_limit_2d();
    if (d->r >= rmax) {
      char buf[160];
      snprintf(buf, sizeof buf, "r = %.6g is at or above the stability limit %.6g of the 2D scheme", d->r, rmax);
      return fail(MS_ECFL, buf);
    }
  } else if (d->scheme == MS_SCHEME_YEE2 && d->r * std::sqrt(2.0) >= 1.0) {
    return fail(MS_ECFL, "Yee scheme requires r < 1/sqrt(2)");
  } else if (d->scheme == MS_SCHEME_NC4 && d->r * std::sqrt(2.0) * (9.0 / 8.0 + 1.0 / 24.0) >= 1.0) {
    return fail(MS_ECFL, "NC scheme requires r < 1/(sqrt(2) (9/8 + 1/24))");
  }
  ms_grid* g = new ms_grid();
  g->desc = *d;
  g->N = d->n;
  g->Z = d->z_imp;
  g->h = 1.0 / d->n;
  g->ht = d->r * g->h;
  g->kappa2 = 24.0 / (g->ht * g->ht);
  g->beta = 1.0 + g->kappa2 * g->h * g->h / 12.0;
  g->c1 = g->kappa2 * g->beta;
  for (int f = 0; f < 3; ++f) g->sh[f] = field_shape(g->N, f);
  auto cleanup = [&](ms_status s) {
    ms_destroy(g);
    return s;
  };
  if (d->stream) {
    g->stream = (cudaStream_t)d->stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(fail(MS_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e)));
    g->own_stream = true;
  }
  // Pade tables (FP64 truncation 1e-18 of the row's absolute sum)
  std::string err;
  // (the Yee and NC comparators use no Pade tables)
  for (int kind = 0; kind < 2 && compact; ++kind) {
    const int M = (kind == HALF_TO_NODE) ? g->N - 1 : g->N;
    if (build_pade_table(M, d->closure, kind, 1e-18, &g->pade[kind], &err) != 0) return cleanup(fail(MS_EINVAL, err));
    PadeTable& t = g->pade[kind];
    std::vector<float> whi(t.w.size()), wlo(t.w.size());
    for (size_t k = 0; k < t.w.size(); ++k) {
      whi[k] = (float)t.w[k];
      wlo[k] = (float)(t.w[k] - (double)whi[k]);
    }
    ms_status s = dalloc(&t.d_w, t.w.size());
    if (s == MS_OK) s = dalloc(&t.d_whi, t.w.size());
    if (s == MS_OK) s = dalloc(&t.d_wlo, t.w.size());
    if (s != MS_OK) return cleanup(s);
    if (cudaMemcpy(t.d_w, t.w.data(), t.w.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t.d_whi, whi.data(), whi.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(t.d_wlo, wlo.data(), wlo.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup(fail(MS_ECUDA, "copy of Pade tables failed"));
  }
  if (compact) {
    ms_status sw = ms_solver_sweeps(2, d->r, MS_FP64, 1e-17, &g->p1_sweeps);
    if (sw != MS_OK) return cleanup(sw);
  }
  const size_t nmax = (size_t)(g->N + 1) * (g->N + 1);
  ms_status s = MS_OK;
  // FP64 scratch is used by the FP64 step and by the diagnostics of both precisions
  if (shared64) {
    for (int k = 0; k < 6; ++k) g->s64[k] = shared64[k];
    g->shared64 = true;
  } else {
    for (int k = 0; k < 6 && s == MS_OK; ++k) s = dalloc(&g->s64[k], nmax);
  }
  if (d->precision == MS_FP64) {
    for (int f = 0; f < 3 && s == MS_OK; ++f) s = dalloc(&g->f64[f], g->sh[f].size());
    if (s == MS_OK && d->scheme == MS_SCHEME_C4_DE) {
      s = dalloc(&g->de64, g->sh[EZ].size());
      if (s == MS_OK) cudaMemsetAsync(g->de64, 0, g->sh[EZ].size() * sizeof(double), g->stream);
    }
  } else {
    for (int f = 0; f < 3 && s == MS_OK; ++f) s = dalloc(&g->hi[f], g->sh[f].size());
    for (int f = 0; f < 3 && s == MS_OK; ++f) s = dalloc(&g->lo[f], g->sh[f].size());
    if (s == MS_OK) {
      s = mixed_setup(g);
      if (s != MS_OK) fail(s, mixed_last_error());
    }
    if (s == MS_OK && d->scheme == MS_SCHEME_C4_DE) {
      s = tracked32_setup(g);
      if (s != MS_OK) fail(s, "cudaMalloc of the tracked Delta E planes failed");
    }
  }
  if (s == MS_OK) s = dalloc(&g->d_result, 8);
  if (s == MS_OK) s = ensure_partial(g, nmax);
  if (s != MS_OK) return cleanup(s);
  for (int f = 0; f < 3; ++f) {
    if (g->f64[f]) cudaMemsetAsync(g->f64[f], 0, g->sh[f].size() * sizeof(double), g->stream);
    if (g->hi[f]) cudaMemsetAsync(g->hi[f], 0, g->sh[f].size() * sizeof(float), g->stream);
    if (g->lo[f]) cudaMemsetAsync(g->lo[f], 0, g->sh[f].size() * sizeof(float), g->stream);
  }
  for (int k = 0; k < 6 && !g->shared64; ++k)
    if (g->s64[k]) cudaMemsetAsync(g->s64[k], 0, nmax * sizeof(double), g->stream);
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e != cudaSuccess) return cleanup(fail(MS_ECUDA, std::string("create: ") + cudaGetErrorString(e)));
  *out = g;
  return MS_OK;
}

ms_status ms_destroy(ms_grid* g) {
  if (!g) return MS_OK;
  if (g->stream) cudaStreamSynchronize(g->stream);
  free_graph(&g->graph1);
  free_graph(&g->graphk);
  adjoint_teardown(g);
  destroy_grid3d(g);
  for (cudaEvent_t e : g->prof.pool) cudaEventDestroy(e);
  for (int k = 0; k < 2; ++k) {
    dev_free(g->pade[k].d_w);
    dev_free(g->pade[k].d_whi);
    dev_free(g->pade[k].d_wlo);
  }
  for (int f = 0; f < 3; ++f) {
    dev_free(g->f64[f]);
    dev_free(g->hi[f]);
    dev_free(g->lo[f]);
  }
  dev_free(g->de64);
  tracked32_teardown(g);
  dev_free(g->d_src);
  dev_free(g->d_srctab);
  dev_free(g->d_srctab32);
  dev_free(g->d_srcfac);
  dev_free(g->d_walldata);
  dev_free(g->d_wresp);
  dev_free(g->d_step);
  for (int k = 0; k < 6 && !g->shared64; ++k) dev_free(g->s64[k]);
  for (int k = 0; k < 8; ++k) dev_free(g->s32[k]);
  mixed_teardown(g);
  dev_free(g->d_partial);
  dev_free(g->d_result);
  dev_free(g->d_modetab);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
  return MS_OK;
}

ms_status ms_init_modes(ms_grid* g, const ms_mode* modes, int nmodes) {
  if (!valid_grid(g)) return fail(MS_EINVAL, "invalid grid");
  if (g->g3) return fail(MS_EINVAL, "3D grids take ms_init_modes3");
  if (nmodes < 0 || (nmodes > 0 && !modes)) return fail(MS_EINVAL, "invalid modes");
  for (int m = 0; m < nmodes; ++m)
    if (modes[m].m < 1 || modes[m].n < 1) return fail(MS_EINVAL, "mode indices must be >= 1");
  if (g->de64 || g->de_hi) {
    // Delta E of a mode is -pi^2 (m^2 + n^2) E: the exact E_z field of the rescaled amplitudes
    std::vector<ms_mode> lap(modes, modes + nmodes);
    for (ms_mode& m : lap) m.amp *= -M_PI * M_PI * ((double)m.m * m.m + (double)m.n * m.n);
    double* dd[3] = {g->de64 ? g->de64 : g->s64[2], g->s64[0], g->s64[1]};
    MS_TRY(exact_fields64(g, lap.data(), nmodes, 0.0, 0.5 * g->ht, dd));
    if (g->de_hi) tracked32_set_de(g, g->s64[2]);
  }
  double* dst[3] = {g->s64[3], g->s64[4], g->s64[5]};
  MS_TRY(exact_fields64(g, modes, nmodes, 0.0, 0.5 * g->ht, dst));
  MS_TRY(store_state(g, dst));
  g->step = 0;
  MS_TRY(sync_step(g));
  MS_CUDA(cudaStreamSynchronize(g->stream));
  return MS_OK;
}

ms_status ms_set_fields_device(ms_grid* g, const double* const* comps, long step) {
  if (!valid_grid(g) || !comps) return fail(MS_EINVAL, "invalid argument");
  if (g->g3) {
    MS_TRY(set_fields3d(g, comps, 0));
    g->step = step;
    return sync_step(g);
  }
  for (int f = 0; f < 3; ++f)
    if (!comps[f]) return fail(MS_EINVAL, "NULL component");
  MS_TRY(store_state(g, comps));
  if (g->de64) launch_lap_e64(g->f64[EZ], g->de64, g->N, g->h, g->stream);  // DE^0 = Delta_h E^0
  if (g->de_hi) {  // DE^0 = Delta_h E^0 of the stored (wall-zeroed) E
    launch_join(g->hi[EZ], g->lo[EZ], g->s64[1], g->sh[EZ].size(), g->stream);
    launch_lap_e64(g->s64[1], g->s64[0], g->N, g->h, g->stream);
    tracked32_set_de(g, g->s64[0]);
  }
  g->step = step;
  MS_TRY(sync_step(g));
  return check_launch("set fields");
}

ms_status ms_get_fields_device(ms_grid* g, double* const* comps) {
  if (!valid_grid(g) || !comps) return fail(MS_EINVAL, "invalid argument");
  if (g->g3) return get_fields3d(g, comps, 0);
  for (int f = 0; f < 3; ++f) {
    if (!comps[f]) return fail(MS_EINVAL, "NULL component");
    const size_t n = g->sh[f].size();
    if (g->desc.precision == MS_FP64)
      MS_CUDA(cudaMemcpyAsync(comps[f], g->f64[f], n * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    else
      launch_join(g->hi[f], g->lo[f], comps[f], n, g->stream);
  }
  return check_launch("get fields");
}

ms_status ms_set_fields(ms_grid* g, const double* const* comps, long step) {
  if (!valid_grid(g) || !comps) return fail(MS_EINVAL, "invalid argument");
  if (g->g3) {
    MS_TRY(set_fields3d(g, comps, 1));
    g->step = step;
    return sync_step(g);
  }
  double* dst[3] = {g->s64[3], g->s64[4], g->s64[5]};
  for (int f = 0; f < 3; ++f) {
    if (!comps[f]) return fail(MS_EINVAL, "NULL component");
    MS_CUDA(cudaMemcpyAsync(dst[f], comps[f], g->sh[f].size() * sizeof(double), cudaMemcpyHostToDevice, g->stream));
  }
  MS_TRY(store_state(g, dst));
  if (g->de64) launch_lap_e64(g->f64[EZ], g->de64, g->N, g->h, g->stream);  // DE^0 = Delta_h E^0
  if (g->de_hi) {  // DE^0 = Delta_h E^0 of the stored (wall-zeroed) E
    launch_join(g->hi[EZ], g->lo[EZ], g->s64[1], g->sh[EZ].size(), g->stream);
    launch_lap_e64(g->s64[1], g->s64[0], g->N, g->h, g->stream);
    tracked32_set_de(g, g->s64[0]);
  }
  g->step = step;
  MS_TRY(sync_step(g));
  return check_launch("set fields");
}

ms_status ms_get_fields(ms_grid* g, double* const* comps) {
  if (!valid_grid(g) || !comps) return fail(MS_EINVAL, "invalid argument");
  if (g->g3) return get_fields3d(g, comps, 1);
  double* tmp[3] = {g->s64[3], g->s64[4], g->s64[5]};
  const double* view[3];
  for (int f = 0; f < 3; ++f)
    if (!comps[f]) return fail(MS_EINVAL, "NULL component");
  MS_TRY(state64(g, tmp, view));
  for (int f = 0; f < 3; ++f)
    MS_CUDA(cudaMemcpyAsync(comps[f], view[f], g->sh[f].size() * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  MS_CUDA(cudaStreamSynchronize(g->stream));
  return MS_OK;
}

ms_status ms_step(ms_grid* g) {
  if (!valid_grid(g)) return fail(MS_EINVAL, "invalid grid");
  MS_TRY(step_any(g));
  g->step += 1;
  return MS_OK;
}

ms_status ms_run(ms_grid* g, long nsteps) {
  if (!valid_grid(g)) return fail(MS_EINVAL, "invalid grid");
  if (nsteps < 0) return fail(MS_EINVAL, "nsteps must be >= 0");
  const int chunk = 16;
  if (nsteps >= chunk) MS_TRY(capture(g, &g->graphk, chunk));
  if (nsteps % chunk) MS_TRY(capture(g, &g->graph1, 1));
  long left = nsteps;
  while (left >= chunk) {
    MS_CUDA(cudaGraphLaunch(g->graphk.exec, g->stream));
    left -= chunk;
  }
  while (left > 0) {
    MS_CUDA(cudaGraphLaunch(g->graph1.exec, g->stream));
    left -= 1;
  }
  g->step += nsteps;
  return MS_OK;
}

ms_status ms_sync(ms_grid* g) {
  if (!valid_grid(g)) return fail(MS_EINVAL, "invalid grid");
  MS_CUDA(cudaStreamSynchronize(g->stream));
  if (g->g3) return transform_status3d(g);
  return MS_OK;
}

ms_status ms_set_solver(ms_grid* g, int solver) {
  if (!valid_grid(g)) return fail(MS_EINVAL, "invalid grid");
  if (solver != MS_SOLVER_RICHARDSON && solver != MS_SOLVER_TRANSFORM_TC) return fail(MS_EINVAL, "unknown solver");
  if (solver == MS_SOLVER_TRANSFORM_TC && (!g->g3 || g->desc.precision != MS_FP32_REFINED))
    return fail(MS_EUNSUPPORTED, "the transform solver is implemented for 3D FP32_REFINED grids");
  if (!g->g3) return MS_OK;
  MS_CUDA(cudaStreamSynchronize(g->stream));
  MS_TRY(set_solver3d(g, solver));
  free_graph(&g->graph1);  // captured steps hold the previous solver's launches
  free_graph(&g->graphk);
  g->launches_per_step = 0;
  return MS_OK;
}

ms_status ms_transform_solve3(ms_grid* g, int comp, const float* b, float* x) {
  if (!valid_grid(g) || !b || !x) return fail(MS_EINVAL, "invalid argument");
  if (!g->g3 || g->desc.precision != MS_FP32_REFINED)
    return fail(MS_EUNSUPPORTED, "the transform solver is implemented for 3D FP32_REFINED grids");
  if (comp < 0 || comp > 5) return fail(MS_EINVAL, "comp must be in [0, 5]");
  return transform_solve3d(g, comp, b, x);
}

ms_status ms_get_step(ms_grid* g, long* step) {
  if (!valid_grid(g) || !step) return fail(MS_EINVAL, "invalid argument");
  *step = g->step;
  return MS_OK;
}

ms_status ms_step_profiled(ms_grid* g, int cap, float* launch_ms, int* kinds, double* bytes, int* count) {
  if (!valid_grid(g) || !count || cap < 0 || (cap > 0 && (!launch_ms || !kinds || !bytes)))
    return fail(MS_EINVAL, "invalid argument");
  Prof& p = g->prof;
  p.on = true;
  p.next = 0;
  p.kinds.clear();
  p.bytes.clear();
  prof_mark(g, -1);
  ms_status s = step_any(g);
  p.on = false;
  if (s != MS_OK) return s;
  g->step += 1;
  MS_CUDA(cudaStreamSynchronize(g->stream));
  const int n = (int)p.next - 1;
  for (int k = 0; k < n && k < cap; ++k) {
    float ms = 0.0f;
    MS_CUDA(cudaEventElapsedTime(&ms, p.pool[k], p.pool[k + 1]));
    launch_ms[k] = ms;
    kinds[k] = p.kinds[k + 1];
    bytes[k] = p.bytes[k + 1];
  }
  *count = n;
  return MS_OK;
}

const char* ms_kernel_kind_name(int kind) { return kernel_kind_name(kind); }

ms_status ms_launches_per_step(ms_grid* g, int* launches) {
  if (!valid_grid(g) || !launches) return fail(MS_EINVAL, "invalid argument");
  if (g->launches_per_step == 0) {
    // count by issuing one captured step into a throw-away graph
    Graph tmp;
    MS_TRY(capture(g, &tmp, 1));
    free_graph(&tmp);
  }
  *launches = g->launches_per_step;
  return MS_OK;
}

ms_status ms_energy(ms_grid* g, double* W) {
  if (!valid_grid(g) || !W) return fail(MS_EINVAL, "invalid argument");
  if (g->g3) return energy3d(g, W);
  if (g->desc.scheme != MS_SCHEME_C4) return fail(MS_EUNSUPPORTED, "energy is defined for the compact scheme");
  // FP64 view of the state in scratch slots that the H increment does not touch
  double* tmp[3] = {nullptr, nullptr, nullptr};
  std::vector<double*> extra;
  const double* view[3];
  if (g->desc.precision != MS_FP64) {
    for (int f = 0; f < 3; ++f) {
      double* p = nullptr;
      MS_TRY(dalloc(&p, g->sh[f].size()));
      tmp[f] = p;
      extra.push_back(p);
    }
  }
  auto release = [&](ms_status s) {
    cudaStreamSynchronize(g->stream);
    for (double* p : extra) dev_free(p);
    return s;
  };
  ms_status s = state64(g, tmp, view);
  if (s != MS_OK) return release(s);
  double* hxs = nullptr;
  double* hys = nullptr;
  s = dalloc(&hxs, g->sh[HX].size());
  if (s == MS_OK) extra.push_back(hxs);
  if (s == MS_OK) s = dalloc(&hys, g->sh[HY].size());
  if (s == MS_OK) extra.push_back(hys);
  if (s != MS_OK) return release(s);
  int nl = 0;
  h_increment64(g, view[EZ], hxs, hys, nullptr, nullptr, &nl);
  // W = h^2 [ Z^-1 E.E + Z (H.H - h_tau H*.H) ]
  const int bE = reduce_blocks(g->sh[EZ].size());
  launch_dot(view[EZ], view[EZ], g->sh[EZ].size(), g->d_partial, bE, g->d_result, 0, 0, g->stream);
  launch_dot(view[HX], view[HX], g->sh[HX].size(), g->d_partial, reduce_blocks(g->sh[HX].size()), g->d_result, 1, 0,
             g->stream);
  launch_dot(view[HY], view[HY], g->sh[HY].size(), g->d_partial, reduce_blocks(g->sh[HY].size()), g->d_result, 1, 1,
             g->stream);
  launch_dot(hxs, view[HX], g->sh[HX].size(), g->d_partial, reduce_blocks(g->sh[HX].size()), g->d_result, 2, 0,
             g->stream);
  launch_dot(hys, view[HY], g->sh[HY].size(), g->d_partial, reduce_blocks(g->sh[HY].size()), g->d_result, 2, 1,
             g->stream);
  s = check_launch("energy");
  if (s != MS_OK) return release(s);
  double r[3];
  if (cudaMemcpyAsync(r, g->d_result, sizeof r, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
      cudaStreamSynchronize(g->stream) != cudaSuccess)
    return release(fail(MS_ECUDA, "energy readback failed"));
  const double h2 = g->h * g->h;
  *W = h2 * (r[0] / g->Z + g->Z * (r[1] - g->ht * r[2]));
  return release(MS_OK);
}

ms_status ms_divergence(ms_grid* g, double* norm) {
  if (!valid_grid(g) || !norm) return fail(MS_EINVAL, "invalid argument");
  if (g->g3) return divergence3d(g, norm);
  if (g->desc.scheme != MS_SCHEME_C4 && g->desc.scheme != MS_SCHEME_C4_DE)
    return fail(MS_EUNSUPPORTED, "the Pade divergence is defined for the compact scheme");
  double* tmp[3] = {g->s64[3], g->s64[4], g->s64[5]};
  const double* view[3];
  MS_TRY(state64(g, tmp, view));
  const int N = g->N;
  double* div = g->s64[0];
  const PadeTable& t = g->pade[NODE_TO_HALF];
  // delta_x H_x: rows j = 0..N-1 of H_x (N+1 nodes) -> N cell centres
  launch_pade64(0, view[HX], div, N, N + 1, N, N, 0, 0, N, t, 1.0 / g->h, 0, g->stream);
  // delta_y H_y: columns i = 0..N-1 of H_y (N+1 nodes) -> N cell centres
  launch_pade64(1, view[HY], div, N, N, N, N, 0, 0, N, t, 1.0 / g->h, 1, g->stream);
  const size_t n = (size_t)N * N;
  launch_dot(div, div, n, g->d_partial, reduce_blocks(n), g->d_result, 0, 0, g->stream);
  MS_TRY(check_launch("divergence"));
  double r;
  MS_CUDA(cudaMemcpyAsync(&r, g->d_result, sizeof r, cudaMemcpyDeviceToHost, g->stream));
  MS_CUDA(cudaStreamSynchronize(g->stream));
  *norm = std::sqrt(g->h * g->h * r);
  return MS_OK;
}

ms_status ms_error_vs_exact(ms_grid* g, const ms_mode* modes, int nmodes, double* l2_abs, double* l2_rel,
                            double* max_abs, double* sum_abs) {
  if (!valid_grid(g)) return fail(MS_EINVAL, "invalid grid");
  if (g->g3) return fail(MS_EINVAL, "3D grids take ms_error_vs_exact3");
  if (nmodes < 0 || (nmodes > 0 && !modes)) return fail(MS_EINVAL, "invalid modes");
  for (int m = 0; m < nmodes; ++m)
    if (modes[m].m < 1 || modes[m].n < 1) return fail(MS_EINVAL, "mode indices must be >= 1");
  double* ex[3] = {g->s64[0], g->s64[1], g->s64[2]};
  MS_TRY(exact_fields64(g, modes, nmodes, g->step * g->ht, (g->step + 0.5) * g->ht, ex));
  double* tmp[3] = {g->s64[3], g->s64[4], g->s64[5]};
  const double* view[3];
  MS_TRY(state64(g, tmp, view));
  for (int f = 0; f < 3; ++f) {
    const size_t n = g->sh[f].size();
    launch_err_reduce(view[f], ex[f], n, g->d_partial, reduce_blocks(n), g->d_result, f > 0, g->stream);
  }
  MS_TRY(check_launch("error reduce"));
  double r[4];
  MS_CUDA(cudaMemcpyAsync(r, g->d_result, sizeof r, cudaMemcpyDeviceToHost, g->stream));
  MS_CUDA(cudaStreamSynchronize(g->stream));
  if (l2_abs) *l2_abs = std::sqrt(g->h * g->h * r[0]);
  if (l2_rel) *l2_rel = r[1] > 0 ? std::sqrt(r[0] / r[1]) : 0.0;
  if (max_abs) *max_abs = r[2];
  if (sum_abs) *sum_abs = r[3];
  return MS_OK;
}

// Replaces the grid's sources (validated by the caller).
static ms_status set_sources_spec(ms_grid* g, const SrcSpec* src, int nsrc) {
  MS_CUDA(cudaStreamSynchronize(g->stream));
  dev_free(g->d_src);
  dev_free(g->d_srctab);
  dev_free(g->d_srctab32);
  dev_free(g->d_srcfac);
  dev_free(g->d_walldata);
  dev_free(g->d_wresp);
  g->d_src = nullptr;
  g->d_srctab = nullptr;
  g->d_srctab32 = nullptr;
  g->d_srcfac = nullptr;
  g->d_walldata = nullptr;
  g->d_wresp = nullptr;
  g->nsrc = 0;
  g->src_wall = 0;
  free_graph(&g->graph1);  // the captured steps do not contain the source launches
  free_graph(&g->graphk);
  g->launches_per_step = 0;
  if (nsrc == 0) return MS_OK;
  std::vector<unsigned char> blob;
  std::vector<double> tabs;
  build_sources(g, src, nsrc, &blob, &tabs);
  MS_TRY(dalloc((unsigned char**)&g->d_src, blob.size()));
  MS_TRY(dalloc(&g->d_srctab, tabs.size()));
  MS_TRY(dalloc(&g->d_srctab32, tabs.size()));
  MS_TRY(dalloc((unsigned char**)&g->d_srcfac, src_factor_bytes()));
  if (!g->d_step) MS_TRY(dalloc(&g->d_step, 1));
  MS_CUDA(cudaMemcpy(g->d_src, blob.data(), blob.size(), cudaMemcpyHostToDevice));
  MS_CUDA(cudaMemcpy(g->d_srctab, tabs.data(), tabs.size() * sizeof(double), cudaMemcpyHostToDevice));
  std::vector<float> tabs32(tabs.begin(), tabs.end());
  MS_CUDA(cudaMemcpy(g->d_srctab32, tabs32.data(), tabs32.size() * sizeof(float), cudaMemcpyHostToDevice));
  MS_CUDA(cudaMemcpy(g->d_step, &g->step, sizeof(long), cudaMemcpyHostToDevice));
  int wall = 0;
  for (int q = 0; q < nsrc; ++q) wall |= (src[q].px | src[q].py);
  if (wall && g->desc.precision == MS_FP32_REFINED) {  // wall terms of the FP32 source kernels
    std::vector<float> wr;
    wall_responses(g->N, &wr);
    MS_TRY(dalloc(&g->d_walldata, wall_data_doubles(g->N)));
    MS_TRY(dalloc(&g->d_wresp, wr.size()));
    MS_CUDA(cudaMemcpy(g->d_wresp, wr.data(), wr.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  // the step reads these two only once every buffer above is in place: a failure above leaves
  // the grid without sources rather than with half of them
  g->nsrc = nsrc;
  g->src_wall = wall;
  return MS_OK;
}

ms_status ms_set_sources3(ms_grid* g, const ms_source3* src, int nsrc) {
  if (!valid_grid(g)) return fail(MS_EINVAL, "invalid grid");
  if (!g->g3) return fail(MS_EUNSUPPORTED, "ms_set_sources3 needs a 3D grid (2D grids: ms_set_sources)");
  MS_TRY(check_sources3(src, nsrc, false));
  MS_CUDA(cudaStreamSynchronize(g->stream));
  free_graph(&g->graph1);  // the captured steps do not contain the source launches
  free_graph(&g->graphk);
  g->launches_per_step = 0;
  if (nsrc > 0 && !g->d_step) MS_TRY(dalloc(&g->d_step, 1));
  MS_TRY(sync_step(g));
  return src3_set(g, src, nsrc);
}

ms_status ms_set_sources(ms_grid* g, const ms_source* src, int nsrc) {
  if (!valid_grid(g)) return fail(MS_EINVAL, "invalid grid");
  if (g->g3 || g->desc.scheme != MS_SCHEME_C4)
    return fail(MS_EUNSUPPORTED, "ms_set_sources takes 2D grids of the compact scheme (3D grids: ms_set_sources3)");
  MS_TRY(check_sources(g, src, nsrc, false));
  std::vector<SrcSpec> sp(nsrc);
  for (int q = 0; q < nsrc; ++q) sp[q] = SrcSpec{src[q].m, src[q].n, 0, 0, src[q].amp, src[q].omega};
  return set_sources_spec(g, sp.data(), nsrc);
}

ms_status ms_set_sources_xy(ms_grid* g, const ms_source_xy* src, int nsrc) {
  if (!valid_grid(g)) return fail(MS_EINVAL, "invalid grid");
  if (g->g3 || g->desc.scheme != MS_SCHEME_C4)
    return fail(MS_EUNSUPPORTED, "sources are implemented for 2D grids of the compact scheme");
  if (nsrc < 0 || nsrc > 64 || (nsrc > 0 && !src)) return fail(MS_EINVAL, "invalid sources (0 <= nsrc <= 64)");
  bool wall = false;
  std::vector<SrcSpec> sp(nsrc);
  for (int q = 0; q < nsrc; ++q) {
    const ms_source_xy& r = src[q];
    if ((r.cos_x != 0 && r.cos_x != 1) || (r.cos_y != 0 && r.cos_y != 1))
      return fail(MS_EINVAL, "cos_x and cos_y must be 0 or 1");
    if (r.m < (r.cos_x ? 0 : 1) || r.n < (r.cos_y ? 0 : 1))
      return fail(MS_EINVAL, "source indices must be >= 1 (sine) or >= 0 (cosine)");
    if (r.m > 1000000 || r.n > 1000000) return fail(MS_EINVAL, "source indices must be <= 1e6");
    if (!std::isfinite(r.amp) || !std::isfinite(r.omega)) return fail(MS_EINVAL, "non-finite source");
    wall |= (r.cos_x || r.cos_y);
    sp[q] = SrcSpec{r.m, r.n, r.cos_x, r.cos_y, r.amp, r.omega};
  }
  if (wall && g->desc.closure != MS_CLOSURE_PAPER)
    return fail(MS_EUNSUPPORTED, "sources that do not vanish on the walls need the PAPER closure");
  if (wall && g->desc.precision == MS_FP32_REFINED && g->N < 5)
    return fail(MS_EUNSUPPORTED, "FP32_REFINED sources that do not vanish on the walls need n >= 5 "
                                 "(the PAPER end rows of a Pade line take four outputs)");
  return set_sources_spec(g, sp.data(), nsrc);
}

ms_status ms_init_driven(ms_grid* g, const ms_source* src, int nsrc) {
  if (!valid_grid(g)) return fail(MS_EINVAL, "invalid grid");
  if (g->g3) return fail(MS_EUNSUPPORTED, "driven solutions are implemented for 2D grids");
  MS_TRY(check_sources(g, src, nsrc, true));
  std::vector<ms_mode> modes;
  std::vector<double> w;
  driven_modes(g, src, nsrc, &modes, &w);
  double* dst[3] = {g->s64[3], g->s64[4], g->s64[5]};
  MS_TRY(exact_fields64(g, modes.data(), nsrc, 0.0, 0.5 * g->ht, dst, w.data()));
  MS_TRY(store_state(g, dst));
  g->step = 0;
  MS_TRY(sync_step(g));
  MS_CUDA(cudaStreamSynchronize(g->stream));
  return MS_OK;
}

ms_status ms_error_vs_driven(ms_grid* g, const ms_source* src, int nsrc, double* l2_abs, double* l2_rel,
                             double* max_abs, double* sum_abs) {
  if (!valid_grid(g)) return fail(MS_EINVAL, "invalid grid");
  if (g->g3) return fail(MS_EUNSUPPORTED, "driven solutions are implemented for 2D grids");
  MS_TRY(check_sources(g, src, nsrc, true));
  std::vector<ms_mode> modes;
  std::vector<double> w;
  driven_modes(g, src, nsrc, &modes, &w);
  double* ex[3] = {g->s64[0], g->s64[1], g->s64[2]};
  MS_TRY(exact_fields64(g, modes.data(), nsrc, g->step * g->ht, (g->step + 0.5) * g->ht, ex, w.data()));
  double* tmp[3] = {g->s64[3], g->s64[4], g->s64[5]};
  const double* view[3];
  MS_TRY(state64(g, tmp, view));
  for (int f = 0; f < 3; ++f) {
    const size_t n = g->sh[f].size();
    launch_err_reduce(view[f], ex[f], n, g->d_partial, reduce_blocks(n), g->d_result, f > 0, g->stream);
  }
  MS_TRY(check_launch("error reduce"));
  double r[4];
  MS_CUDA(cudaMemcpyAsync(r, g->d_result, sizeof r, cudaMemcpyDeviceToHost, g->stream));
  MS_CUDA(cudaStreamSynchronize(g->stream));
  if (l2_abs) *l2_abs = std::sqrt(g->h * g->h * r[0]);
  if (l2_rel) *l2_rel = r[1] > 0 ? std::sqrt(r[0] / r[1]) : 0.0;
  if (max_abs) *max_abs = r[2];
  if (sum_abs) *sum_abs = r[3];
  return MS_OK;
}

ms_status ms_apply_op(ms_grid* g, int op, const double* const* in, double* const* out) {
  if (!valid_grid(g) || !in || !out) return fail(MS_EINVAL, "invalid argument");
  if (g->g3 || g->desc.precision != MS_FP64 || g->desc.scheme != MS_SCHEME_C4)
    return fail(MS_EUNSUPPORTED, "operator entry points need an FP64 compact-scheme grid");
  int nl = 0;
  const double c1h2 = g->c1 * g->h * g->h;
  switch (op) {
    case MS_OP_FILTER_EZ:
    case MS_OP_FILTER_HX:
    case MS_OP_FILTER_HY:
      launch_filter64(in[0], out[0], g->sh[op - MS_OP_FILTER_EZ], g->beta, g->stream);
      break;
    case MS_OP_CURL_HE:
      curl_he64(g, in[0], in[1], out[0], &nl);
      break;
    case MS_OP_CURL_EH:
      curl_eh64(g, in[0], out[0], out[1], &nl);
      break;
    case MS_OP_P1_EZ:
    case MS_OP_P1_HX:
    case MS_OP_P1_HY:
      launch_p1_apply64(in[0], out[0], g->sh[op - MS_OP_P1_EZ], c1h2, 1.0 / (g->h * g->h), g->stream);
      break;
    case MS_OP_P1SOLVE_EZ:
    case MS_OP_P1SOLVE_HX:
    case MS_OP_P1SOLVE_HY:
      p1_solve64(g, op - MS_OP_P1SOLVE_EZ, in[0], out[0], nullptr, 0.0, &nl);
      break;
    default:
      return fail(MS_EINVAL, "unknown operator");
  }
  return check_launch("apply op");
}

}  // extern "C"

// =======================================================================================
// Batches of cavities

struct ms_batch {
  ms_grid_desc desc{};
  std::vector<ms_grid*> cav;
  double* s64[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  ms::TiledBatch tb;
  ms::Graph graph1, graphk;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  long long cells = 0;
  int plan[3] = {0, 16, 0};  // work-list order, steps per captured graph, persistent launches
  bool touched = false;      // some cavity's fields were set (the state may be nonzero)
};

namespace {

bool valid_batch(ms_batch* b) { return b != nullptr && !b->cav.empty(); }

ms_status batch_cavity(ms_batch* b, int cavity, ms_grid** g) {
  if (!valid_batch(b)) return fail(MS_EINVAL, "invalid batch");
  if (cavity < 0 || cavity >= (int)b->cav.size()) return fail(MS_EINVAL, "cavity index out of range");
  *g = b->cav[cavity];
  return MS_OK;
}

ms_status batch_step_launch(ms_batch* b) {
  tiled_batch_step(b->tb, b->stream, b->plan[2]);
  return check_launch("batch step");
}

// Apply a plan: rebuild the work lists when the order changes, drop the captured graphs.
ms_status batch_apply_plan(ms_batch* b, const int* plan) {
  if (plan[0] != b->plan[0]) {
    MS_CUDA(cudaStreamSynchronize(b->stream));
    tiled_batch_free(&b->tb);
    std::string err;
    if (tiled_batch_build(b->cav.data(), (int)b->cav.size(), plan[0], &b->tb, &err) != 0) return fail(MS_ENOMEM, err);
  }
  free_graph(&b->graph1);
  free_graph(&b->graphk);
  for (int k = 0; k < 3; ++k) b->plan[k] = plan[k];
  return MS_OK;
}

bool valid_plan(const int* plan) {
  return plan && plan[0] >= 0 && plan[0] <= 2 && plan[1] >= 1 && plan[1] <= 256 && (plan[2] == 0 || plan[2] == 1);
}

// ---- autotune cache: key -> plan, in memory and (if MS_AUTOTUNE_CACHE names a file) on disk ----
std::mutex g_tune_mu;
std::map<std::string, std::array<int, 3>> g_tune;

bool valid_key(const char* key) {
  if (!key || !*key || std::strlen(key) > 512) return false;
  for (const char* c = key; *c; ++c)
    if (!(std::isalnum((unsigned char)*c) || std::strchr(":;._-=,", *c))) return false;
  return true;
}

bool tune_file_lookup(const std::string& key, std::array<int, 3>* plan) {
  const char* path = std::getenv("MS_AUTOTUNE_CACHE");
  if (!path || !*path) return false;
  FILE* fp = std::fopen(path, "r");
  if (!fp) return false;
  char k[600];
  int a, b, c;
  bool found = false;
  while (std::fscanf(fp, "%599s %d %d %d", k, &a, &b, &c) == 4) {
    const int p[3] = {a, b, c};
    if (key == k && valid_plan(p)) {  // the last entry of a key wins
      *plan = {a, b, c};
      found = true;
    }
  }
  std::fclose(fp);
  return found;
}

// Key of a batch: the cavity sizes (FNV-1a hash and count), r, Z, closure, and the device's SM count
// and name, so a cached plan is reused only for the same work on the same kind of GPU.
std::string batch_key(const ms_batch* b) {
  unsigned long long h = 1469598103934665603ull;
  for (const ms_grid* g : b->cav) {
    h ^= (unsigned long long)g->N;
    h *= 1099511628211ull;
  }
  int dev = 0, sms = 0;
  cudaDeviceProp prop{};
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetDeviceProperties(&prop, dev);
  std::string name;
  for (const char* c = prop.name; *c; ++c) name += std::isalnum((unsigned char)*c) ? *c : '_';
  char buf[400];
  snprintf(buf, sizeof buf, "batch:%016llx:%zu;r=%.17g;z=%.17g;c=%d;sm=%d;%s", h, b->cav.size(), b->desc.r,
           b->desc.z_imp, b->desc.closure, sms, name.c_str());
  return buf;
}

ms_status batch_capture(ms_batch* b, Graph* gr, int steps) {
  if (gr->exec) return MS_OK;
  MS_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  ms_status st = MS_OK;
  for (int k = 0; k < steps && st == MS_OK; ++k) st = batch_step_launch(b);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  if (st != MS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(MS_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&gr->exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(MS_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  gr->graph = graph;
  gr->steps = steps;
  return MS_OK;
}

}  // namespace

extern "C" {

ms_status ms_batch_destroy(ms_batch* b) {
  if (!b) return MS_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_graph(&b->graph1);
  free_graph(&b->graphk);
  tiled_batch_free(&b->tb);
  for (ms_grid* g : b->cav) ms_destroy(g);
  for (int k = 0; k < 6; ++k) dev_free(b->s64[k]);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return MS_OK;
}

ms_status ms_create_batch(const ms_grid_desc* d, const int* n, int count, ms_batch** out) {
  g_last_error.clear();
  if (!out) return fail(MS_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d || !n) return fail(MS_EINVAL, "desc or n is NULL");
  if (count < 1 || count > (1 << 20)) return fail(MS_EINVAL, "count must be in [1, 2^20]");
  if (d->dim != 2) return fail(MS_EUNSUPPORTED, "batches hold 2D cavities");
  if (d->precision != MS_FP32_REFINED || d->scheme != MS_SCHEME_C4)
    return fail(MS_EUNSUPPORTED, "batches run the compact scheme in MS_FP32_REFINED");
  int nmax = 0;
  for (int c = 0; c < count; ++c) {
    if (n[c] < 4 || n[c] > 32768) return fail(MS_EINVAL, "every n[b] must be in [4, 32768]");
    nmax = n[c] > nmax ? n[c] : nmax;
  }
  ms_batch* b = new ms_batch();
  b->desc = *d;
  auto cleanup = [&](ms_status s) {
    ms_batch_destroy(b);
    return s;
  };
  if (d->stream) {
    b->stream = (cudaStream_t)d->stream;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(fail(MS_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e)));
    b->own_stream = true;
  }
  const size_t plane = (size_t)(nmax + 1) * (nmax + 1);
  for (int k = 0; k < 6; ++k) {
    ms_status s = dalloc(&b->s64[k], plane);
    if (s != MS_OK) return cleanup(s);
  }
  b->cav.reserve(count);
  for (int c = 0; c < count; ++c) {
    ms_grid_desc dc = *d;
    dc.n = n[c];
    dc.stream = b->stream;
    ms_grid* g = nullptr;
    ms_status s = create_grid_impl(&dc, b->s64, &g);
    if (s != MS_OK) return cleanup(s);
    b->cav.push_back(g);
    b->cells += (long long)n[c] * n[c];
  }
  std::string err;
  if (tiled_batch_build(b->cav.data(), count, b->plan[0], &b->tb, &err) != 0) return cleanup(fail(MS_ENOMEM, err));
  *out = b;
  return MS_OK;
}

ms_status ms_batch_init_modes(ms_batch* b, int cavity, const ms_mode* modes, int nmodes) {
  ms_grid* g;
  MS_TRY(batch_cavity(b, cavity, &g));
  b->touched = true;
  return ms_init_modes(g, modes, nmodes);
}

ms_status ms_batch_set_fields(ms_batch* b, int cavity, const double* const* comps, long step) {
  ms_grid* g;
  MS_TRY(batch_cavity(b, cavity, &g));
  b->touched = true;
  return ms_set_fields(g, comps, step);
}

ms_status ms_batch_set_plan(ms_batch* b, const int* plan) {
  if (!valid_batch(b)) return fail(MS_EINVAL, "invalid batch");
  if (!valid_plan(plan)) return fail(MS_EINVAL, "plan must be {order 0..2, chunk 1..256, persistent 0|1}");
  return batch_apply_plan(b, plan);
}

ms_status ms_batch_get_plan(ms_batch* b, int* plan) {
  if (!valid_batch(b) || !plan) return fail(MS_EINVAL, "invalid argument");
  for (int k = 0; k < 3; ++k) plan[k] = b->plan[k];
  return MS_OK;
}

ms_status ms_autotune_cache_get(const char* key, int* plan, int* found) {
  if (!valid_key(key) || !plan || !found) return fail(MS_EINVAL, "invalid key or output");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  *found = 0;
  auto it = g_tune.find(key);
  std::array<int, 3> p{};
  if (it != g_tune.end()) {
    p = it->second;
  } else if (tune_file_lookup(key, &p)) {
    g_tune[key] = p;
  } else {
    return MS_OK;
  }
  for (int k = 0; k < 3; ++k) plan[k] = p[k];
  *found = 1;
  return MS_OK;
}

ms_status ms_autotune_cache_put(const char* key, const int* plan) {
  if (!valid_key(key)) return fail(MS_EINVAL, "invalid key");
  if (!valid_plan(plan)) return fail(MS_EINVAL, "invalid plan");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = {plan[0], plan[1], plan[2]};
  const char* path = std::getenv("MS_AUTOTUNE_CACHE");
  if (path && *path) {
    FILE* fp = std::fopen(path, "a");
    if (!fp) return fail(MS_EINVAL, std::string("cannot append to the autotune cache ") + path);
    const bool ok = std::fprintf(fp, "%s %d %d %d\n", key, plan[0], plan[1], plan[2]) > 0;
    if (std::fclose(fp) != 0 || !ok) return fail(MS_EINVAL, std::string("writing the autotune cache failed: ") + path);
  }
  return MS_OK;
}

ms_status ms_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
  return MS_OK;
}

ms_status ms_batch_autotune(ms_batch* b, int trial_steps, int* plan, int* from_cache) {
  if (!valid_batch(b)) return fail(MS_EINVAL, "invalid batch");
  if (trial_steps < 1 || trial_steps > 4096) return fail(MS_EINVAL, "trial_steps must be in [1, 4096]");
  if (b->touched)
    return fail(MS_EINVAL, "autotune before setting any cavity's fields: its trial steps run on the zero state");
  const std::string key = batch_key(b);
  int cached[3], found = 0;
  MS_TRY(ms_autotune_cache_get(key.c_str(), cached, &found));
  if (from_cache) *from_cache = found;
  if (found) {
    MS_TRY(batch_apply_plan(b, cached));
    if (plan)
      for (int k = 0; k < 3; ++k) plan[k] = b->plan[k];
    return MS_OK;
  }
  // trials: every candidate captured as its own graph and timed with CUDA events over whole graph
  // launches; the state is zero and stays zero, and the cavities' step counters are not advanced
  cudaEvent_t e0, e1;
  MS_CUDA(cudaEventCreate(&e0));
  MS_CUDA(cudaEventCreate(&e1));
  int best[3] = {0, 16, 0};
  float best_ms = 1e30f;
  ms_status st = MS_OK;
  for (int order = 0; order <= 2 && st == MS_OK; ++order)
    for (int chunk : {8, 32})
      for (int pers = 0; pers <= 1 && st == MS_OK; ++pers) {
        const int cand[3] = {order, chunk, pers};
        st = batch_apply_plan(b, cand);
        if (st == MS_OK) st = batch_capture(b, &b->graphk, chunk);
        if (st != MS_OK) break;
        const int reps = trial_steps > chunk ? (trial_steps + chunk - 1) / chunk : 1;
        if (cudaGraphLaunch(b->graphk.exec, b->stream) != cudaSuccess ||  // warm-up
            cudaEventRecord(e0, b->stream) != cudaSuccess) {
          st = fail(MS_ECUDA, "autotune trial launch failed");
          break;
        }
        for (int r = 0; r < reps && st == MS_OK; ++r)
          if (cudaGraphLaunch(b->graphk.exec, b->stream) != cudaSuccess) st = fail(MS_ECUDA, "autotune trial launch failed");
        float ms = 0.0f;
        if (st == MS_OK && (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
          st = fail(MS_ECUDA, "autotune timing failed");
        if (st != MS_OK) break;
        const float per_step = ms / (float)(reps * chunk);
        if (per_step < best_ms) {
          best_ms = per_step;
          for (int k = 0; k < 3; ++k) best[k] = cand[k];
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MS_OK) return st;
  MS_TRY(batch_apply_plan(b, best));
  MS_TRY(ms_autotune_cache_put(key.c_str(), best));
  if (plan)
    for (int k = 0; k < 3; ++k) plan[k] = best[k];
  return MS_OK;
}

ms_status ms_batch_get_fields(ms_batch* b, int cavity, double* const* comps) {
  ms_grid* g;
  MS_TRY(batch_cavity(b, cavity, &g));
  return ms_get_fields(g, comps);
}

ms_status ms_batch_error_vs_exact(ms_batch* b, int cavity, const ms_mode* modes, int nmodes, double* l2_abs,
                                  double* l2_rel, double* max_abs, double* sum_abs) {
  ms_grid* g;
  MS_TRY(batch_cavity(b, cavity, &g));
  return ms_error_vs_exact(g, modes, nmodes, l2_abs, l2_rel, max_abs, sum_abs);
}

ms_status ms_batch_step(ms_batch* b) {
  if (!valid_batch(b)) return fail(MS_EINVAL, "invalid batch");
  MS_TRY(batch_step_launch(b));
  for (ms_grid* g : b->cav) g->step += 1;
  return MS_OK;
}

ms_status ms_batch_run(ms_batch* b, long nsteps) {
  if (!valid_batch(b)) return fail(MS_EINVAL, "invalid batch");
  if (nsteps < 0) return fail(MS_EINVAL, "nsteps must be >= 0");
  const int chunk = b->plan[1];
  if (nsteps >= chunk) MS_TRY(batch_capture(b, &b->graphk, chunk));
  if (nsteps % chunk) MS_TRY(batch_capture(b, &b->graph1, 1));
  long left = nsteps;
  while (left >= chunk) {
    MS_CUDA(cudaGraphLaunch(b->graphk.exec, b->stream));
    left -= chunk;
  }
  while (left > 0) {
    MS_CUDA(cudaGraphLaunch(b->graph1.exec, b->stream));
    left -= 1;
  }
  for (ms_grid* g : b->cav) g->step += nsteps;
  return MS_OK;
}

ms_status ms_batch_sync(ms_batch* b) {
  if (!valid_batch(b)) return fail(MS_EINVAL, "invalid batch");
  MS_CUDA(cudaStreamSynchronize(b->stream));
  return MS_OK;
}

ms_status ms_batch_info(ms_batch* b, int* count, long long* cells, int* launches) {
  if (!valid_batch(b)) return fail(MS_EINVAL, "invalid batch");
  if (count) *count = (int)b->cav.size();
  if (cells) *cells = b->cells;
  if (launches) *launches = 4;
  return MS_OK;
}

}  // extern "C"
