// Taylor initialisation of non-mode data and the reverse (adjoint) pass of the time step, in
// FP64, on the grid's stream.
//
// One step (Sec. 3.4) is the linear map M = S2 S1 on the unknowns (E_z, H_x, H_y):
//   S1: E += h_tau P1_E^{-1} C_HE F_H H,   C_HE = kappa^2 Z (delta_x (.)_y - delta_y (.)_x)
//   S2: H += h_tau P1_H^{-1} C_EH F_E E,   C_EH = (kappa^2/Z) (-delta_y, delta_x)
// with F the right-hand-side filter of Eq. "eq:ell" and P1 of Definition "def:operatorsP".
// F and P1 are symmetric on the unknowns (Dirichlet zeros, even Neumann ghosts), so
//   S2^T: l_E += h_tau F_E C_EH^T P1_H^{-1} l_H,   S1^T: l_H += h_tau F_H C_HE^T P1_E^{-1} l_E,
// and M^T = S1^T S2^T applies S2^T first.  The transposed Pade derivative delta^T is the
// transpose of the truncated band the forward kernels apply (build_pade_table_T), so the
// reverse pass is the transpose of the forward FP64 step up to rounding.
#include <string>

#include "k_fp64.cuh"
#include "k_mixed.cuh"

namespace ms {

namespace {

ms_status afail(ms_status s, const std::string& msg) {
  set_last_error(msg.c_str());
  return s;
}

#define MS_ACUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return afail(MS_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define MS_ATRY(expr)           \
  do {                          \
    ms_status s_ = (expr);      \
    if (s_ != MS_OK) return s_; \
  } while (0)

// out (+)= a u + b L u at the unknowns of one field, L = h^2 Delta_h the 5-point Laplacian with
// the ghost rules of Table "tab:bc" (Dirichlet neighbours are the stored zeros, Neumann
// neighbours across the wall are even ghosts).  Without accumulation the Dirichlet boundary
// points of out are set to 0; with it they are left unchanged.
__global__ void k_lap_axpby64(const double* __restrict__ u, double* __restrict__ out, int nx, int ny, int bcx, int bcy,
                              double a, double b, int accumulate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  const size_t p = (size_t)j * nx + i;
  if (!interior(bcx, i, nx) || !interior(bcy, j, ny)) {
    if (!accumulate) out[p] = 0.0;
    return;
  }
  const int im = clampi(i - 1, nx), ip = clampi(i + 1, nx), jm = clampi(j - 1, ny), jp = clampi(j + 1, ny);
  const double c = u[p];
  const double lap = u[(size_t)j * nx + im] + u[(size_t)j * nx + ip] + u[(size_t)jm * nx + i] +
                     u[(size_t)jp * nx + i] - 4.0 * c;
  const double v = a * c + b * lap;
  if (accumulate) out[p] += v;
  else out[p] = v;
}

void lap_axpby64(const double* u, double* out, const Shape& s, double a, double b, int accumulate, cudaStream_t st) {
  dim3 blk(32, 8);
  dim3 grd((s.nx + blk.x - 1) / blk.x, (s.ny + blk.y - 1) / blk.y);
  k_lap_axpby64<<<grd, blk, 0, st>>>(u, out, s.nx, s.ny, s.bcx, s.bcy, a, b, accumulate);
}

ms_status check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return afail(MS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return MS_OK;
}

// Transposed tables and the six adjoint planes, on first use.
ms_status adjoint_setup(ms_grid* g) {
  if (g->adj[0]) return MS_OK;
  if (g->shared64) return afail(MS_EUNSUPPORTED, "the reverse pass is not available on batch cavities");
  // on any failure everything allocated here is released, so the next call starts afresh
  auto release = [&]() {
    for (int kind = 0; kind < 2; ++kind) {
      dev_free(g->padeT[kind].d_w);
      g->padeT[kind].d_w = nullptr;
    }
    for (int k = 0; k < 6; ++k) {
      dev_free(g->adj[k]);
      g->adj[k] = nullptr;
    }
  };
  for (int kind = 0; kind < 2; ++kind) {
    PadeTable& t = g->padeT[kind];
    build_pade_table_T(g->pade[kind], &t);
    const cudaError_t e = dev_malloc((void**)&t.d_w, t.w.size() * sizeof(double));
    if (e != cudaSuccess) {
      release();
      return afail(MS_ENOMEM, std::string("cudaMalloc of the transposed Pade tables: ") + cudaGetErrorString(e));
    }
    if (cudaMemcpy(t.d_w, t.w.data(), t.w.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
      release();
      return afail(MS_ECUDA, "copy of the transposed Pade tables failed");
    }
  }
  const size_t nmax = (size_t)(g->N + 1) * (g->N + 1);
  for (int k = 0; k < 6; ++k) {
    const cudaError_t e = dev_malloc((void**)&g->adj[k], nmax * sizeof(double) + 256);
    if (e != cudaSuccess) {
      release();
      return afail(MS_ENOMEM, std::string("cudaMalloc of adjoint planes: ") + cudaGetErrorString(e));
    }
    if (cudaMemsetAsync(g->adj[k], 0, nmax * sizeof(double), g->stream) != cudaSuccess) {
      release();
      return afail(MS_ECUDA, "clearing the adjoint planes failed");
    }
  }
  return MS_OK;
}

// H^{1/2} = Z^{-1} (t1 + (t1^3/6) Delta_h) (-delta_y E, delta_x E), t1 = h_tau/2 (Sec. 5.1,
// Eq. "talorh" with H^0 = 0).  Scratch: s64[1], s64[2].
void taylor_h64(ms_grid* g, const double* ez, double* hx, double* hy) {
  const int N = g->N;
  const double t1 = 0.5 * g->ht, c3 = t1 * t1 * t1 / 6.0, h2 = g->h * g->h;
  double* cx = g->s64[1];
  double* cy = g->s64[2];
  const PadeTable& t = g->pade[NODE_TO_HALF];
  launch_pade64(1, ez, cx, N + 1, N + 1, N, N + 1, 0, 1, N, t, -1.0 / g->h, 0, g->stream);
  launch_pade64(0, ez, cy, N + 1, N + 1, N, N, 0, 1, N, t, 1.0 / g->h, 0, g->stream);
  lap_axpby64(cx, hx, g->sh[HX], t1 / g->Z, c3 / (g->Z * h2), 0, g->stream);
  lap_axpby64(cy, hy, g->sh[HY], t1 / g->Z, c3 / (g->Z * h2), 0, g->stream);
}

// out (+)= T_H^T (l_hx, l_hy), the transpose of taylor_h64; out's Dirichlet boundary zeroed.
// Scratch: adj[4], adj[5].
void taylor_h64_T(ms_grid* g, const double* lhx, const double* lhy, double* out, int accumulate) {
  const int N = g->N;
  const double t1 = 0.5 * g->ht, c3 = t1 * t1 * t1 / 6.0, h2 = g->h * g->h;
  double* wx = g->adj[4];
  double* wy = g->adj[5];
  lap_axpby64(lhx, wx, g->sh[HX], t1 / g->Z, c3 / (g->Z * h2), 0, g->stream);
  lap_axpby64(lhy, wy, g->sh[HY], t1 / g->Z, c3 / (g->Z * h2), 0, g->stream);
  const PadeTable& t = g->padeT[NODE_TO_HALF];
  launch_pade64(0, wy, out, N + 1, N, N + 1, N + 1, 0, 1, N, t, 1.0 / g->h, accumulate, g->stream);
  launch_pade64(1, wx, out, N + 1, N + 1, N + 1, N + 1, 0, 1, N, t, -1.0 / g->h, 1, g->stream);
  launch_zero_dirichlet64(out, g->sh[EZ], g->stream);
}

// One transposed step on the adjoint state adj[0..2] = (l_E, l_Hx, l_Hy), in place.
// Scratch: adj[3..5] and the FP64 solve's s64[3], s64[4].
void adjoint_step64(ms_grid* g) {
  const int N = g->N;
  int nl = 0;
  double *lE = g->adj[0], *lHx = g->adj[1], *lHy = g->adj[2];
  double *e = g->adj[3], *x = g->adj[4], *y = g->adj[5];
  const double s_eh = g->kappa2 / (g->Z * g->h), s_he = g->kappa2 * g->Z / g->h;
  // S2^T: u_H = P1_H^{-1} l_H; v = (kappa^2/Z)(delta_x^T u_y - delta_y^T u_x); l_E += h_tau F_E v
  p1_solve64(g, HX, lHx, x, nullptr, 0.0, &nl);
  p1_solve64(g, HY, lHy, y, nullptr, 0.0, &nl);
  const PadeTable& tn = g->padeT[NODE_TO_HALF];
  launch_pade64(0, y, e, N + 1, N, N + 1, N + 1, 0, 1, N, tn, s_eh, 0, g->stream);
  launch_pade64(1, x, e, N + 1, N + 1, N + 1, N + 1, 0, 1, N, tn, -s_eh, 1, g->stream);
  launch_zero_dirichlet64(e, g->sh[EZ], g->stream);
  lap_axpby64(e, lE, g->sh[EZ], g->ht * g->beta, g->ht / 12.0, 1, g->stream);
  // S1^T: u_E = P1_E^{-1} l_E; (v_x, v_y) = kappa^2 Z (-delta_y^T u_E, delta_x^T u_E) from the
  // interior nodes of u_E; l_H += h_tau F_H v
  p1_solve64(g, EZ, lE, e, nullptr, 0.0, &nl);
  const PadeTable& th = g->padeT[HALF_TO_NODE];
  launch_pade64(0, e + 1, y, N + 1, N + 1, N, N, 0, 1, N, th, s_he, 0, g->stream);
  launch_pade64(1, e + (N + 1), x, N + 1, N + 1, N, N + 1, 0, 1, N, th, -s_he, 0, g->stream);
  lap_axpby64(x, lHx, g->sh[HX], g->ht * g->beta, g->ht / 12.0, 1, g->stream);
  lap_axpby64(y, lHy, g->sh[HY], g->ht * g->beta, g->ht / 12.0, 1, g->stream);
}

ms_status adj_capture(ms_grid* g, Graph* gr, int steps) {
  if (gr->exec) return MS_OK;
  MS_ACUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < steps; ++k) adjoint_step64(g);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
  if (e != cudaSuccess) return afail(MS_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&gr->exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return afail(MS_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  gr->graph = graph;
  gr->steps = steps;
  return MS_OK;
}

// (M^T)^nsteps on adj[0..2], replaying captured chunks of 16 steps.
ms_status adjoint_steps(ms_grid* g, long nsteps) {
  const int chunk = 16;
  if (nsteps >= chunk) MS_ATRY(adj_capture(g, &g->adj_graphk, chunk));
  if (nsteps % chunk) MS_ATRY(adj_capture(g, &g->adj_graph1, 1));
  long left = nsteps;
  for (; left >= chunk; left -= chunk) MS_ACUDA(cudaGraphLaunch(g->adj_graphk.exec, g->stream));
  for (; left > 0; --left) MS_ACUDA(cudaGraphLaunch(g->adj_graph1.exec, g->stream));
  return MS_OK;
}

bool valid(ms_grid* g) { return g != nullptr && g->N > 0; }

ms_status check_grid(ms_grid* g) {
  if (!valid(g)) return afail(MS_EINVAL, "invalid grid");
  if (g->g3) return afail(MS_EUNSUPPORTED, "the reverse pass is implemented for 2D grids");
  if (g->desc.scheme != MS_SCHEME_C4) return afail(MS_EUNSUPPORTED, "the reverse pass is for the compact scheme");
  return adjoint_setup(g);
}

void free_graph(Graph* gr) {
  if (gr->exec) cudaGraphExecDestroy(gr->exec);
  if (gr->graph) cudaGraphDestroy(gr->graph);
  *gr = Graph{};
}

ms_status copy_in(ms_grid* g, double* dst, const double* src, size_t n, cudaMemcpyKind kind) {
  MS_ACUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), kind, g->stream));
  return MS_OK;
}

ms_status taylor_init_dev(ms_grid* g, const double* ez0) {
  double* e = g->adj[3];
  if (ez0 != e) MS_ATRY(copy_in(g, e, ez0, g->sh[EZ].size(), cudaMemcpyDeviceToDevice));
  launch_zero_dirichlet64(e, g->sh[EZ], g->stream);
  taylor_h64(g, e, g->adj[4], g->adj[5]);
  MS_ATRY(check("taylor init"));
  const double* comps[3] = {g->adj[3], g->adj[4], g->adj[5]};
  return ms_set_fields_device(g, comps, 0);
}

// The reverse pass in FP32 (adjoint32.cu) on FP32_REFINED grids unless FP64 was selected.
bool use32(const ms_grid* g) {
  const int prec = g->adj_precision < 0 ? g->desc.precision : g->adj_precision;
  return prec == MS_FP32_REFINED;
}

// (M^T)^nsteps on adj[0..2] in the selected arithmetic (FP32: through the float-float state).
ms_status adjoint_steps_any(ms_grid* g, long nsteps) {
  if (!use32(g)) return adjoint_steps(g, nsteps);
  MS_ATRY(adjoint32_setup(g));
  const double* in[3] = {g->adj[0], g->adj[1], g->adj[2]};
  adjoint32_load(g, in);
  MS_ATRY(adjoint32_steps(g, nsteps));
  double* out[3] = {g->adj[0], g->adj[1], g->adj[2]};
  adjoint32_store(g, out);
  return check("FP32 adjoint steps");
}

// adj[0..2] = (l_E, 0, 0) from a device array, then (M^T)^nsteps, then out = l_E + T_H^T l_H.
ms_status adjoint_run_dev(ms_grid* g, long nsteps, const double* lEz, double* out) {
  if (nsteps < 0) return afail(MS_EINVAL, "nsteps must be >= 0");
  MS_ATRY(copy_in(g, g->adj[0], lEz, g->sh[EZ].size(), cudaMemcpyDeviceToDevice));
  launch_zero_dirichlet64(g->adj[0], g->sh[EZ], g->stream);
  MS_ACUDA(cudaMemsetAsync(g->adj[1], 0, g->sh[HX].size() * sizeof(double), g->stream));
  MS_ACUDA(cudaMemsetAsync(g->adj[2], 0, g->sh[HY].size() * sizeof(double), g->stream));
  MS_ATRY(adjoint_steps_any(g, nsteps));
  MS_ATRY(copy_in(g, out, g->adj[0], g->sh[EZ].size(), cudaMemcpyDeviceToDevice));
  taylor_h64_T(g, g->adj[1], g->adj[2], out, 1);
  return check("adjoint run");
}

}  // namespace

void adjoint_teardown(ms_grid* g) {
  adjoint32_teardown(g);
  free_graph(&g->adj_graph1);
  free_graph(&g->adj_graphk);
  for (int k = 0; k < 2; ++k) {
    dev_free(g->padeT[k].d_w);
    g->padeT[k].d_w = nullptr;
  }
  for (int k = 0; k < 6; ++k) {
    dev_free(g->adj[k]);
    g->adj[k] = nullptr;
  }
}

}  // namespace ms

using namespace ms;

extern "C" {

ms_status ms_taylor_init_device(ms_grid* g, const double* ez0) {
  MS_ATRY(check_grid(g));
  if (!ez0) return afail(MS_EINVAL, "ez0 is NULL");
  return taylor_init_dev(g, ez0);
}

ms_status ms_taylor_init(ms_grid* g, const double* ez0) {
  MS_ATRY(check_grid(g));
  if (!ez0) return afail(MS_EINVAL, "ez0 is NULL");
  MS_ATRY(copy_in(g, g->adj[3], ez0, g->sh[EZ].size(), cudaMemcpyHostToDevice));
  MS_ATRY(taylor_init_dev(g, g->adj[3]));
  MS_ACUDA(cudaStreamSynchronize(g->stream));
  return MS_OK;
}

ms_status ms_adjoint_run_device(ms_grid* g, long nsteps, const double* dL_dEzT, double* dL_dEz0) {
  MS_ATRY(check_grid(g));
  if (!dL_dEzT || !dL_dEz0) return afail(MS_EINVAL, "NULL array");
  return adjoint_run_dev(g, nsteps, dL_dEzT, dL_dEz0);
}

ms_status ms_adjoint_run(ms_grid* g, long nsteps, const double* dL_dEzT, double* dL_dEz0) {
  MS_ATRY(check_grid(g));
  if (!dL_dEzT || !dL_dEz0) return afail(MS_EINVAL, "NULL array");
  const size_t n = g->sh[EZ].size();
  // host gradient staged through adj[3] (input) and adj[4] is not free (Taylor^T scratch): use s64[5]
  double* din = g->s64[5];
  MS_ATRY(copy_in(g, din, dL_dEzT, n, cudaMemcpyHostToDevice));
  MS_ATRY(adjoint_run_dev(g, nsteps, din, din));
  MS_ACUDA(cudaMemcpyAsync(dL_dEz0, din, n * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  MS_ACUDA(cudaStreamSynchronize(g->stream));
  return MS_OK;
}

ms_status ms_adjoint_steps_device(ms_grid* g, long nsteps, double* const* lam) {
  MS_ATRY(check_grid(g));
  if (!lam || !lam[0] || !lam[1] || !lam[2]) return afail(MS_EINVAL, "NULL array");
  if (nsteps < 0) return afail(MS_EINVAL, "nsteps must be >= 0");
  for (int f = 0; f < 3; ++f) {
    MS_ATRY(copy_in(g, g->adj[f], lam[f], g->sh[f].size(), cudaMemcpyDeviceToDevice));
    launch_zero_dirichlet64(g->adj[f], g->sh[f], g->stream);
  }
  MS_ATRY(adjoint_steps_any(g, nsteps));
  for (int f = 0; f < 3; ++f) MS_ATRY(copy_in(g, lam[f], g->adj[f], g->sh[f].size(), cudaMemcpyDeviceToDevice));
  return check("adjoint steps");
}

ms_status ms_adjoint_steps(ms_grid* g, long nsteps, double* const* lam) {
  MS_ATRY(check_grid(g));
  if (!lam || !lam[0] || !lam[1] || !lam[2]) return afail(MS_EINVAL, "NULL array");
  if (nsteps < 0) return afail(MS_EINVAL, "nsteps must be >= 0");
  for (int f = 0; f < 3; ++f) {
    MS_ATRY(copy_in(g, g->adj[f], lam[f], g->sh[f].size(), cudaMemcpyHostToDevice));
    launch_zero_dirichlet64(g->adj[f], g->sh[f], g->stream);
  }
  MS_ATRY(adjoint_steps_any(g, nsteps));
  for (int f = 0; f < 3; ++f)
    MS_ACUDA(cudaMemcpyAsync(lam[f], g->adj[f], g->sh[f].size() * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  MS_ACUDA(cudaStreamSynchronize(g->stream));
  return check("adjoint steps");
}

ms_status ms_set_adjoint_precision(ms_grid* g, int precision) {
  if (!valid(g)) return afail(MS_EINVAL, "invalid grid");
  if (precision != MS_FP64 && precision != MS_FP32_REFINED) return afail(MS_EINVAL, "unknown precision");
  if (precision == MS_FP32_REFINED && g->desc.precision != MS_FP32_REFINED)
    return afail(MS_EUNSUPPORTED, "the FP32 reverse pass needs an FP32_REFINED grid (its FP32 tables)");
  g->adj_precision = precision;
  return MS_OK;
}

ms_status ms_taylor_init_T(ms_grid* g, const double* l_hx, const double* l_hy, double* dEz0) {
  MS_ATRY(check_grid(g));
  if (!l_hx || !l_hy || !dEz0) return afail(MS_EINVAL, "NULL array");
  MS_ATRY(copy_in(g, g->adj[1], l_hx, g->sh[HX].size(), cudaMemcpyHostToDevice));
  MS_ATRY(copy_in(g, g->adj[2], l_hy, g->sh[HY].size(), cudaMemcpyHostToDevice));
  launch_zero_dirichlet64(g->adj[1], g->sh[HX], g->stream);
  launch_zero_dirichlet64(g->adj[2], g->sh[HY], g->stream);
  double* out = g->adj[3];
  taylor_h64_T(g, g->adj[1], g->adj[2], out, 0);
  MS_ACUDA(cudaMemcpyAsync(dEz0, out, g->sh[EZ].size() * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  MS_ACUDA(cudaStreamSynchronize(g->stream));
  return check("taylor init T");
}

}  // extern "C"
