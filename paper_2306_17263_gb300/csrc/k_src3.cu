// Current sources on 3D grids: divergence-free driven modes shaped like a cavity mode's E,
//   J = (a_x cos ax sin by sin cz, a_y sin ax cos by sin cz, a_z sin ax sin by cos cz) sin(w t),
// (a, b, c) = pi (m, n, p), (a_x, a_y, a_z) . (m, n, p) = 0.  The source terms of Sec. 3.1 (the
// Taylor expansion written out with Faraday's and Ampere's laws), each through the filter of
// Eq. "eq:ell" with the exact Laplacian of the source, filt = beta - (h^2/12)(a^2 + b^2 + c^2):
//   Step 1, t^{n+1/2}:  R_E += -Z filt (kappa^2 - w^2) sin(w t) a_c (E-mode shape of component c),
//   Step 2, t^{n+1}:    R_H += filt w cos(w t) (curl of the shape)_c (H-mode shape of component c),
// (curl)_x = a_z b - a_y c, (curl)_y = a_x c - a_z a, (curl)_z = a_y a - a_x b.  Every shape is a
// product of one table per axis (sine at the nodes of a Dirichlet axis, cosine at the half-nodes of
// a Neumann axis), so a source term is a separable sum; the time factors of the current step come
// from one small kernel reading the step index on the device, so captured step graphs stay valid.
#include <cmath>
#include <string>
#include <vector>

#include "k_fp64.cuh"
#include "k_src3.cuh"

namespace ms {
namespace {

constexpr int kMaxSrc3 = 64;
const dim3 kSrcBlk(32, 8, 1);

ms_status sfail(ms_status s, const std::string& m) {
  set_last_error(m.c_str());
  return s;
}

// fac[c][q] = coef[c][q] x (time factor of the side of c at the current step) x units of c's side.
__global__ void k_src3_time(const double* __restrict__ coef, const double* __restrict__ omega, int nsrc,
                            const long* __restrict__ d_step, double ht, double kappa2, double unit_e, double unit_h,
                            double* __restrict__ fac, float* __restrict__ fac32) {
  const int q = threadIdx.x;
  if (q >= nsrc) return;
  const double w = omega[q];
  const double n = (double)*d_step;
  const double te = (kappa2 - w * w) * sin(w * (n + 0.5) * ht);
  const double th = w * cos(w * (n + 1.0) * ht);
  for (int c = 0; c < 6; ++c) {
    const double f = coef[c * nsrc + q] * (c < 3 ? te : th);
    fac[c * nsrc + q] = f;
    fac32[c * nsrc + q] = (float)(f * (c < 3 ? unit_e : unit_h));
  }
}

// R += sum_q fac[q] X_q(i) Y_q(j) Z_q(k) at the unknowns of a component (walls stay zero).
template <typename T>
__global__ void k_src3_add(T* __restrict__ R, Shape3 s, const T* __restrict__ tab, const T* __restrict__ fac,
                           int nsrc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= s.n[0] || j >= s.n[1]) return;
  if (!(interior(s.bc[0], i, s.n[0]) && interior(s.bc[1], j, s.n[1]) && interior(s.bc[2], k, s.n[2]))) return;
  const int per = s.n[0] + s.n[1] + s.n[2];
  T v = (T)0;
  for (int q = 0; q < nsrc; ++q) {
    const T* t = tab + (size_t)q * per;
    v += fac[q] * t[i] * t[s.n[0] + j] * t[s.n[0] + s.n[1] + k];
  }
  const size_t p = ((size_t)k * s.n[1] + j) * s.n[0] + i;
  R[p] += v;
}

// Table value on axis position i of a component's axis with boundary type bc, wavenumber index kk.
double axis_value(int bc, int kk, int i, int N) {
  if (bc == DIR) {
    if (i == 0 || i == N) return 0.0;
    const long q = ((long)kk * i) % (2L * N);
    return std::sin(M_PI * (double)q / N);
  }
  const long q = ((long)kk * (2L * i + 1)) % (4L * N);
  return std::cos(M_PI * (double)q / (2.0 * N));
}

void shapes3(const ms_grid* g, const ms_source3* src, int nsrc, int c, std::vector<double>* out) {
  const Shape3 s = field_shape3(g->N, c);
  const int per = s.n[0] + s.n[1] + s.n[2];
  out->assign((size_t)nsrc * per, 0.0);
  for (int q = 0; q < nsrc; ++q) {
    const int kk[3] = {src[q].m, src[q].n, src[q].p};
    size_t o = (size_t)q * per;
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < s.n[a]; ++i) (*out)[o++] = axis_value(s.bc[a], kk[a], i, g->N);
  }
}

}  // namespace

void src3_free(ms_grid* g) {
  Src3* S = g->src3;
  if (!S) return;
  dev_free(S->tab);
  dev_free(S->tab32);
  dev_free(S->coef);
  dev_free(S->omega);
  dev_free(S->fac);
  dev_free(S->fac32);
  delete S;
  g->src3 = nullptr;
}

ms_status src3_set(ms_grid* g, const ms_source3* src, int nsrc) {
  src3_free(g);
  if (nsrc == 0) return MS_OK;
  std::vector<double> tab, tq, coef(6 * (size_t)nsrc), omega(nsrc);
  Src3 S;
  S.nsrc = nsrc;
  for (int c = 0; c < 6; ++c) {
    S.tab_off[c] = tab.size();
    shapes3(g, src, nsrc, c, &tq);
    tab.insert(tab.end(), tq.begin(), tq.end());
  }
  const double h = g->h;
  for (int q = 0; q < nsrc; ++q) {
    const double k3[3] = {M_PI * src[q].m, M_PI * src[q].n, M_PI * src[q].p};
    const double filt = g->beta - (h * h / 12.0) * (k3[0] * k3[0] + k3[1] * k3[1] + k3[2] * k3[2]);
    const double ax = src[q].ax, ay = src[q].ay, az = src[q].az;
    const double e[3] = {ax, ay, az};
    const double cu[3] = {az * k3[1] - ay * k3[2], ax * k3[2] - az * k3[0], ay * k3[0] - ax * k3[1]};
    for (int c = 0; c < 3; ++c) {
      coef[c * (size_t)nsrc + q] = -g->Z * filt * e[c];
      coef[(3 + c) * (size_t)nsrc + q] = filt * cu[c];
    }
    omega[q] = src[q].omega;
  }
  std::vector<float> tab32(tab.begin(), tab.end());
  Src3* D = new Src3(S);
  g->src3 = D;
  auto alloc = [](void** p, size_t bytes) { return dev_malloc(p, bytes) == cudaSuccess; };
  bool ok = alloc((void**)&D->tab, tab.size() * sizeof(double)) && alloc((void**)&D->tab32, tab32.size() * sizeof(float)) &&
            alloc((void**)&D->coef, coef.size() * sizeof(double)) && alloc((void**)&D->omega, omega.size() * sizeof(double)) &&
            alloc((void**)&D->fac, coef.size() * sizeof(double)) && alloc((void**)&D->fac32, coef.size() * sizeof(float));
  if (!ok) {
    src3_free(g);
    return sfail(MS_ENOMEM, "cudaMalloc of the 3D source tables failed");
  }
  ok = cudaMemcpy(D->tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(D->tab32, tab32.data(), tab32.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(D->coef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(D->omega, omega.data(), omega.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    src3_free(g);
    return sfail(MS_ECUDA, "copy of the 3D source tables failed");
  }
  return MS_OK;
}

void src3_time(ms_grid* g) {
  const Src3* S = g->src3;
  // units of the FP32 right-hand side b: 6 h^2 P1 x = b with E += (12 Z / r) x, H += (12 / (r Z)) x
  const double hr2 = g->h * g->h * g->h * g->desc.r * g->desc.r;
  k_src3_time<<<1, kMaxSrc3, 0, g->stream>>>(S->coef, S->omega, S->nsrc, g->d_step, g->ht, g->kappa2,
                                             hr2 / (2.0 * g->Z), hr2 * g->Z / 2.0, S->fac, S->fac32);
}

void src3_add(ms_grid* g, int c, void* R) {
  const Src3* S = g->src3;
  const Shape3 s = field_shape3(g->N, c);
  const dim3 grd((s.n[0] + kSrcBlk.x - 1) / kSrcBlk.x, (s.n[1] + kSrcBlk.y - 1) / kSrcBlk.y, s.n[2]);
  if (g->desc.precision == MS_FP64)
    k_src3_add<double><<<grd, kSrcBlk, 0, g->stream>>>((double*)R, s, S->tab + S->tab_off[c], S->fac + c * S->nsrc,
                                                       S->nsrc);
  else
    k_src3_add<float><<<grd, kSrcBlk, 0, g->stream>>>((float*)R, s, S->tab32 + S->tab_off[c], S->fac32 + c * S->nsrc,
                                                      S->nsrc);
}

// The exact driven solution of the sources for component c at times tE (E) and tH (H).
ms_status exact_driven3(ms_grid* g, const ms_source3* src, int nsrc, double tE, double tH, int c, double* out) {
  // E = A cos(w tE) a, H = -(A sin(w tH) / (Z w)) curl(shape), A = Z w / (w^2 - |k|^2), per source
  std::vector<double> tq;
  shapes3(g, src, nsrc, c, &tq);
  std::vector<double> coef(nsrc);
  for (int q = 0; q < nsrc; ++q) {
    const double k3[3] = {M_PI * src[q].m, M_PI * src[q].n, M_PI * src[q].p};
    const double w = src[q].omega, k2 = k3[0] * k3[0] + k3[1] * k3[1] + k3[2] * k3[2];
    const double A = g->Z * w / (w * w - k2);
    const double ax = src[q].ax, ay = src[q].ay, az = src[q].az;
    const double ce = A * std::cos(w * tE), sh = -A * std::sin(w * tH) / (g->Z * w);
    const double amp[6] = {ce * ax, ce * ay, ce * az, sh * (az * k3[1] - ay * k3[2]), sh * (ax * k3[2] - az * k3[0]),
                           sh * (ay * k3[0] - ax * k3[1])};
    coef[q] = amp[c];
  }
  return mode_field3_tables(g, c, tq, coef, out);
}

}  // namespace ms
