// Current sources of the 2D TM_z problem (J = J_z z, div J = 0): a sum of driven sine modes
//   J_z = a sin(m pi x) sin(n pi y) sin(w t),
// which vanish on the walls together with every derivative the Neumann data of Sec. 3.3 use, so
// the even ghosts stay exact.  The modified Helmholtz equations of Eq. "eq:mh" gain
//   E:  P(J)^{n+1/2} = -Z (kappa^2 - w^2) J^{n+1/2},    H:  (curl d_t J)^{n+1} = (d_y d_t J_z, -d_x d_t J_z),
// (from the Taylor expansion of Sec. 3.1 with Faraday's and Ampere's laws), each through the
// right-hand-side filter of Eq. "eq:ell" with the exact Laplacian of the source, factor
// f = beta - (h^2/12) pi^2 (m^2 + n^2).  The kernels add these terms to a right-hand side before
// the solve; the step index is read from device memory so that captured graphs stay valid.
#include <cmath>
#include <cstring>
#include <vector>

#include "k_fp64.cuh"

namespace ms {
namespace {

// Per source: ce = -Z (kappa^2 - w^2) f a,  ch = f a w,  kx = pi m,  ky = pi n,  w.
struct SrcDev {
  double ce, ch, kx, ky, w;
};

// R (+)= scale * sum_q ce_q sin(w_q t) sx_q(i) sy_q(j) at the interior E_z nodes, t = (n + 1/2) h_tau.
template <typename T>
__global__ void k_src_e(T* __restrict__ R, int N, const SrcDev* __restrict__ s, int nsrc, const double* __restrict__ tab,
                        const long* __restrict__ d_step, double ht, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i < 1 || j < 1 || i >= N || j >= N) return;
  const double t = ((double)*d_step + 0.5) * ht;
  const size_t per = 4 * (size_t)(N + 1);  // per-source table block: sx, sy, cxh, cyh
  double v = 0.0;
  for (int q = 0; q < nsrc; ++q) {
    const double* tq = tab + q * per;
    v += s[q].ce * sin(s[q].w * t) * tq[i] * tq[(N + 1) + j];
  }
  R[(size_t)j * (N + 1) + i] += (T)(scale * v);
}

// R_x += scale sum ch_q cos(w_q t) ky_q sx_q(i) cyh_q(j);  R_y -= scale sum ch_q cos(w_q t) kx_q cxh_q(i) sy_q(j),
// t = (n + 1) h_tau.
template <typename T>
__global__ void k_src_h(T* __restrict__ Rx, T* __restrict__ Ry, int N, const SrcDev* __restrict__ s, int nsrc,
                        const double* __restrict__ tab, const long* __restrict__ d_step, double ht, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > N || j > N) return;
  const double t = ((double)*d_step + 1.0) * ht;
  const size_t per = 4 * (size_t)(N + 1);
  if (j < N && i >= 1 && i < N) {
    double v = 0.0;
    for (int q = 0; q < nsrc; ++q) {
      const double* tq = tab + q * per;
      v += s[q].ch * cos(s[q].w * t) * s[q].ky * tq[i] * tq[3 * (N + 1) + j];
    }
    Rx[(size_t)j * (N + 1) + i] += (T)(scale * v);
  }
  if (i < N && j >= 1 && j < N) {
    double v = 0.0;
    for (int q = 0; q < nsrc; ++q) {
      const double* tq = tab + q * per;
      v += s[q].ch * cos(s[q].w * t) * s[q].kx * tq[2 * (N + 1) + i] * tq[(N + 1) + j];
    }
    Ry[(size_t)j * N + i] -= (T)(scale * v);
  }
}

__global__ void k_tick(long* d_step) { *d_step += 1; }

}  // namespace

// Host tables: per source, sin(pi m i / N) (i = 0..N), sin(pi n j / N), cos(pi m (i + 1/2) / N)
// (i = 0..N-1), cos(pi n (j + 1/2) / N), with the arguments reduced exactly in integers.
int build_sources(ms_grid* g, const ms_source* src, int nsrc, std::vector<unsigned char>* dev_blob,
                  std::vector<double>* tabs) {
  const int N = g->N;
  const double h = g->h, pi = M_PI;
  std::vector<SrcDev> sd(nsrc);
  tabs->assign((size_t)nsrc * 4 * (N + 1), 0.0);
  auto sin_node = [&](int k, int i) {
    if (i == 0 || i == N) return 0.0;
    long q = ((long)k * i) % (2L * N);
    return std::sin(pi * (double)q / N);
  };
  auto cos_half = [&](int k, int i) {
    long q = ((long)k * (2L * i + 1)) % (4L * N);
    return std::cos(pi * (double)q / (2.0 * N));
  };
  for (int q = 0; q < nsrc; ++q) {
    const int m = src[q].m, n = src[q].n;
    const double a = src[q].amp, w = src[q].omega;
    const double f = g->beta - (h * h / 12.0) * pi * pi * ((double)m * m + (double)n * n);
    sd[q].ce = -g->Z * (g->kappa2 - w * w) * f * a;
    sd[q].ch = f * a * w;
    sd[q].kx = pi * m;
    sd[q].ky = pi * n;
    sd[q].w = w;
    double* tq = tabs->data() + (size_t)q * 4 * (N + 1);
    for (int i = 0; i <= N; ++i) tq[i] = sin_node(m, i);
    for (int j = 0; j <= N; ++j) tq[(N + 1) + j] = sin_node(n, j);
    for (int i = 0; i < N; ++i) tq[2 * (N + 1) + i] = cos_half(m, i);
    for (int j = 0; j < N; ++j) tq[3 * (N + 1) + j] = cos_half(n, j);
  }
  dev_blob->resize(sd.size() * sizeof(SrcDev));
  std::memcpy(dev_blob->data(), sd.data(), dev_blob->size());
  return (int)sizeof(SrcDev);
}

void launch_src_e64(ms_grid* g, double* R, double scale) {
  dim3 blk(32, 8), grd((g->N + 1 + 31) / 32, (g->N + 1 + 7) / 8);
  k_src_e<double><<<grd, blk, 0, g->stream>>>(R, g->N, (const SrcDev*)g->d_src, g->nsrc, g->d_srctab, g->d_step,
                                               g->ht, scale);
}
void launch_src_h64(ms_grid* g, double* Rx, double* Ry, double scale) {
  dim3 blk(32, 8), grd((g->N + 1 + 31) / 32, (g->N + 1 + 7) / 8);
  k_src_h<double><<<grd, blk, 0, g->stream>>>(Rx, Ry, g->N, (const SrcDev*)g->d_src, g->nsrc, g->d_srctab, g->d_step,
                                               g->ht, scale);
}
void launch_src_e32(ms_grid* g, float* R, double scale) {
  dim3 blk(32, 8), grd((g->N + 1 + 31) / 32, (g->N + 1 + 7) / 8);
  k_src_e<float><<<grd, blk, 0, g->stream>>>(R, g->N, (const SrcDev*)g->d_src, g->nsrc, g->d_srctab, g->d_step, g->ht,
                                              scale);
}
void launch_src_h32(ms_grid* g, float* Rx, float* Ry, double scale) {
  dim3 blk(32, 8), grd((g->N + 1 + 31) / 32, (g->N + 1 + 7) / 8);
  k_src_h<float><<<grd, blk, 0, g->stream>>>(Rx, Ry, g->N, (const SrcDev*)g->d_src, g->nsrc, g->d_srctab, g->d_step,
                                              g->ht, scale);
}
void launch_tick(ms_grid* g) { k_tick<<<1, 1, 0, g->stream>>>(g->d_step); }

}  // namespace ms
