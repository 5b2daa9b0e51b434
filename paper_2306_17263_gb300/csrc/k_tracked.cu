// Tracked-Delta-E variant of the step (MS_SCHEME_C4_DE, FP64): Sec. 3.4 as printed.  Delta E_z
// is carried as state DE, advanced after Step 1 by the modified Helmholtz equation of Eq.
// "eq:mhe" (J = 0),
//   DE^{n+1} = DE^n + kappa^2 (E^{n+1} - E^n) - Z (24/h_tau) curl_h H^{n+1/2},
// and Step 2 filters E with it as in Eq. "eq:helm2": G_E = (1 + kappa^2 h^2/12) E + (h^2/12) DE.
// DE and G_E are 0 on the PEC nodes (Table "tab:bc_terms").
#include "k_fp64.cuh"

namespace ms {
namespace {

// de += k2ht * es - c / ck, then ge = beta e + h2_12 de (0 on the boundary), where
// es = E* (E^{n+1} = E^n + h_tau E*), c = kappa^2 Z curl_h H and ck = kappa^4 h_tau / 24.
__global__ void k_de_update64(double* __restrict__ de, const double* __restrict__ es, const double* __restrict__ c,
                              const double* __restrict__ e, double* __restrict__ ge, int n, double k2ht,
                              double c24ht, double k2, double beta, double h2_12) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const size_t p = (size_t)j * n + i;
  if (i == 0 || j == 0 || i == n - 1 || j == n - 1) {
    de[p] = 0.0;
    ge[p] = 0.0;
    return;
  }
  const double d = de[p] + (k2ht * es[p] - c24ht * c[p] / k2);
  de[p] = d;
  ge[p] = beta * e[p] + h2_12 * d;
}

// de = Delta_h e (5 points, stored wall zeros) at the interior nodes, 0 on the boundary.
__global__ void k_lap_e64(const double* __restrict__ e, double* __restrict__ de, int n, double ih2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const size_t p = (size_t)j * n + i;
  if (i == 0 || j == 0 || i == n - 1 || j == n - 1) {
    de[p] = 0.0;
    return;
  }
  const double c = e[p];
  de[p] = ((e[p - 1] - 2.0 * c + e[p + 1]) + (e[p - n] - 2.0 * c + e[p + n])) * ih2;
}

}  // namespace

void launch_de_update64(double* de, const double* es, const double* c, const double* e, double* ge, int N, double ht,
                        double k2, double beta, double h, cudaStream_t st) {
  dim3 blk(32, 8);
  dim3 grd((N + 1 + 31) / 32, (N + 1 + 7) / 8);
  k_de_update64<<<grd, blk, 0, st>>>(de, es, c, e, ge, N + 1, k2 * ht, 24.0 / ht, k2, beta, h * h / 12.0);
}

void launch_lap_e64(const double* e, double* de, int N, double h, cudaStream_t st) {
  dim3 blk(32, 8);
  dim3 grd((N + 1 + 31) / 32, (N + 1 + 7) / 8);
  k_lap_e64<<<grd, blk, 0, st>>>(e, de, N + 1, 1.0 / (h * h));
}

}  // namespace ms
