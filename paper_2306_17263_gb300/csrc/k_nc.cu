// Non-compact fourth-order comparator NC (Sec. 5.2): the leapfrog updating rules of the Yee
// scheme with the stencil K4 of Eq. "eq:K4" at a = 0,
//   D u_i = (9/8 (u_{i+1/2} - u_{i-1/2}) - 1/24 (u_{i+3/2} - u_{i-3/2})) / h,
// and the standard fourth-order one-sided staggered difference at the first and last output of
// each line, (-23 u_0 + 21 u_1 + 3 u_2 - u_3) / (24 h) and its mirror image.  FP64, one kernel
// per half-step like the Yee comparator.
#include "k_fp64.cuh"

namespace ms {
namespace {

// Derivative at output k (between inputs k and k+1) of a line of nin inputs f[q * st].
__device__ __forceinline__ double nc_d(const double* __restrict__ f, int st, int k, int nin, double ih) {
  double v;
  if (k >= 1 && k + 2 < nin) {
    v = (9.0 / 8.0) * (f[(k + 1) * st] - f[k * st]) - (1.0 / 24.0) * (f[(k + 2) * st] - f[(k - 1) * st]);
  } else if (k == 0) {
    v = (-23.0 * f[0] + 21.0 * f[st] + 3.0 * f[2 * st] - f[3 * st]) / 24.0;
  } else {
    const int m = nin - 1;
    v = (23.0 * f[m * st] - 21.0 * f[(m - 1) * st] - 3.0 * f[(m - 2) * st] + f[(m - 3) * st]) / 24.0;
  }
  return v * ih;
}

// E_z += h_tau Z D_x H_y, then -= h_tau Z D_y H_x, at the interior nodes.
__global__ void k_nc_e64(double* __restrict__ ez, const double* __restrict__ hx, const double* __restrict__ hy, int N,
                         double ce, double ih) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i < 1 || j < 1 || i >= N || j >= N) return;
  const double dx = nc_d(hy + (size_t)j * N, 1, i - 1, N, ih);      // H_y row j: N half-node values
  const double dy = nc_d(hx + i, N + 1, j - 1, N, ih);              // H_x column i: N half-node values
  double e = ez[(size_t)j * (N + 1) + i];
  e += ce * dx;
  e -= ce * dy;
  ez[(size_t)j * (N + 1) + i] = e;
}

// H_x -= (h_tau/Z) D_y E_z, H_y += (h_tau/Z) D_x E_z.
__global__ void k_nc_h64(const double* __restrict__ ez, double* __restrict__ hx, double* __restrict__ hy, int N,
                         double ch, double ih) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > N || j > N) return;
  if (j < N && i >= 1 && i < N)  // E_z column i: N+1 node values
    hx[(size_t)j * (N + 1) + i] -= ch * nc_d(ez + i, N + 1, j, N + 1, ih);
  if (i < N && j >= 1 && j < N)  // E_z row j
    hy[(size_t)j * N + i] += ch * nc_d(ez + (size_t)j * (N + 1), 1, i, N + 1, ih);
}

}  // namespace

void launch_nc_e64(double* ez, const double* hx, const double* hy, int N, double c_e, cudaStream_t st) {
  dim3 blk(32, 8);
  dim3 grd((N + 1 + 31) / 32, (N + 1 + 7) / 8);
  k_nc_e64<<<grd, blk, 0, st>>>(ez, hx, hy, N, c_e, (double)N);
}

void launch_nc_h64(const double* ez, double* hx, double* hy, int N, double c_h, cudaStream_t st) {
  dim3 blk(32, 8);
  dim3 grd((N + 1 + 31) / 32, (N + 1 + 7) / 8);
  k_nc_h64<<<grd, blk, 0, st>>>(ez, hx, hy, N, c_h, (double)N);
}

}  // namespace ms
