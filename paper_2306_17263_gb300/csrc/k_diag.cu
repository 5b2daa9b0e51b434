// Diagnostics and state conversion kernels: exact cavity-mode fields, deterministic FP64
// reductions (error norms, energy inner products) and FP64 <-> FP32 hi/lo conversion.
#include "k_fp64.cuh"

namespace ms {

static constexpr int kRedThreads = 256;

int reduce_blocks(size_t n) {
  size_t b = (n + kRedThreads - 1) / kRedThreads;
  if (b > 1024) b = 1024;
  if (b < 1) b = 1;
  return (int)b;
}

// out(i, j) = sum_m coef[m] * tab_x[m][i] * tab_y[m][j]  (separable cavity modes, Eq. "eq:data")
__global__ void k_mode_field(double* __restrict__ out, int nx, int ny, const double* __restrict__ tx,
                             const double* __restrict__ ty, const double* __restrict__ coef, int nmodes) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  double v = 0.0;
  for (int m = 0; m < nmodes; ++m) v = fma(coef[m] * tx[(size_t)m * nx + i], ty[(size_t)m * ny + j], v);
  out[(size_t)j * nx + i] = v;
}

void launch_mode_field(double* out, const Shape& s, const double* tab_x, const double* tab_y, const double* coef,
                       int nmodes, cudaStream_t st) {
  dim3 blk(32, 8), grd((s.nx + 31) / 32, (s.ny + 7) / 8);
  k_mode_field<<<grd, blk, 0, st>>>(out, s.nx, s.ny, tab_x, tab_y, coef, nmodes);
}

// Block tree reduction of NV values per thread (sum, or max for the slots flagged in maxmask).
template <int NV>
__device__ void block_reduce(double (&v)[NV], int maxmask) {
  __shared__ double sh[NV][kRedThreads];
  for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < NV; ++k) {
        double a = sh[k][threadIdx.x], b = sh[k][threadIdx.x + s];
        sh[k][threadIdx.x] = ((maxmask >> k) & 1) ? fmax(a, b) : a + b;
      }
    __syncthreads();
  }
  for (int k = 0; k < NV; ++k) v[k] = sh[k][0];
}

__global__ void k_err_partial(const double* __restrict__ a, const double* __restrict__ b, size_t n,
                              double* __restrict__ partial) {
  double v[4] = {0, 0, 0, 0};
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const double d = a[p] - b[p];
    v[0] += d * d;
    v[1] += b[p] * b[p];
    v[2] = fmax(v[2], fabs(d));
    v[3] += fabs(d);
  }
  block_reduce<4>(v, 0x4);
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) partial[(size_t)blockIdx.x * 4 + k] = v[k];
}

__global__ void k_err_final(const double* __restrict__ partial, int blocks, double* __restrict__ res, int acc) {
  double v[4] = {0, 0, 0, 0};
  for (int p = threadIdx.x; p < blocks; p += blockDim.x) {
    v[0] += partial[(size_t)p * 4 + 0];
    v[1] += partial[(size_t)p * 4 + 1];
    v[2] = fmax(v[2], partial[(size_t)p * 4 + 2]);
    v[3] += partial[(size_t)p * 4 + 3];
  }
  block_reduce<4>(v, 0x4);
  if (threadIdx.x == 0) {
    if (acc) {
      res[0] += v[0];
      res[1] += v[1];
      res[2] = fmax(res[2], v[2]);
      res[3] += v[3];
    } else {
      for (int k = 0; k < 4; ++k) res[k] = v[k];
    }
  }
}

void launch_err_reduce(const double* a, const double* b, size_t n, double* partial, int blocks, double* results,
                       int accumulate, cudaStream_t st) {
  k_err_partial<<<blocks, kRedThreads, 0, st>>>(a, b, n, partial);
  k_err_final<<<1, kRedThreads, 0, st>>>(partial, blocks, results, accumulate);
}

__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b, size_t n,
                              double* __restrict__ partial) {
  double v[1] = {0};
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    v[0] = fma(a[p], b[p], v[0]);
  block_reduce<1>(v, 0);
  if (threadIdx.x == 0) partial[blockIdx.x] = v[0];
}

__global__ void k_dot_final(const double* __restrict__ partial, int blocks, double* __restrict__ res, int slot,
                            int acc) {
  double v[1] = {0};
  for (int p = threadIdx.x; p < blocks; p += blockDim.x) v[0] += partial[p];
  block_reduce<1>(v, 0);
  if (threadIdx.x == 0) res[slot] = acc ? res[slot] + v[0] : v[0];
}

void launch_dot(const double* a, const double* b, size_t n, double* partial, int blocks, double* results, int slot,
                int accumulate, cudaStream_t st) {
  k_dot_partial<<<blocks, kRedThreads, 0, st>>>(a, b, n, partial);
  k_dot_final<<<1, kRedThreads, 0, st>>>(partial, blocks, results, slot, accumulate);
}

// v = hi + lo with hi = fl32(v), lo = fl32(v - hi): the FP32 pair represents v to ~2^-48.
__global__ void k_split(const double* __restrict__ v, float* __restrict__ hi, float* __restrict__ lo, size_t n) {
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x) {
    const double x = v[p];
    const float h = (float)x;
    hi[p] = h;
    lo[p] = (float)(x - (double)h);
  }
}

__global__ void k_join(const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ v, size_t n) {
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (size_t)gridDim.x * blockDim.x)
    v[p] = (double)hi[p] + (double)lo[p];
}

void launch_split(const double* v, float* hi, float* lo, size_t n, cudaStream_t st) {
  k_split<<<reduce_blocks(n), kRedThreads, 0, st>>>(v, hi, lo, n);
}

void launch_join(const float* hi, const float* lo, double* v, size_t n, cudaStream_t st) {
  k_join<<<reduce_blocks(n), kRedThreads, 0, st>>>(hi, lo, v, n);
}

__global__ void k_zero_dirichlet64(double* __restrict__ u, int nx, int ny, int bcx, int bcy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= nx || j >= ny) return;
  if (!interior(bcx, i, nx) || !interior(bcy, j, ny)) u[(size_t)j * nx + i] = 0.0;
}

void launch_zero_dirichlet64(double* u, const Shape& s, cudaStream_t st) {
  dim3 blk(32, 8), grd((s.nx + 31) / 32, (s.ny + 7) / 8);
  k_zero_dirichlet64<<<grd, blk, 0, st>>>(u, s.nx, s.ny, s.bcx, s.bcy);
}

}  // namespace ms
