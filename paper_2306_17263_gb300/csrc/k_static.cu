// ms_p1_solve_static: the FP64 P1 solve without any device allocation.
//
// The regular solve (ms_apply_op with MS_OP_P1SOLVE_*) iterates between two scratch buffers
// that the grid allocates with cudaMalloc.  This variant keeps those two buffers in a
// file-scope __device__ array instead, so a caller that must not allocate device memory can
// still run the solve on its own input and output arrays.  The array is part of the loaded
// module: every GPU that loads this library holds it (MS_STATIC_SCRATCH_BYTES) until exit.
//
// Host code cannot use the array's name as a device address (it names a host-side shadow), so
// the device address is obtained once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on that device.
#include <cmath>
#include <mutex>

#include "k_fp64.cuh"

namespace {

constexpr int kMaxN = MS_STATIC_MAX_N;
constexpr size_t kPlane = (size_t)(kMaxN + 1) * (kMaxN + 1);  // largest field of a kMaxN grid

// Two ping-pong planes of the Richardson iteration.  Every point of a plane is written by a
// sweep before the next sweep reads it, so nothing has to be cleared between calls.
static __device__ __align__(256) double g_p1_scratch[2 * kPlane];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

ms_status fail(ms_status s, const char* msg) {
  ms::set_last_error(msg);
  return s;
}

}  // namespace

extern "C" ms_status ms_p1_solve_static(int n, double r, int field, const double* b, double* x, void* stream) {
  if (n < 4 || n > kMaxN) return fail(MS_EINVAL, "ms_p1_solve_static: n must be in [4, MS_STATIC_MAX_N]");
  if (!(r > 0.0) || !std::isfinite(r)) return fail(MS_EINVAL, "ms_p1_solve_static: r must be positive");
  if (field < 0 || field > 2) return fail(MS_EINVAL, "ms_p1_solve_static: field must be 0 (E_z), 1 (H_x) or 2 (H_y)");
  if (!b || !x || b == x) return fail(MS_EINVAL, "ms_p1_solve_static: b and x must be distinct device arrays");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(MS_ECUDA, "ms_p1_solve_static: no usable current device");
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_p1_scratch);
      if (e != cudaSuccess || !p) return fail(MS_ECUDA, "ms_p1_solve_static: cudaGetSymbolAddress failed");
      g_addr[dev] = (double*)p;
    }
    base = g_addr[dev];
  }
  const ms::Shape s = ms::field_shape(n, field);
  // P~ = h^2 P1 = c1h2 - Lx - Ly - (1/6) Lx Ly, c1h2 = (24/r^2)(1 + 2/r^2), spectrum in
  // [c1h2, c1h2 + 16/3]; the same sweep count, relaxation and kernel as the grid's FP64 solve.
  const double c1h2 = (24.0 / (r * r)) * (1.0 + 2.0 / (r * r));
  const double rho = (16.0 / 3.0) / (2.0 * c1h2 + 16.0 / 3.0);
  int S = (int)std::ceil(std::log(1e-17) / std::log(rho));
  S = S < 1 ? 1 : (S > 64 ? 64 : S);
  const double omega = 2.0 / (2.0 * c1h2 + 16.0 / 3.0);
  const double h2 = 1.0 / ((double)n * n);
  cudaStream_t st = (cudaStream_t)stream;
  double* buf[2] = {base, base + kPlane};
  const double* xin = nullptr;
  for (int k = 0; k < S; ++k) {
    double* xo = (k == S - 1) ? x : buf[k & 1];
    ms::launch_p1_sweep64(b, xin, xo, s, c1h2, omega, h2, k == 0, nullptr, 0.0, st);
    xin = xo;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(MS_ECUDA, "ms_p1_solve_static: kernel launch failed");
  return MS_OK;
}
