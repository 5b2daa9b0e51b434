// Separable transform solve of P1 on the tensor cores (k_transform.cu), for 3D FP32_REFINED grids.
#pragma once

#include <cstdint>
#include <string>

#include "grid3d.cuh"

namespace ms {

// Per-grid state of the transform solver: the padded working arrays, the per-axis transform
// matrices of both boundary types in the tensor-core operand layout (forward and transposed, each
// split into bf16 hi + lo), and the eigenvalue tables of -h^2 D_aa.
struct TransformSolver {
  int N = 0;                 // cells per side
  int P = 0;                 // padded transform length (multiple of 128)
  float* w[2] = {};          // P^3 FP32 working arrays
  uint4* q[2][2][2] = {};    // [boundary type DIR / NEU][forward / inverse][hi / lo]
  float* mu[2] = {};         // eigenvalues of -h^2 D_aa per boundary type, P entries (0 on pads)
  int* d_err = nullptr;      // set by a kernel whose bounded wait gave up
};

int ts_setup(int N, TransformSolver* ts, std::string* err);
void ts_free(TransformSolver* ts);
// Launches of one solve, on `st`: x ~ (6 h^2 P1)^{-1} b for the component of shape s (b, x in the
// component's full layout, wall points of x set to zero), d6 = 6 c1 h^2.  Returns the launch count.
int ts_solve(const TransformSolver& ts, const Shape3& s, const float* b, float* x, float d6, cudaStream_t st,
             ms_grid* prof_grid);

}  // namespace ms
