// Tiled FP32_REFINED kernels (k_tiled.cu): curl tile + solve tile per half-step.
#pragma once

#include "ms_internal.h"

namespace ms {

constexpr int kTiledKMax = 12;       // largest Pade band half-width the tiles hold
constexpr int kTiledMaxSweeps = 6;   // largest Richardson sweep count (halo = sweeps - 1)
constexpr int kTiledKFast = 7;       // band half-width of the interior fast path

int tiled_configure();
size_t tiled_curl_smem();
size_t tiled_solve_smem();
// step 0: b0 = Step 1 right-hand side on E_z; step 1: b0, b1 = Step 2 right-hand sides on H_x, H_y.
void tiled_curl(ms_grid* g, int step, float cb_hi, float cb_lo, float* b0, float* b1);
// S sweeps of 6 h^2 P1 x = b and the float-float update (hi, lo) += (s_hi + s_lo) x for 1 or 2 fields.
void tiled_solve(ms_grid* g, int nfields, const int* fields, const float* const* b, int S, float d_hi, float d_lo,
                 float omega, float s_hi, float s_lo);

}  // namespace ms
