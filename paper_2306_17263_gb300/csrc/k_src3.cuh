// Current sources on 3D grids (k_src3.cu): divergence-free driven modes.
#pragma once

#include "grid3d.cuh"

namespace ms {

// Host-side and device data of a grid's 3D sources: per component c the separable tables
// [source q][x values | y values | z values] (sine on node axes, cosine on half-node axes, exact in
// integers) in FP64 and FP32, the spatial coefficient of every (component, source), the driving
// frequencies, and the per-step factors (coefficient x time factor x the units of the right-hand
// side) written by the time kernel.
struct Src3 {
  int nsrc = 0;
  size_t tab_off[6] = {};     // offset of component c's tables in tab / tab32
  double* tab = nullptr;
  float* tab32 = nullptr;
  double* coef = nullptr;     // [6][nsrc]: E: -Z filt a_c; H: filt (curl of the shape)_c
  double* omega = nullptr;    // [nsrc]
  double* fac = nullptr;      // [6][nsrc], FP64 right-hand-side units
  float* fac32 = nullptr;     // [6][nsrc], FP32_REFINED right-hand-side units
};

ms_status src3_set(ms_grid* g, const ms_source3* src, int nsrc);
void src3_free(ms_grid* g);
// Per-step factors for step g->step (read on the device from g->d_step); one tiny launch.
void src3_time(ms_grid* g);
// R (+)= the source term of component c (0..5) in the units of the step's right-hand side:
// FP64 grids: R of Step 1 / Step 2; FP32_REFINED grids: b of the tile solve.
void src3_add(ms_grid* g, int c, void* R);
ms_status exact_driven3(ms_grid* g, const ms_source3* src, int nsrc, double tE, double tH, int c, double* out);

}  // namespace ms
