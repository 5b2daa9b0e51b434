// Three-dimensional grids (six components) behind the same C ABI (grid3d.cu).
#pragma once

#include <vector>

#include "ms_internal.h"

namespace ms {

// One 3D component in the full staggered layout [z][y][x] (Eq. "eq:meshes"): n[a] points and the
// boundary type bc[a] along axis a (Table "tab:bc": Dirichlet on node axes, Neumann on half axes).
struct Shape3 {
  int n[3];
  int bc[3];
  __host__ __device__ size_t size() const { return (size_t)n[0] * n[1] * n[2]; }
};
Shape3 field_shape3(int N, int c);

struct Grid3D;

constexpr int kMaxSweeps3d32 = 8;  // largest Richardson sweep count of the FP32 3D solve

// 3D counterparts of the grid life cycle and state access, dispatched from capi.cu.
ms_status create_grid3d(const ms_grid_desc* d, ms_grid** out);
void destroy_grid3d(ms_grid* g);
ms_status step3d(ms_grid* g);
// comps: 6 arrays (E_x, E_y, E_z, H_x, H_y, H_z); host != 0: host memory, synchronous.
ms_status set_fields3d(ms_grid* g, const double* const* comps, int host);
ms_status get_fields3d(ms_grid* g, double* const* comps, int host);
double stability_limit_3d();
// Diagnostics of a 3D FP64 grid (MS_EUNSUPPORTED for FP32_REFINED grids): the discrete energy and
// the norm of the Pade divergence of H on the cell centres.
ms_status energy3d(ms_grid* g, double* W);
ms_status divergence3d(ms_grid* g, double* norm);
// P1 solver of a 3D FP32_REFINED grid (MS_SOLVER_*); the transform solver's set-up happens on its
// first selection.  transform_solve3d: x ~ (6 h^2 P1)^{-1} b for component c by the transforms alone
// (device FP32 arrays in the component's layout).  transform_status3d: MS_ETIMEOUT if a transform
// kernel gave up a bounded wait since the last check.
ms_status set_solver3d(ms_grid* g, int solver);
ms_status transform_solve3d(ms_grid* g, int c, const float* b, float* x);
ms_status transform_status3d(ms_grid* g);
// out = sum_q coef[q] X_q(i) Y_q(j) Z_q(k) on the unknowns of component c (zero elsewhere), the
// tables given per term as [x values | y values | z values]; synchronous.
ms_status check_sources3(const ms_source3* src, int nsrc, bool need_off_resonance);
ms_status mode_field3_tables(ms_grid* g, int c, const std::vector<double>& tq, const std::vector<double>& coef,
                             double* out);
// Device arrays of the state of a 3D grid: component c has n[c] points in f64[c] (MS_FP64) or in
// hi[c] + lo[c] (MS_FP32_REFINED; the other pointers are NULL).  Returns the component count (6).
int state_arrays3d(ms_grid* g, double** f64, float** hi, float** lo, size_t* n);

}  // namespace ms
