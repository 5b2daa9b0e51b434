// FP32 path with exact-coefficient refinement and a float-float state (MS_FP32_REFINED).
#pragma once

#include "ms_internal.h"

namespace ms {

ms_status mixed_setup(ms_grid* g);
void mixed_teardown(ms_grid* g);
ms_status step_mixed(ms_grid* g, int* launches);
const char* mixed_last_error();

// FP32 reverse pass of the FP32_REFINED step (adjoint32.cu): float-float adjoint state on the
// device, set up on first use; load / store from and to FP64 device arrays (E_z, H_x, H_y).
struct Adj32;
ms_status adjoint32_setup(ms_grid* g);
void adjoint32_teardown(ms_grid* g);
void adjoint32_load(ms_grid* g, const double* const* l);
void adjoint32_store(ms_grid* g, double* const* l);
ms_status adjoint32_steps(ms_grid* g, long nsteps);

}  // namespace ms
