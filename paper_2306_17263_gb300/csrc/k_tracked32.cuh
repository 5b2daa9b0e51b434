// Tracked-Delta-E variant of the FP32_REFINED step (k_tracked32.cu).
#pragma once

#include "ms_internal.h"

namespace ms {

// Delta E_z (float-float) and the scratch planes of the variant; on failure the caller destroys
// the grid, which releases whatever was allocated.
ms_status tracked32_setup(ms_grid* g);
void tracked32_teardown(ms_grid* g);
// DE from an FP64 field on the E_z nodes (split into hi + lo).
void tracked32_set_de(ms_grid* g, const double* de);
// One step: Step 1, the Delta E update of Eq. "eq:mhe", Step 2 with G_E of Eq. "eq:helm2".
ms_status step_mixed_tracked(ms_grid* g, int* nl);

}  // namespace ms
