// FP32 path with exact-coefficient refinement and a float-float state (MS_FP32_REFINED).
#pragma once

#include "ms_internal.h"

namespace ms {

ms_status mixed_setup(ms_grid* g);
void mixed_teardown(ms_grid* g);
ms_status step_mixed(ms_grid* g, int* launches);
const char* mixed_last_error();

}  // namespace ms
