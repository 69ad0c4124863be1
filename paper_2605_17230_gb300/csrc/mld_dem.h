// Detector-picture contraction of code-capacity error models (d = 3..9).
#pragma once

#include "mld_internal.h"

namespace mld {

// Device copies of the code tables (made once, guarded like the plan cache).
mld_status ensure_code_device(mld_code* C);

}  // namespace mld
