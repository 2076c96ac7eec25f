// Internal declarations shared by the host translation units of libpbicgstab.
#pragma once
#include <cstdarg>
#include <algorithm>
#include <type_traits>
#include <cuda_runtime.h>
#include "../../include/pbicgstab.h"

namespace pbcg {
pbcg_status set_error(pbcg_status st, const char* fmt, ...);
pbcg_status cuda_status(cudaError_t e, const char* what);
int sm_count();
}  // namespace pbcg
