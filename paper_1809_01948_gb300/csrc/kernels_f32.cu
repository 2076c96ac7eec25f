// Mixed-precision builds of the persistent solver (Algorithm 2 with FP32 recurrences), one
// row per thread: the 64-register build and the 40-register streaming build.
#include "capi_internal.h"

namespace pbcg {

const void* pipelined_kernel_f32(bool automated, bool stream, bool scalar, bool vec) {
  if (vec) return pipelined_kernel_f32_vec(scalar, stream);
  if (automated) return (const void*)pbicgstab_kernel<float, true>;
  if (stream)
    return scalar ? (const void*)pbicgstab_kernel<float, false, true, true> : (const void*)pbicgstab_kernel<float, false, true>;
  return scalar ? (const void*)pbicgstab_kernel<float, false, false, true> : (const void*)pbicgstab_kernel<float, false>;
}

}  // namespace pbcg
