// Four-rows-per-thread builds of the persistent solver (structured-stencil storage).
#include "capi_internal.h"

namespace pbcg {

const void* pipelined_kernel_f64_vec(bool scalar) {
  return scalar ? (const void*)pbicgstab_kernel<double, false, false, true, true>
                : (const void*)pbicgstab_kernel<double, false, false, false, true>;
}

const void* pipelined_kernel_f32_vec(bool scalar, bool stream) {
  if (stream)
    return scalar ? (const void*)pbicgstab_kernel<float, false, true, true, true>
                  : (const void*)pbicgstab_kernel<float, false, true, false, true>;
  return scalar ? (const void*)pbicgstab_kernel<float, false, false, true, true>
                : (const void*)pbicgstab_kernel<float, false, false, false, true>;
}

}  // namespace pbcg
