// FP64 builds of the persistent solvers (Algorithm 2, Algorithm 1), one row per thread.
#include "capi_internal.h"

namespace pbcg {

const void* pipelined_kernel_f64(bool automated, bool scalar, bool vec) {
  if (vec) return pipelined_kernel_f64_vec(scalar);
  if (automated) return (const void*)pbicgstab_kernel<double, true>;
  return scalar ? (const void*)pbicgstab_kernel<double, false, false, true> : (const void*)pbicgstab_kernel<double, false>;
}

const void* classic_kernel_f64(bool scalar) {
  return scalar ? (const void*)classic_kernel<double, true> : (const void*)classic_kernel<double, false>;
}

}  // namespace pbcg
