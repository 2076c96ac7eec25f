// Column max-norms of the error propagation products of Eq. (all_error_matrices):
// U, OU, BA, UEA, BAEA, BPA, UC, BAC, BD, built from the matrices of Eq. (all_matrices)
// for the scalars alpha_i, omega_i, beta_{i+1} that a solve records.
//
// Every matrix is upper triangular and its column j depends on the scalars of the first
// j iterations only, so each product is generated column by column: multiplying a left
// factor X on the right by one of the structured matrices is a recurrence over columns,
//   X U : R_j = R_{j-1} + X_j                 X A : R_j = R_{j-1} - alpha_{j-1} X_{j-1}
//   X B : R_j = beta_j R_{j-1} + X_j          X E : as X B with R_0 = 0
//   X P : R_j = beta_j (R_{j-1} - omega_{j-1} X_{j-1})
//   X C : R_j = R_{j-1} - omega_{j-1} X_{j-1} X D : R_j = R_{j-1} + omega_{j-1} alpha_{j-1} X_{j-1}
// with the left-most factor's columns known in closed form (B_j = beta_j B_{j-1} + e_j,
// U_j = ones on rows 0..j, (O U) gains -omega_{j-1} e_j).  The recurrences act on each row
// separately, so one thread carries one row through all columns (O(m^2) work in total),
// and each column's maximum is reduced per block and merged with one atomic per block.
#include <cstdint>

#include "capi_internal.h"

using namespace pbcg;

namespace {

constexpr int kProducts = 9;          // U OU BA UEA BAEA BPA UC BAC BD
constexpr int kPropThreads = 256;
constexpr int kMaxPropagationIters = 65536;   // O(iters^2) work: about a second at the limit

// Non-negative doubles order like their bit patterns read as unsigned integers.
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void __launch_bounds__(kPropThreads) propagation_norms_kernel(const double* __restrict__ hist, int stride,
                                                                         int m, double* __restrict__ norms) {
  __shared__ double red[kPropThreads / 32][kProducts];
  const int r = blockIdx.x * kPropThreads + threadIdx.x;   // this thread's row
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j0 = blockIdx.x * kPropThreads;                 // rows of this block are zero before column j0
  double B = 0, BA = 0, QUE = 0, UEA = 0, QBAE = 0, BAEA = 0, QBP = 0, BPA = 0, UC = 0, BAC = 0, BD = 0, OU = 0;
  for (int j = j0; j < m; ++j) {
    if (j == 0) {
      B = (r == 0) ? 1.0 : 0.0;        // column 0: B = U = e_0, every other product 0
    } else if (r <= j) {
      const double a = __ldg(hist + (size_t)(j - 1) * stride + 0);   // alpha_{j-1}
      const double w = __ldg(hist + (size_t)(j - 1) * stride + 1);   // omega_{j-1}
      const double b = __ldg(hist + (size_t)(j - 1) * stride + 2);   // beta_j
      const double Uo = (r <= j - 1) ? 1.0 : 0.0;
      const double Bo = B, BAo = BA, QUEo = QUE, QBAEo = QBAE, QBPo = QBP;
      BA = fma(-a, Bo, BA);
      UEA = fma(-a, QUEo, UEA);
      BAEA = fma(-a, QBAEo, BAEA);
      BPA = fma(-a, QBPo, BPA);
      QBP = b * fma(-w, Bo, QBPo);
      UC = fma(-w, Uo, UC);
      BAC = fma(-w, BAo, BAC);
      BD = fma(w * a, Bo, BD);
      B = fma(b, Bo, r == j ? 1.0 : 0.0);
      QUE = fma(b, QUEo, 1.0);                 // r <= j: U_j has a one in this row
      QBAE = fma(b, QBAEo, BA);
      if (r == j) OU = -w;
    }
    double v[kProducts - 1] = {fabs(OU), fabs(BA), fabs(UEA), fabs(BAEA), fabs(BPA), fabs(UC), fabs(BAC), fabs(BD)};
#pragma unroll
    for (int p = 0; p < kProducts - 1; ++p) {
      v[p] = warp_max(v[p]);
      if (lane == 0) red[warp][p] = v[p];
    }
    __syncthreads();
    if (threadIdx.x < kProducts - 1) {
      double mx = 0.0;
#pragma unroll
      for (int q = 0; q < kPropThreads / 32; ++q) mx = fmax(mx, red[q][threadIdx.x]);
      atomic_max_nonneg(norms + (size_t)(threadIdx.x + 1) * m + j, mx);
    } else if (threadIdx.x == kProducts - 1 && blockIdx.x == 0) {
      norms[j] = 1.0;                          // U: ones on and above the diagonal
    }
    __syncthreads();
  }
}

}  // namespace

extern "C" pbcg_status pbicgstab_propagation_norms(const double* hist, int32_t stride, int32_t iters, double* norms,
                                                   void* stream) {
  if (!norms || (!hist && iters > 0))
    return set_error(PBCG_INVALID_ARG, "pbicgstab_propagation_norms needs norms, and hist when iters > 0");
  if (stride < 3) return set_error(PBCG_INVALID_ARG, "stride must be >= 3 doubles");
  if (iters < 0 || iters > kMaxPropagationIters)
    return set_error(PBCG_INVALID_ARG, "iters must be in [0, %d]", (int)kMaxPropagationIters);
  const int m = iters + 1;
  cudaStream_t s = (cudaStream_t)stream;
  pbcg_status st = cuda_status(cudaMemsetAsync(norms, 0, sizeof(double) * kProducts * (size_t)m, s), "memset norms");
  if (st != PBCG_OK) return st;
  const int blocks = (m + kPropThreads - 1) / kPropThreads;
  propagation_norms_kernel<<<blocks, kPropThreads, 0, s>>>(hist, stride, m, norms);
  return cuda_status(cudaGetLastError(), "propagation_norms_kernel");
}
