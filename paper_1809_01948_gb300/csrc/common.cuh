// Device building blocks shared by the p-BiCGStab kernels: sparse matrix views and
// row products (SPMV, Section 1), deterministic block / grid reductions of dot
// products (DOTPR + GLRED), a grid-wide barrier whose wait gives up after a time
// limit, and compensated FP32 accumulation for the mixed-precision dots.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pbcg {

constexpr int kMaxDiag = 16;
constexpr int kMaxThreads = 1024;
constexpr int kMaxDots = 8;

enum DevStatus : int {
  kRunning = -1, kOK = 0, kNotConverged = 4, kBreakdown = 5, kStagnated = 6, kTimeout = 7
};

// ---------------------------------------------------------------- matrices
// A CSR matrix (row_ptr/col int32) or a DIA matrix (ndiag diagonals, diagonal-major
// values, val[d*n + i] = A[i, i+off[d]]).  For the operator A D^{-1} of the Jacobi
// fold, DIA drops its main diagonal (whose exact value is 1) and sets unit_diag.
template <typename V>
struct MatView {
  int fmt;          // 0 CSR, 1 DIA
  int n;
  const int* __restrict__ row_ptr;
  const int* __restrict__ col;
  const V* __restrict__ val;
  int ndiag;
  int unit_diag;    // DIA: add x[i] (exact unit main diagonal) before the stored diagonals
  int off[kMaxDiag];
};

// y_i = sum_j a_ij x_j for one row i, accumulated with FMA in type Acc, stored
// diagonals / columns in ascending order.
template <typename Acc, typename V, typename X>
__device__ __forceinline__ Acc row_dot(const MatView<V>& A, const X* __restrict__ x, int i) {
  Acc acc = Acc(0);
  if (A.fmt == 0) {
    const int e0 = __ldg(A.row_ptr + i), e1 = __ldg(A.row_ptr + i + 1);
    for (int e = e0; e < e1; ++e) {
      acc = fma(Acc(__ldg(A.val + e)), Acc(x[__ldg(A.col + e)]), acc);
    }
  } else {
    if (A.unit_diag) acc = Acc(x[i]);
    const int n = A.n;
#pragma unroll 4
    for (int d = 0; d < A.ndiag; ++d) {
      const int j = i + A.off[d];
      if (j >= 0 && j < n) acc = fma(Acc(__ldg(A.val + (size_t)d * n + i)), Acc(x[j]), acc);
    }
  }
  return acc;
}

// ---------------------------------------------------------------- timing / sync
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier over a co-resident (cooperatively launched) grid.  The counter
// is monotone within a launch: barrier number `epoch` (1, 2, ...) completes when it
// reaches epoch * gridDim.x.  Thread 0 of each block arrives (release) and polls
// (acquire); the poll gives up after timeout_ns and raises *err = kTimeout.
// Returns false when the grid must stop (timeout here or elsewhere).
__device__ __forceinline__ bool grid_barrier(unsigned* counter, unsigned epoch, int* err,
                                             unsigned long long timeout_ns) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    red_release_add(counter, 1u);
    const unsigned target = epoch * gridDim.x;
    const unsigned long long t0 = global_ns();
    unsigned spins = 0;
    while (ld_acquire_u32(counter) < target) {
      if ((++spins & 63u) == 0 && (global_ns() - t0 > timeout_ns || *(volatile int*)err)) {
        atomicCAS(err, 0, (int)kTimeout);
        ok = 0;
        break;
      }
    }
    __threadfence();   // order this block's later plain loads after the other blocks' writes
    if (ok && *(volatile int*)err) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------- reductions
// Block-wide sum of ND doubles per thread, deterministic (fixed shuffle tree, fixed
// warp order).  The result is returned to every thread.  smem: >= 32*ND doubles.
template <int ND>
__device__ __forceinline__ void block_sum(double (&v)[ND], double* smem) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int d = 0; d < ND; ++d) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[d] += __shfl_xor_sync(0xffffffffu, v[d], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int d = 0; d < ND; ++d) smem[d * 32 + wid] = v[d];
  }
  __syncthreads();
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    double s = (lane < nw) ? smem[d * 32 + lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    v[d] = s;
  }
}

// Write this block's ND partial sums to part[blockIdx.x * kMaxDots + d].
template <int ND>
__device__ __forceinline__ void block_publish(double (&v)[ND], double* smem, double* part) {
  block_sum<ND>(v, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int d = 0; d < ND; ++d) part[blockIdx.x * kMaxDots + d] = v[d];
  }
}

// After a grid barrier: every block sums all blocks' partials in the same fixed
// order, so every block obtains bit-identical totals (the GLRED result).
template <int ND>
__device__ __forceinline__ void grid_combine(const double* part, double (&out)[ND], double* smem) {
#pragma unroll
  for (int d = 0; d < ND; ++d) out[d] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int d = 0; d < ND; ++d) out[d] += __ldcg(part + b * kMaxDots + d);
  }
  block_sum<ND>(out, smem);
}

// ---------------------------------------------------------------- dot accumulators
// FP64 accumulation of a*b.
struct DAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double value() const { return s; }
};

// Mixed-precision dot accumulation for FP32 vectors.  Each FP32 product a*b is split
// exactly into p + e (p = fl(a*b), e = fma(a, b, -p)), and p + e is added to an
// unevaluated sum hi + lo of two floats with Knuth's TwoSum (error-free), so the
// per-thread partial carries about 48 significant bits; it is widened to FP64 once
// per thread and all further (block and grid) sums are FP64.  Intrinsics with
// explicit rounding keep the compiler from contracting or reassociating the steps.
struct FAcc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename T> struct AccOf { using type = DAcc; };
template <> struct AccOf<float> { using type = FAcc; };

template <typename T> __device__ __forceinline__ bool finite_d(T v) { return isfinite((double)v); }

}  // namespace pbcg
