// Host side of libpbicgstab: argument validation, matrix preparation, workspace,
// cooperative launch of the persistent solver, FP64 true residual.  C ABI in
// include/pbicgstab.h.
#include <cmath>
#include <type_traits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cstdint>
#include <new>
#include <string>

#include "../../include/pbicgstab.h"
#include "capi_internal.h"

using namespace pbcg;

namespace pbcg {
thread_local std::string g_last_error;

pbcg_status set_error(pbcg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

pbcg_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PBCG_OK;
  cudaGetLastError();  // clear sticky-free errors
  if (e == cudaErrorMemoryAllocation)
    return set_error(PBCG_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
  return set_error(PBCG_CUDA_ERROR, "%s: %s", what, cudaGetErrorString(e));
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}
}  // namespace pbcg

int l2_bytes() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev);
  return v > 0 ? v : 0;
}

#define CK(call, what)                                   \
  do {                                                   \
    pbcg_status st__ = cuda_status((call), (what));      \
    if (st__ != PBCG_OK) return st__;                    \
  } while (0)

// ----------------------------------------------------------------------------
// preparation kernels
// ----------------------------------------------------------------------------
// flags: bit0 row_ptr not monotone / wrong ends, bit1 column out of range or not
// increasing, bit2 non-finite value, bit3 missing or zero diagonal (when required)
__global__ void validate_csr_kernel(int n, long long nnz, const int* row_ptr, const int* col,
                                    const void* val, int f32, int need_diag, int* flags, double* diag,
                                    int* bandwidth, int* maxnnz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = 0;
  const int e0 = row_ptr[i], e1 = row_ptr[i + 1];
  if (i == 0 && e0 != 0) f |= 1;
  if (i == n - 1 && (long long)e1 != nnz) f |= 1;
  if (e1 < e0 || e0 < 0 || (long long)e1 > nnz) {
    atomicOr(flags, f | 1);
    return;
  }
  double dg = 0.0;
  int prev = -1, bw = 0;
  for (int e = e0; e < e1; ++e) {
    const int c = col[e];
    if (c < 0 || c >= n || c <= prev) f |= 2;
    prev = c;
    bw = max(bw, abs(c - i));
    const double v = f32 ? (double)((const float*)val)[e] : ((const double*)val)[e];
    if (!isfinite(v)) f |= 4;
    if (c == i) dg = v;
  }
  if (need_diag && dg == 0.0) f |= 8;
  diag[i] = dg;
  if (bw) atomicMax(bandwidth, bw);
  atomicMax(maxnnz, e1 - e0);
  if (f) atomicOr(flags, f);
}

// Constants of the error bounds (automated replacement).  Non-negative doubles are
// compared through their bit patterns, and column sums are accumulated in fixed point
// (each |a_ij| rounded up to a multiple of maxabs * 2^-40) with integer atomics, so the
// results do not depend on the order of the atomic operations.
// Warp-wide maximum, then one atomic per warp (a single global address would otherwise
// serialise an atomic per element).
__device__ __forceinline__ void warp_atomic_max(unsigned long long* addr, unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  if ((threadIdx.x & 31) == 0 && v) atomicMax(addr, v);
}

__global__ void absmax_kernel(MatView<double> A, long long nval, unsigned long long* bits) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const double v = e < nval ? fabs(A.val[e]) : 0.0;
  warp_atomic_max(bits, v > 0.0 ? (unsigned long long)__double_as_longlong(v) : 0ull);
}

__global__ void row_col_sums_kernel(MatView<double> A, const unsigned long long* maxabs_bits, unsigned long long* rowmax_bits,
                                    unsigned long long* colsum) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double maxabs = __longlong_as_double((long long)*maxabs_bits);
  if (!(maxabs > 0.0)) return;   // uniform across the grid
  const double scale = 1099511627776.0 / maxabs;   // 2^40 / maxabs
  double rs = 0.0;
  if (i >= A.n) {
  } else if (A.fmt == 0) {
    for (int e = A.row_ptr[i]; e < A.row_ptr[i + 1]; ++e) {
      const double a = fabs(A.val[e]);
      rs += a;
      atomicAdd(colsum + A.col[e], (unsigned long long)ceil(a * scale));
    }
  } else {
    for (int d = 0; d < A.ndiag; ++d) {
      const int j = i + A.off[d];
      if (j < 0 || j >= A.n) continue;
      const double a = fabs(A.val[(size_t)d * A.n + i]);
      rs += a;
      atomicAdd(colsum + j, (unsigned long long)ceil(a * scale));
    }
  }
  warp_atomic_max(rowmax_bits, (unsigned long long)__double_as_longlong(rs));
}

__global__ void max_u64_kernel(int n, const unsigned long long* v, unsigned long long* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  warp_atomic_max(out, i < n ? v[i] : 0ull);
}

// Smallest and largest diagonal entry as order-preserving integer images (warp-reduced).
__device__ __forceinline__ unsigned long long ordered_u64(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void diag_range_kernel(int n, const double* diag, unsigned long long* range) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long lo = ~0ull, hi = 0ull;
  if (i < n) lo = hi = ordered_u64(diag[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o), b = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = b > hi ? b : hi;
  }
  if ((threadIdx.x & 31) == 0) {
    if (lo != ~0ull) atomicMin(range, lo);
    if (hi != 0ull) atomicMax(range + 1, hi);
  }
}

template <typename T>
__global__ void dinv_max_kernel(int n, const T* dinv, unsigned long long* bits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  warp_atomic_max(bits, i < n ? (unsigned long long)__double_as_longlong(fabs((double)dinv[i])) : 0ull);
}

__global__ void validate_dia_kernel(int n, int ndiag, MatView<double> offs_only, const void* val, int f32,
                                    int need_diag, int* flags, double* diag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = 0;
  double dg = 0.0;
  for (int d = 0; d < ndiag; ++d) {
    const size_t idx = (size_t)d * n + i;
    const double v = f32 ? (double)((const float*)val)[idx] : ((const double*)val)[idx];
    const int j = i + offs_only.off[d];
    if (j < 0 || j >= n) continue;
    if (!isfinite(v)) f |= 4;
    if (offs_only.off[d] == 0) dg = v;
  }
  if (need_diag && dg == 0.0) f |= 8;
  diag[i] = dg;
  if (f) atomicOr(flags, f);
}

__global__ void to_f64_kernel(long long m, const void* src, int f32, double* dst) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= m) return;
  dst[i] = f32 ? (double)((const float*)src)[i] : ((const double*)src)[i];
}

template <typename T>
__global__ void cast_kernel(long long m, const double* src, T* dst) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < m) dst[i] = T(src[i]);
}

__global__ void dinv_kernel(int n, const double* diag, double* dinv64) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dinv64[i] = 1.0 / diag[i];
}

// A D^{-1}: column j scaled by d_inv[j], rounded once to T.
template <typename T>
__global__ void fold_csr_kernel(int n, const int* row_ptr, const int* col, const double* val,
                                const double* dinv, T* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) out[e] = T(val[e] * dinv[col[e]]);
}

// DIA fold: the main diagonal of A D^{-1} is exactly 1 and is not stored
// (MatView::unit_diag); the other diagonals are scaled by d_inv of their column.
template <typename T>
__global__ void fold_dia_kernel(int n, MatView<double> src, const double* dinv, T* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int dd = 0;
  for (int d = 0; d < src.ndiag; ++d) {
    if (src.off[d] == 0) continue;
    const int j = i + src.off[d];
    const double v = src.val[(size_t)d * n + i];
    out[(size_t)dd * n + i] = (j >= 0 && j < n) ? T(v * dinv[j]) : T(0);
    ++dd;
  }
}

// FP64 ||b - A x||^2 and ||b||^2, block partials then one fixed-order final sum.
__global__ void true_res_partial_kernel(MatView<double> A, const double* b, const double* x, double* part) {
  __shared__ double smem[kWork + kMaxDots];
  double v[2] = {0.0, 0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
    const double r = b[i] - row_dot<double>(A, x, i);
    v[0] = fma(r, r, v[0]);
    v[1] = fma(b[i], b[i], v[1]);
  }
  block_publish<2>(v, smem, part, blockIdx.x);
}

__global__ void true_res_final_kernel(const double* part, int nparts, double* out) {
  __shared__ double smem[kWork + kMaxDots];
  double v[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
    v[0] += part[b * kMaxDots + 0];
    v[1] += part[b * kMaxDots + 1];
  }
  block_sum<2>(v, smem);
  if (threadIdx.x == 0) out[0] = v[1] > 0.0 ? sqrt(v[0]) / sqrt(v[1]) : sqrt(v[0]);
}

__global__ void spmv_kernel(MatView<double> A, const double* x, double* y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x)
    y[i] = row_dot<double>(A, x, i);
}

// Test hook: every block waits for gridDim.x + extra arrivals, which never come.
__global__ void barrier_timeout_kernel(unsigned* counter, int* err, int extra, unsigned long long timeout_ns) {
  __syncthreads();
  if (threadIdx.x == 0) {
    red_release_add(counter, 1u);
    const unsigned target = gridDim.x + (unsigned)extra;
    const unsigned long long t0 = global_ns();
    unsigned spins = 0;
    while (ld_acquire_u32(counter) < target) {
      if ((++spins & 63u) == 0 && global_ns() - t0 > timeout_ns) {
        atomicCAS(err, 0, (int)kTimeout);
        break;
      }
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------
// context
// ----------------------------------------------------------------------------
static void free_ctx(pbcg_ctx* c) {
  if (!c) return;
  if (c->valAu && c->valAu != (void*)c->val64) cudaFree(c->valAu);
  void* ptrs[] = {c->row_ptr, c->col, c->val64, c->valAt, c->diag64, c->dinv64, c->dinvT, c->st_mask,
                  c->vecs, c->part, c->dstate, c->multi_vecs, c->multi_part, c->multi_state, c->multi_params,
                  c->xbest, c->tperm};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->hstate) cudaFreeHost(c->hstate);
  if (c->multi_hstate) cudaFreeHost(c->multi_hstate);
  if (c->multi_hparams) cudaFreeHost(c->multi_hparams);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

pbcg_status check_options(const pbcg_options* o, long long n) {
  if (o->precision != PBCG_FP64 && o->precision != PBCG_MIXED)
    return set_error(PBCG_INVALID_ARG, "options.precision must be PBCG_FP64 or PBCG_MIXED");
  if (o->max_it < 0) return set_error(PBCG_INVALID_ARG, "options.max_it must be >= 0");
  if (!(o->tol >= 0.0) || !std::isfinite(o->tol)) return set_error(PBCG_INVALID_ARG, "options.tol must be finite and >= 0");
  if (o->rr_period < 0) return set_error(PBCG_INVALID_ARG, "options.rr_period must be >= 0");
  if (o->rr_auto != 0 && o->rr_auto != 1) return set_error(PBCG_INVALID_ARG, "options.rr_auto must be 0 or 1");
  if (!(o->rr_tau >= 0.0) || !std::isfinite(o->rr_tau)) return set_error(PBCG_INVALID_ARG, "options.rr_tau must be >= 0");
  if (!(o->rr_theta >= 0.0 && o->rr_theta < 1.0)) return set_error(PBCG_INVALID_ARG, "options.rr_theta must be in [0, 1)");
  if (o->record_iterates < 0 || (o->record_iterates > 0 && !o->hist_x))
    return set_error(PBCG_INVALID_ARG, "options.record_iterates > 0 needs hist_x");
  if (o->hist_len < 0 || (o->hist_len > 0 && !o->hist_scalars))
    return set_error(PBCG_INVALID_ARG, "options.hist_len > 0 needs hist_scalars");
  if (o->block_threads != 0 && (o->block_threads < 32 || o->block_threads > kMaxThreads || o->block_threads % 32))
    return set_error(PBCG_INVALID_ARG, "options.block_threads must be 0 or a multiple of 32 in [32, 1024]");
  if (o->grid_blocks < 0) return set_error(PBCG_INVALID_ARG, "options.grid_blocks must be >= 0");
  if (o->max_restarts < 0 || o->max_restarts > 1000) return set_error(PBCG_INVALID_ARG, "options.max_restarts must be in [0, 1000]");
  if (o->operator_storage != PBCG_STORAGE_AUTO && o->operator_storage != PBCG_STORAGE_GENERAL)
    return set_error(PBCG_INVALID_ARG, "options.operator_storage must be PBCG_STORAGE_AUTO or PBCG_STORAGE_GENERAL");
  if (o->method != PBCG_PIPELINED && o->method != PBCG_CLASSIC)
    return set_error(PBCG_INVALID_ARG, "options.method must be PBCG_PIPELINED or PBCG_CLASSIC");
  if (o->restart_period < 0) return set_error(PBCG_INVALID_ARG, "options.restart_period must be >= 0");
  if (o->stag_window < 0) return set_error(PBCG_INVALID_ARG, "options.stag_window must be >= 0");
  if (!(o->rr_cutoff >= 0.0 && o->rr_cutoff < 1.0))
    return set_error(PBCG_INVALID_ARG, "options.rr_cutoff must be in [0, 1)");
  if (o->prefetch_trips > 16) return set_error(PBCG_INVALID_ARG, "options.prefetch_trips must be at most 16");
  if (o->method == PBCG_CLASSIC) {
    if (o->precision != PBCG_FP64) return set_error(PBCG_INVALID_ARG, "PBCG_CLASSIC runs in PBCG_FP64 only");
    if (o->rr_period != 0 || o->rr_theta != 0.0 || o->rr_auto != 0 || o->max_restarts != 0 ||
        o->restart_period != 0 || o->stag_window != 0)
      return set_error(PBCG_INVALID_ARG, "PBCG_CLASSIC takes no replacement or restart policy and no restarts");
  }
  (void)n;
  return PBCG_OK;
}

// Preconditioners each method's kernels apply.
static pbcg_status check_method_precond(const pbcg_options* o, int prec_kind) {
  if (o->rr_auto && prec_kind == PBCG_PREC_NEUMANN)
    return set_error(PBCG_INVALID_ARG, "automated replacement (rr_auto) supports no or Jacobi preconditioning");
  if (o->method == PBCG_CLASSIC && prec_kind == PBCG_PREC_NEUMANN)
    return set_error(PBCG_INVALID_ARG, "PBCG_CLASSIC supports no or Jacobi preconditioning");
  return PBCG_OK;
}

// The mixed solver streams from DRAM (STREAM build, 512-thread blocks) when its working set
// exceeds L2; everything else uses the 1024-thread build.
static bool streaming(const pbcg_ctx* c) {
  return c->precision == PBCG_MIXED && !c->opt.rr_auto && c->opt.method == PBCG_PIPELINED &&
         hot_bytes(c) > (double)l2_bytes();
}

// Four rows per thread in the hot passes (VEC kernels): stencil storage of a system whose
// row count is a multiple of 4, Algorithm 2 without the automated policy, b, x and the
// iterate history 16-byte aligned (the quads move as 128-bit accesses), and a block size
// the kernels' 128-register budget allows (0 = their default, or at most 512 threads).
bool quad_rows(const pbcg_ctx* c, const double* b, const double* x) {
  const auto al = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
  return c->stencil && c->n % 4 == 0 && !c->opt.rr_auto && c->opt.method == PBCG_PIPELINED && al(b) && al(x) &&
         (c->opt.record_iterates == 0 || al(c->opt.hist_x)) &&
         c->opt.block_threads <= (streaming(c) ? pbcg::SolverLaunch<float, true, true>::kThreads
                                               : pbcg::SolverLaunch<double, false, true>::kThreads);
}

template <typename T>
static const void* kernel_ptr(const pbcg_ctx* c, bool vec) {
  const pbcg_options& o = c->opt;
  const bool sc = scalar_jacobi(c);
  if constexpr (std::is_same<T, double>::value) {
    if (o.method == PBCG_CLASSIC) return classic_kernel_f64(sc);
    return pipelined_kernel_f64(o.rr_auto != 0, sc, vec);
  } else {
    return pipelined_kernel_f32(o.rr_auto != 0, streaming(c), sc, vec);
  }
}

// Default shape: the solver kernels' register budgets (SolverLaunch): one 1024-thread block
// per SM (measured faster than two 512-thread blocks on the 2D and 3D convection-diffusion
// systems: fewer blocks at each grid barrier and reduction), three 512-thread blocks per
// SM for the streaming mixed build, two 512-thread blocks for the four-row kernels.
static int kernel_threads(const pbcg_ctx* c, bool vec) {
  if (c->opt.block_threads) return c->opt.block_threads;
  if (vec)
    return streaming(c) ? pbcg::SolverLaunch<float, true, true>::kThreads : pbcg::SolverLaunch<double, false, true>::kThreads;
  return streaming(c) ? pbcg::SolverLaunch<float, true>::kThreads : pbcg::SolverLaunch<double, false>::kThreads;
}

// Dynamic shared memory of the staged Neumann sweeps (options.staged_sweeps): two stages
// of the layout stage_layout gives for a block's 8 x threads rows; 0 where they do not
// apply (another kernel build, an offset the layout cannot stage, or no room beside the
// kernel's static shared memory).  Automatic: where a sweep's operands (three FP32 vectors
// and the masks, 14 bytes per row) exceed L2 — measured 12% faster per sweep on the 3D
// 256^3 system, slower where the sweep's vectors stay in L2 (3D 160^3).
size_t staged_bytes(const pbcg_ctx* c, int threads, bool vec) {
  if (c->opt.staged_sweeps < 0 || !vec || c->precision != PBCG_MIXED || c->prec_kind != PBCG_PREC_NEUMANN ||
      !c->stencil || threads % 32 != 0)
    return 0;
  if (c->opt.staged_sweeps == 0 && 14.0 * (double)c->n <= (double)l2_bytes()) return 0;
  const pbcg::MatView<float> v = make_stencil_view<float>(c, false);
  pbcg::StageLayout L;
  pbcg::stage_layout(L, v.off, v.ndiag, 8 * threads);
  if (!L.ok) return 0;
  const size_t bytes = (size_t)2 * (size_t)L.stage_f * sizeof(float);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel_ptr<float>(c, vec)) != cudaSuccess) return 0;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return fa.sharedSizeBytes + bytes <= (size_t)optin ? bytes : 0;
}

pbcg_status launch_shape(const pbcg_ctx* c, int* grid, int* threads, bool vec) {
  const int nt = kernel_threads(c, vec);
  int per_sm = 0;
  const void* k = c->precision == PBCG_MIXED ? kernel_ptr<float>(c, vec) : kernel_ptr<double>(c, vec);
  cudaFuncAttributes fa;
  CK(cudaFuncGetAttributes(&fa, k), "kernel attributes");
  if (nt > fa.maxThreadsPerBlock)
    return set_error(PBCG_INVALID_ARG, "block_threads %d above this solver's limit of %d", nt, fa.maxThreadsPerBlock);
  const size_t dyn = staged_bytes(c, nt, vec);
  if (dyn > 0)
    CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn), "shared memory attribute");
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, dyn), "occupancy query");
  const int sms = sm_count();
  const int max_coresident = per_sm * sms;
  if (max_coresident <= 0) return set_error(PBCG_INVALID_ARG, "kernel cannot be resident with %d threads per block", nt);
  int g = c->opt.grid_blocks;
  if (g == 0) {
    // every co-resident block slot busy, but at least 32 rows per block
    const long long want = (c->n + 31) / 32;
    g = (int)std::min<long long>(std::max<long long>(1, want), (long long)max_coresident);
  }
  if (g > max_coresident)
    return set_error(PBCG_INVALID_ARG, "grid_blocks %d exceeds the %d co-resident blocks", g, max_coresident);
  if (g > c->max_blocks) return set_error(PBCG_INVALID_ARG, "grid_blocks %d exceeds workspace (%d)", g, c->max_blocks);
  *grid = g;
  *threads = nt;
  return PBCG_OK;
}

extern "C" pbcg_status pbicgstab_default_options(pbcg_options* o) {
  if (!o) return set_error(PBCG_INVALID_ARG, "opt is NULL");
  memset(o, 0, sizeof *o);
  o->precision = PBCG_FP64;
  o->max_it = 10000;
  o->tol = 1e-10;
  o->timeout_ms = 2000.0;
  return PBCG_OK;
}

extern "C" const char* pbicgstab_last_error(void) { return g_last_error.c_str(); }

// copy_pattern: copy A's CSR row pointers and columns (create); false: A's pattern is the
// context's own (pbicgstab_update_values), only the values are new.
static pbcg_status prepare_matrix(pbcg_ctx* c, const pbcg_matrix* A, bool copy_pattern = true) {
  const int n = c->n;
  const int nb = (n + 255) / 256;
  const int f32 = A->val_dtype == PBCG_F32;
  const bool need_diag = c->prec_kind != PBCG_PREC_NONE;
  int* dflags = &c->dstate->flags;
  CK(cudaMemsetAsync(dflags, 0, sizeof(int), c->stream), "memset");
  CK(cudaMalloc(&c->diag64, sizeof(double) * n), "cudaMalloc diag");
  long long nval;
  if (c->fmt == PBCG_FMT_CSR) {
    nval = c->nnz;
    if (copy_pattern) {
      CK(cudaMalloc(&c->row_ptr, sizeof(int) * (n + 1)), "cudaMalloc row_ptr");
      CK(cudaMalloc(&c->col, sizeof(int) * std::max<long long>(1, c->nnz)), "cudaMalloc col");
      CK(cudaMemcpyAsync(c->row_ptr, A->row_ptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, c->stream),
         "copy row_ptr");
      if (c->nnz)
        CK(cudaMemcpyAsync(c->col, A->col, sizeof(int) * c->nnz, cudaMemcpyDeviceToDevice, c->stream), "copy col");
    }
    CK(cudaMemsetAsync(&c->dstate->reserved, 0, 2 * sizeof(int), c->stream), "memset");
    validate_csr_kernel<<<nb, 256, 0, c->stream>>>(n, c->nnz, c->row_ptr, c->col, A->val, f32, need_diag, dflags, c->diag64,
                                                    &c->dstate->reserved, &c->dstate->maxnnz);
    CK(cudaGetLastError(), "validate kernel launch");
  } else {
    nval = (long long)c->ndiag * n;
    MatView<double> offs;
    memset(&offs, 0, sizeof offs);
    for (int d = 0; d < c->ndiag; ++d) offs.off[d] = c->offsets[d];
    validate_dia_kernel<<<nb, 256, 0, c->stream>>>(n, c->ndiag, offs, A->val, f32, need_diag, dflags, c->diag64);
  }
  CK(cudaGetLastError(), "validate kernel");
  CK(cudaMalloc(&c->val64, sizeof(double) * std::max<long long>(1, nval)), "cudaMalloc values");
  const long long nbv = (nval + 255) / 256;
  if (nval) to_f64_kernel<<<(unsigned)nbv, 256, 0, c->stream>>>(nval, A->val, f32, c->val64);
  CK(cudaGetLastError(), "convert kernel");
  int hflags = 0, hbw[2] = {0, 0};
  CK(cudaMemcpyAsync(&hflags, dflags, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "copy flags");
  if (c->fmt == PBCG_FMT_CSR)
    CK(cudaMemcpyAsync(hbw, &c->dstate->reserved, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream), "copy bandwidth");
  CK(cudaStreamSynchronize(c->stream), "validate");
  if (c->fmt == PBCG_FMT_CSR) {
    c->bandwidth = hbw[0];
    c->maxnnz = hbw[1];
  } else {
    for (int d = 0; d < c->ndiag; ++d) c->bandwidth = std::max(c->bandwidth, std::abs(c->offsets[d]));
    c->maxnnz = c->ndiag;
  }
  if (hflags & 1) return set_error(PBCG_INVALID_ARG, "CSR row_ptr is not monotone from 0 to nnz");
  if (hflags & 2) return set_error(PBCG_INVALID_ARG, "CSR column index out of range or not strictly increasing in a row");
  if (hflags & 4) return set_error(PBCG_INVALID_ARG, "matrix has a non-finite value");
  if (hflags & 8) return set_error(PBCG_INVALID_ARG, "the preconditioner needs a non-zero diagonal entry in every row");

  const size_t es = elem_size(c->precision);
  const bool mixed = c->precision == PBCG_MIXED;
  if (need_diag) {
    // a constant diagonal makes Jacobi a scalar preconditioner (the SCALAR kernel builds)
    unsigned long long* rng = nullptr;
    CK(cudaMalloc(&rng, 2 * sizeof(unsigned long long)), "cudaMalloc");
    const unsigned long long init[2] = {~0ull, 0ull};
    CK(cudaMemcpyAsync(rng, init, sizeof init, cudaMemcpyHostToDevice, c->stream), "copy");
    diag_range_kernel<<<nb, 256, 0, c->stream>>>(n, c->diag64, rng);
    unsigned long long hr[2];
    CK(cudaMemcpyAsync(hr, rng, sizeof hr, cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "diagonal range");
    cudaFree(rng);
    if (hr[0] == hr[1]) {
      const unsigned long long u = (hr[0] >> 63) ? (hr[0] & 0x7fffffffffffffffull) : ~hr[0];
      double d;
      memcpy(&d, &u, sizeof d);
      c->dconst = 1;
      c->dconst_inv = 1.0 / d;
    }
    CK(cudaMalloc(&c->dinv64, sizeof(double) * n), "cudaMalloc dinv");
    dinv_kernel<<<nb, 256, 0, c->stream>>>(n, c->diag64, c->dinv64);
    if (mixed) {
      CK(cudaMalloc(&c->dinvT, sizeof(float) * n), "cudaMalloc dinv32");
      cast_kernel<float><<<nb, 256, 0, c->stream>>>(n, c->dinv64, (float*)c->dinvT);
    } else {
      c->dinvT = nullptr;
    }
  }
  // unfolded A in T
  if (mixed) {
    CK(cudaMalloc(&c->valAu, sizeof(float) * std::max<long long>(1, nval)), "cudaMalloc A32");
    if (nval) cast_kernel<float><<<(unsigned)nbv, 256, 0, c->stream>>>(nval, c->val64, (float*)c->valAu);
  } else {
    c->valAu = c->val64;
  }
  // hot operator: A D^{-1} with a preconditioner, A otherwise
  if (!need_diag) {
    c->valAt = nullptr;
    c->ndiag_t = c->ndiag;
    for (int d = 0; d < c->ndiag; ++d) c->offsets_t[d] = c->offsets[d];
    c->at_unit_diag = 0;
  } else if (c->fmt == PBCG_FMT_CSR) {
    CK(cudaMalloc(&c->valAt, es * std::max<long long>(1, nval)), "cudaMalloc A D^-1");
    if (mixed) fold_csr_kernel<float><<<nb, 256, 0, c->stream>>>(n, c->row_ptr, c->col, c->val64, c->dinv64, (float*)c->valAt);
    else fold_csr_kernel<double><<<nb, 256, 0, c->stream>>>(n, c->row_ptr, c->col, c->val64, c->dinv64, (double*)c->valAt);
  } else {
    int dd = 0;
    for (int d = 0; d < c->ndiag; ++d)
      if (c->offsets[d] != 0) c->offsets_t[dd++] = c->offsets[d];
    c->ndiag_t = dd;
    c->at_unit_diag = 1;
    CK(cudaMalloc(&c->valAt, es * std::max<long long>(1, (long long)dd * n)), "cudaMalloc A D^-1");
    MatView<double> src = make_view<double>(c, c->val64, false);
    if (mixed) fold_dia_kernel<float><<<nb, 256, 0, c->stream>>>(n, src, c->dinv64, (float*)c->valAt);
    else fold_dia_kernel<double><<<nb, 256, 0, c->stream>>>(n, src, c->dinv64, (double*)c->valAt);
  }
  CK(cudaGetLastError(), "prepare kernels");
  // constants of the error bounds: sqrt(||A||_1 ||A||_inf) and max |d_inv|
  {
    unsigned long long* colsum = nullptr;
    CK(cudaMalloc(&colsum, sizeof(unsigned long long) * n), "cudaMalloc column sums");
    CK(cudaMemsetAsync(colsum, 0, sizeof(unsigned long long) * n, c->stream), "memset");
    CK(cudaMemsetAsync(&c->dstate->maxabs_bits, 0, 4 * sizeof(unsigned long long), c->stream), "memset");
    MatView<double> A64v = make_view<double>(c, c->val64, false);
    if (nval) absmax_kernel<<<(unsigned)nbv, 256, 0, c->stream>>>(A64v, nval, &c->dstate->maxabs_bits);
    row_col_sums_kernel<<<nb, 256, 0, c->stream>>>(A64v, &c->dstate->maxabs_bits, &c->dstate->rowsum_bits, colsum);
    max_u64_kernel<<<nb, 256, 0, c->stream>>>(n, colsum, &c->dstate->colsum_max);
    if (need_diag) {
      if (mixed) dinv_max_kernel<float><<<nb, 256, 0, c->stream>>>(n, (const float*)c->dinvT, &c->dstate->dinv_bits);
      else dinv_max_kernel<double><<<nb, 256, 0, c->stream>>>(n, c->dinv64, &c->dstate->dinv_bits);
    }
    unsigned long long hb[4] = {0, 0, 0, 0};
    CK(cudaGetLastError(), "bound constant kernels");
    CK(cudaMemcpyAsync(hb, &c->dstate->maxabs_bits, sizeof hb, cudaMemcpyDeviceToHost, c->stream), "copy");
    CK(cudaStreamSynchronize(c->stream), "bound constants");
    cudaFree(colsum);
    double maxabs, rowmax, dmax;
    memcpy(&maxabs, &hb[0], 8);
    memcpy(&rowmax, &hb[1], 8);
    memcpy(&dmax, &hb[3], 8);
    const double colmax = (double)hb[2] * (maxabs / 1099511627776.0);
    c->norm_bound = std::sqrt(colmax * rowmax);
    c->dinv_max = need_diag ? dmax : 1.0;
  }
  if (c->opt.operator_storage == PBCG_STORAGE_AUTO) return build_stencil(c);
  return PBCG_OK;
}

extern "C" pbcg_status pbicgstab_create(pbcg_ctx** out, const pbcg_matrix* A, const pbcg_precond* M,
                                        const pbcg_options* opt, void* stream) {
  if (!out || !A || !M || !opt) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_create");
  *out = nullptr;
  if (A->n <= 0 || A->n > PBCG_MAX_ROWS) return set_error(PBCG_INVALID_ARG, "n must be in [1, 2^30]");
  if (A->format != PBCG_FMT_CSR && A->format != PBCG_FMT_DIA) return set_error(PBCG_INVALID_ARG, "unknown matrix format");
  if (A->val_dtype != PBCG_F64 && A->val_dtype != PBCG_F32) return set_error(PBCG_INVALID_ARG, "unknown value dtype");
  if (!A->val) return set_error(PBCG_INVALID_ARG, "matrix values are NULL");
  if (A->format == PBCG_FMT_CSR) {
    if (!A->row_ptr || (A->nnz > 0 && !A->col)) return set_error(PBCG_INVALID_ARG, "CSR arrays are NULL");
    if (A->nnz < 0 || A->nnz >= 2147483647LL) return set_error(PBCG_INVALID_ARG, "nnz must be in [0, 2^31-2]");
  } else {
    if (A->ndiag < 1 || A->ndiag > kMaxDiag || !A->offsets)
      return set_error(PBCG_INVALID_ARG, "DIA needs 1..%d diagonals and host offsets", kMaxDiag);
    bool has0 = false;
    for (int d = 0; d < A->ndiag; ++d) {
      if (d > 0 && A->offsets[d] <= A->offsets[d - 1]) return set_error(PBCG_INVALID_ARG, "DIA offsets must increase");
      if (A->offsets[d] <= -A->n || A->offsets[d] >= A->n) return set_error(PBCG_INVALID_ARG, "DIA offset out of range");
      has0 |= A->offsets[d] == 0;
    }
    if (!has0) return set_error(PBCG_INVALID_ARG, "DIA offsets must contain the main diagonal 0");
  }
  if (M->kind < PBCG_PREC_NONE || M->kind > PBCG_PREC_NEUMANN) return set_error(PBCG_INVALID_ARG, "unknown preconditioner");
  if (M->kind == PBCG_PREC_NEUMANN && (M->degree < 1 || M->degree > 8))
    return set_error(PBCG_INVALID_ARG, "Neumann degree must be in [1, 8]");
  pbcg_status st = check_options(opt, A->n);
  if (st != PBCG_OK) return st;
  st = check_method_precond(opt, M->kind);
  if (st != PBCG_OK) return st;

  pbcg_ctx* c = new (std::nothrow) pbcg_ctx();
  if (!c) return set_error(PBCG_OUT_OF_MEMORY, "host allocation failed");
  c->n = (int)A->n;
  c->nnz = A->format == PBCG_FMT_CSR ? A->nnz : 0;
  c->fmt = A->format;
  c->precision = opt->precision;
  c->prec_kind = M->kind;
  c->degree = M->kind == PBCG_PREC_NEUMANN ? M->degree : 0;
  c->stream = (cudaStream_t)stream;
  c->opt = *opt;
  c->ndiag = A->format == PBCG_FMT_DIA ? A->ndiag : 0;
  for (int d = 0; d < c->ndiag; ++d) c->offsets[d] = A->offsets[d];
#define CKC(call, what)                                  \
  do {                                                   \
    pbcg_status s__ = cuda_status((call), (what));       \
    if (s__ != PBCG_OK) { free_ctx(c); return s__; }     \
  } while (0)
  CKC(cudaMalloc(&c->dstate, sizeof(DevState)), "cudaMalloc state");
  CKC(cudaMallocHost(&c->hstate, sizeof(DevState)), "cudaMallocHost state");
  CKC(cudaEventCreate(&c->ev0), "event");
  CKC(cudaEventCreate(&c->ev1), "event");
  st = prepare_matrix(c, A);
  if (st != PBCG_OK) { free_ctx(c); return st; }
  const size_t es = elem_size(c->precision);
  CKC(cudaMalloc(&c->vecs, es * (size_t)c->n * c->nvec), "cudaMalloc workspace");
  CKC(cudaMalloc(&c->xbest, sizeof(double) * (size_t)c->n), "cudaMalloc best iterate");
  c->max_blocks = 4 * kMaxThreads;  // generous: any co-resident grid fits
  CKC(cudaMalloc(&c->part, sizeof(double) * 4 * kMaxDots * (size_t)c->max_blocks), "cudaMalloc partials");
  CKC(cudaStreamSynchronize(c->stream), "create");
  *out = c;
  return PBCG_OK;
#undef CKC
}

// Release what depends on the matrix values (kept: the pattern, the workspace, the state).
static void free_values(pbcg_ctx* c) {
  if (c->valAu && c->valAu != (void*)c->val64) cudaFree(c->valAu);
  void* ptrs[] = {c->val64, c->valAt, c->diag64, c->dinv64, c->dinvT, c->st_mask};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  c->val64 = nullptr; c->valAt = nullptr; c->valAu = nullptr; c->diag64 = nullptr; c->dinv64 = nullptr;
  c->dinvT = nullptr; c->st_mask = nullptr;
  c->stencil = 0; c->st_n = 0; c->st_dinv = 0.0; c->dconst = 0; c->dconst_inv = 0.0;
  c->bandwidth = 0; c->maxnnz = 0; c->ndiag_t = 0; c->at_unit_diag = 0; c->norm_bound = 0.0; c->dinv_max = 1.0;
}

extern "C" pbcg_status pbicgstab_update_values(pbcg_ctx* c, const void* val, int32_t val_dtype) {
  if (!c || !val) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_update_values");
  if (val_dtype != PBCG_F64 && val_dtype != PBCG_F32) return set_error(PBCG_INVALID_ARG, "unknown value dtype");
  CK(cudaStreamSynchronize(c->stream), "pending work");   // no solve may still read the old values
  pbcg_matrix A;
  memset(&A, 0, sizeof A);
  A.format = c->fmt;
  A.val_dtype = val_dtype;
  A.n = c->n;
  A.nnz = c->nnz;
  A.row_ptr = c->row_ptr;
  A.col = c->col;
  A.val = val;
  A.ndiag = c->ndiag;
  A.offsets = c->offsets;
  free_values(c);
  const pbcg_status st = prepare_matrix(c, &A, false);
  if (st != PBCG_OK) c->valid = 0;
  else c->valid = 1;
  return st;
}

extern "C" pbcg_status pbicgstab_set_options(pbcg_ctx* c, const pbcg_options* opt) {
  if (!c || !opt) return set_error(PBCG_INVALID_ARG, "NULL argument");
  pbcg_status st = check_options(opt, c->n);
  if (st != PBCG_OK) return st;
  if (opt->precision != c->precision) return set_error(PBCG_INVALID_ARG, "precision cannot change after create");
  if (opt->operator_storage != c->opt.operator_storage)
    return set_error(PBCG_INVALID_ARG, "operator_storage cannot change after create");
  st = check_method_precond(opt, c->prec_kind);
  if (st != PBCG_OK) return st;
  c->opt = *opt;
  return PBCG_OK;
}

extern "C" pbcg_status pbicgstab_destroy(pbcg_ctx* c) {
  if (!c) return PBCG_OK;
  cudaStreamSynchronize(c->stream);
  free_ctx(c);
  return PBCG_OK;
}

pbcg_status enqueue_true_residual(pbcg_ctx* c, const double* b, const double* x, double* out_dev) {
  const int sms = sm_count();
  const int nb = std::min(c->max_blocks, std::max(1, std::min(2 * sms, (c->n + 255) / 256)));
  true_res_partial_kernel<<<nb, 256, 0, c->stream>>>(pbcg_view64(c), b, x, c->part);
  true_res_final_kernel<<<1, 256, 0, c->stream>>>(c->part, nb, out_dev);
  CK(cudaGetLastError(), "true residual kernels");
  return PBCG_OK;
}

static pbcg_status enqueue_solve(pbcg_ctx* c, const double* b, double* x) {
  if (!c->valid) return set_error(PBCG_INVALID_ARG, "the context's last pbicgstab_update_values failed");
  int grid = 0, threads = 0;
  const bool vec = quad_rows(c, b, x);
  pbcg_status st = launch_shape(c, &grid, &threads, vec);
  if (st != PBCG_OK) return st;
  st = check_barrier_budget(c->opt.max_it, c->opt.max_restarts, c->degree, grid, c->opt.restart_period,
                            c->opt.stag_window);
  if (st != PBCG_OK) return st;
  CK(cudaMemsetAsync(c->dstate, 0, sizeof(DevState), c->stream), "memset state");
  CK(cudaEventRecord(c->ev0, c->stream), "event record");
  if (c->precision == PBCG_MIXED) {
    SolverParams<float> p = make_params<float>(c, b, x, grid, vec);
    const size_t dyn = staged_bytes(c, threads, vec);
    p.staged = dyn > 0 ? 1 : 0;
    c->launch[0] = grid; c->launch[1] = threads; c->launch[2] = vec ? 4 : 1;
    c->launch[3] = p.prefetch + 256 * p.overlap + 512 * p.staged;
    void* args[] = {&p};
    CK(cudaLaunchCooperativeKernel(kernel_ptr<float>(c, vec), grid, threads, args, dyn, c->stream),
       "cooperative launch");
  } else {
    SolverParams<double> p = make_params<double>(c, b, x, grid, vec);
    c->launch[0] = grid; c->launch[1] = threads; c->launch[2] = vec ? 4 : 1; c->launch[3] = p.prefetch + 256 * p.overlap;
    void* args[] = {&p};
    CK(cudaLaunchCooperativeKernel(kernel_ptr<double>(c, vec), grid, threads, args, 0, c->stream), "cooperative launch");
  }
  CK(cudaEventRecord(c->ev1, c->stream), "event record");
  return enqueue_true_residual(c, b, x, &c->dstate->true_rel);
}

static pbcg_status collect(pbcg_ctx* c, pbcg_result* res) {
  CK(cudaMemcpyAsync(c->hstate, c->dstate, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "copy state");
  CK(cudaStreamSynchronize(c->stream), "solve");
  const DevState& h = *c->hstate;
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1), "event timing");
  memset(res, 0, sizeof *res);
  res->status = h.err ? PBCG_TIMEOUT : h.res.status;
  res->iterations = h.res.iterations;
  res->n_replacements = h.res.nrep;
  res->n_restarts = h.res.nrestart;
  res->rel_res_recursive = h.res.rn_rel;
  res->rel_res_true = h.true_rel;
  res->time_ms = ms;
  if (res->status == PBCG_TIMEOUT) return set_error(PBCG_TIMEOUT, "a grid-wide wait exceeded timeout_ms");
  return (pbcg_status)res->status;
}

extern "C" pbcg_status pbicgstab_solve(pbcg_ctx* c, const double* b, double* x, pbcg_result* res) {
  if (!c || !b || !x) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_solve");
  pbcg_status st = enqueue_solve(c, b, x);
  if (st != PBCG_OK) return st;
  if (!res) return PBCG_OK;
  return collect(c, res);
}

extern "C" pbcg_status pbicgstab_solve_host(pbcg_ctx* c, const double* b_host, double* x_host, pbcg_result* res) {
  if (!c || !b_host || !x_host || !res) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_solve_host");
  // stream-ordered device copies of b and x for this call, freed on every path
  double* db = nullptr;
  double* dx = nullptr;
  const size_t bytes = sizeof(double) * (size_t)c->n;
  pbcg_status st = cuda_status(cudaMallocAsync((void**)&db, bytes, c->stream), "cudaMallocAsync b");
  if (st == PBCG_OK) st = cuda_status(cudaMallocAsync((void**)&dx, bytes, c->stream), "cudaMallocAsync x");
  if (st == PBCG_OK) st = cuda_status(cudaMemcpyAsync(db, b_host, bytes, cudaMemcpyHostToDevice, c->stream), "copy b");
  if (st == PBCG_OK) st = cuda_status(cudaMemcpyAsync(dx, x_host, bytes, cudaMemcpyHostToDevice, c->stream), "copy x0");
  if (st == PBCG_OK) st = enqueue_solve(c, db, dx);
  if (st == PBCG_OK) st = cuda_status(cudaMemcpyAsync(x_host, dx, bytes, cudaMemcpyDeviceToHost, c->stream), "copy x");
  if (st == PBCG_OK) st = collect(c, res);
  if (db) cudaFreeAsync(db, c->stream);
  if (dx) cudaFreeAsync(dx, c->stream);
  cudaStreamSynchronize(c->stream);
  return st;
}

extern "C" pbcg_status pbicgstab_spmv(pbcg_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_spmv");
  const int nb = std::max(1, std::min(4 * sm_count(), (c->n + 255) / 256));
  spmv_kernel<<<nb, 256, 0, c->stream>>>(pbcg_view64(c), x, y);
  CK(cudaGetLastError(), "spmv kernel");
  return PBCG_OK;
}

// dst_i = scale * src_i widened to FP64.
template <typename T>
__global__ void widen_kernel(int n, const T* src, double scale, double* dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = scale * (double)src[i];
}

extern "C" pbcg_status pbicgstab_get_vector(pbcg_ctx* c, int32_t which, double* dst) {
  if (!c || !dst) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_get_vector");
  // slot order of the workspace: r, rh, k, w, g, s, l, z (make_params)
  if (which < PBCG_VEC_R || which > PBCG_VEC_Z) return set_error(PBCG_INVALID_ARG, "unknown vector %d", which);
  // the scaled form keeps k, g, l multiplied by the constant diagonal d
  const bool pre = which == PBCG_VEC_K || which == PBCG_VEC_G || which == PBCG_VEC_L;
  const double scale = (pre && scalar_jacobi(c)) ? c->dconst_inv : 1.0;
  const int nb = std::max(1, std::min(4 * sm_count(), (c->n + 255) / 256));
  if (c->precision == PBCG_MIXED)
    widen_kernel<float><<<nb, 256, 0, c->stream>>>(c->n, (const float*)c->vecs + (size_t)which * c->n, scale, dst);
  else
    widen_kernel<double><<<nb, 256, 0, c->stream>>>(c->n, (const double*)c->vecs + (size_t)which * c->n, scale, dst);
  CK(cudaGetLastError(), "widen kernel");
  return PBCG_OK;
}

extern "C" pbcg_status pbicgstab_launch_info(const pbcg_ctx* c, int32_t info[4]) {
  if (!c || !info) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_launch_info");
  for (int j = 0; j < 4; ++j) info[j] = c->launch[j];
  return PBCG_OK;
}

extern "C" pbcg_status pbicgstab_true_residual(pbcg_ctx* c, const double* b, const double* x, double* rel) {
  if (!c || !b || !x || !rel) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_true_residual");
  pbcg_status st = enqueue_true_residual(c, b, x, &c->dstate->true_rel);
  if (st != PBCG_OK) return st;
  CK(cudaMemcpyAsync(rel, &c->dstate->true_rel, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy");
  CK(cudaStreamSynchronize(c->stream), "true residual");
  return PBCG_OK;
}

extern "C" pbcg_status pbicgstab_test_barrier_timeout(double timeout_ms, int32_t extra, int32_t* kernel_status) {
  if (!kernel_status || extra < 1 || !(timeout_ms > 0 && timeout_ms <= 10000))
    return set_error(PBCG_INVALID_ARG, "need extra >= 1, 0 < timeout_ms <= 10000 and a status pointer");
  unsigned* bar = nullptr;
  int* err = nullptr;
  cudaError_t e = cudaMalloc(&bar, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(bar, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
  const int grid = sm_count();
  unsigned long long tns = (unsigned long long)(timeout_ms * 1e6);
  int ex = extra;
  void* args[] = {&bar, &err, &ex, &tns};
  if (e == cudaSuccess) e = cudaLaunchCooperativeKernel((const void*)barrier_timeout_kernel, grid, 64, args, 0, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (bar) cudaFree(bar);
  if (err) cudaFree(err);
  CK(e, "barrier timeout kernel");
  *kernel_status = h ? PBCG_TIMEOUT : PBCG_OK;
  return PBCG_OK;
}
