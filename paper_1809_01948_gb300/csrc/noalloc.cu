// pbicgstab_solve_noalloc: the single-system FP64 solver for callers that cannot
// allocate GPU memory.  All scratch memory lives in one file-scope __device__
// array of fixed size; nothing here calls cudaMalloc/cudaFree or an allocating
// library routine.
#include <cstring>

#include "../../include/pbicgstab.h"
#include "capi_internal.h"
#include "solver.cuh"

using namespace pbcg;

namespace {

// Layout of the static scratch (offsets in bytes, each 256-byte aligned).
constexpr long long kMaxN = PBCG_NOALLOC_MAX_N;
constexpr long long kMaxVals = PBCG_NOALLOC_MAX_VALUES;
constexpr int kMaxGrid = 1024;
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffState = 0;
constexpr size_t kOffPart = align256(kOffState + 256);
constexpr size_t kOffDiag = align256(kOffPart + sizeof(double) * 3 * kMaxDots * kMaxGrid);
constexpr size_t kOffDinv = align256(kOffDiag + sizeof(double) * kMaxN);
constexpr size_t kOffFold = align256(kOffDinv + sizeof(double) * kMaxN);
constexpr size_t kOffVecs = align256(kOffFold + sizeof(double) * kMaxVals);
constexpr size_t kScratchBytes = align256(kOffVecs + sizeof(double) * 15 * kMaxN);

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct NoAllocState {
  DevResult res;
  unsigned bar;
  int err;
  double true_rel;
  int flags;
  int reserved;
  unsigned long long drange[2];   // smallest / largest diagonal entry (order-preserving images)
};
static_assert(sizeof(NoAllocState) <= 256, "the scratch reserves 256 bytes for the state");

// Smallest and largest diagonal entry, as the context-based solver computes them: with a
// constant diagonal both entry points run Jacobi in the same scaled form.
__device__ __forceinline__ unsigned long long na_ordered(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void na_diag_range(int n, const double* diag, unsigned long long* range) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long lo = ~0ull, hi = 0ull;
  if (i < n) lo = hi = na_ordered(diag[i]);
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

// Device address of g_scratch in the current context.  In host code the name g_scratch
// is only a host-side stand-in, so the address comes from cudaGetSymbolAddress, with the
// device current.  It is looked up on every call (the lookup allocates nothing): a cached
// address could be stale after cudaDeviceReset or in another context of the same device.
pbcg_status scratch_address(void** out) {
  void* p = nullptr;
  pbcg_status st = cuda_status(cudaGetSymbolAddress(&p, g_scratch), "cudaGetSymbolAddress(scratch)");
  if (st != PBCG_OK) return st;
  *out = p;
  return PBCG_OK;
}

__global__ void na_validate_csr(int n, long long nnz, const int* row_ptr, const int* col, const double* val,
                                int need_diag, int* flags, double* diag, int* bandwidth) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = 0;
  const int e0 = row_ptr[i], e1 = row_ptr[i + 1];
  if (i == 0 && e0 != 0) f |= 1;
  if (i == n - 1 && (long long)e1 != nnz) f |= 1;
  if (e1 < e0 || e0 < 0 || (long long)e1 > nnz) { atomicOr(flags, f | 1); return; }
  double dg = 0.0;
  int prev = -1, bw = 0;
  for (int e = e0; e < e1; ++e) {
    const int c = col[e];
    if (c < 0 || c >= n || c <= prev) f |= 2;
    prev = c;
    bw = max(bw, abs(c - i));
    if (!isfinite(val[e])) f |= 4;
    if (c == i) dg = val[e];
  }
  if (need_diag && dg == 0.0) f |= 8;
  diag[i] = dg;
  if (bw) atomicMax(bandwidth, bw);
  if (f) atomicOr(flags, f);
}

__global__ void na_validate_dia(MatView<double> A, int need_diag, int* flags, double* diag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  int f = 0;
  double dg = 0.0;
  for (int d = 0; d < A.ndiag; ++d) {
    const int j = i + A.off[d];
    if (j < 0 || j >= A.n) continue;
    const double v = A.val[(size_t)d * A.n + i];
    if (!isfinite(v)) f |= 4;
    if (A.off[d] == 0) dg = v;
  }
  if (need_diag && dg == 0.0) f |= 8;
  diag[i] = dg;
  if (f) atomicOr(flags, f);
}

// D^{-1} and the operator A D^{-1} (DIA: without its exact unit main diagonal).
__global__ void na_fold(MatView<double> A, const double* diag, double* dinv, double* fold) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  dinv[i] = 1.0 / diag[i];
  if (A.fmt == 0) {
    for (int e = A.row_ptr[i]; e < A.row_ptr[i + 1]; ++e) fold[e] = A.val[e] * (1.0 / diag[A.col[e]]);
  } else {
    int dd = 0;
    for (int d = 0; d < A.ndiag; ++d) {
      if (A.off[d] == 0) continue;
      const int j = i + A.off[d];
      fold[(size_t)dd * A.n + i] = (j >= 0 && j < A.n) ? A.val[(size_t)d * A.n + i] * (1.0 / diag[j]) : 0.0;
      ++dd;
    }
  }
}

__global__ void na_true_res(MatView<double> A, const double* b, const double* x, double* out) {
  __shared__ double smem[kWork + kMaxDots];
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < A.n; i += blockDim.x) {
    const double r = b[i] - row_dot<double>(A, x, i);
    v[0] = fma(r, r, v[0]);
    v[1] = fma(b[i], b[i], v[1]);
  }
  block_sum<2>(v, smem);
  if (threadIdx.x == 0) out[0] = v[1] > 0.0 ? sqrt(v[0]) / sqrt(v[1]) : sqrt(v[0]);
}

#define NCK(call, what)                                  \
  do {                                                   \
    pbcg_status s__ = cuda_status((call), (what));       \
    if (s__ != PBCG_OK) return s__;                      \
  } while (0)

}  // namespace

extern "C" pbcg_status pbicgstab_solve_noalloc(const pbcg_matrix* A, const pbcg_precond* M, const pbcg_options* opt,
                                               const double* b, double* x, pbcg_result* res, void* stream) {
  if (!A || !M || !opt || !b || !x || !res) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_solve_noalloc");
  if (A->n < 1 || A->n > kMaxN)
    return set_error(PBCG_INVALID_ARG, "pbicgstab_solve_noalloc: n = %lld outside [1, %lld] (static scratch limit)",
                     (long long)A->n, kMaxN);
  if (A->val_dtype != PBCG_F64 || !A->val) return set_error(PBCG_INVALID_ARG, "pbicgstab_solve_noalloc needs FP64 values");
  if (opt->precision != PBCG_FP64) return set_error(PBCG_INVALID_ARG, "pbicgstab_solve_noalloc supports FP64 only");
  if (M->kind != PBCG_PREC_NONE && M->kind != PBCG_PREC_JACOBI)
    return set_error(PBCG_INVALID_ARG, "pbicgstab_solve_noalloc supports no preconditioner or Jacobi");
  {
    const pbcg_status os = check_options(opt, A->n);   // the context solver's option checks
    if (os != PBCG_OK) return os;
  }
  if (opt->rr_auto != 0) return set_error(PBCG_INVALID_ARG, "pbicgstab_solve_noalloc does not run the automated policy");
  if (opt->method != PBCG_PIPELINED) return set_error(PBCG_INVALID_ARG, "pbicgstab_solve_noalloc runs Algorithm 2 only");
  const int n = (int)A->n;
  MatView<double> A64;
  memset(&A64, 0, sizeof A64);
  A64.n = n;
  A64.val = (const double*)A->val;
  if (A->format == PBCG_FMT_CSR) {
    if (!A->row_ptr || (A->nnz > 0 && !A->col) || A->nnz < 0) return set_error(PBCG_INVALID_ARG, "CSR arrays are NULL");
    if (A->nnz > kMaxVals)
      return set_error(PBCG_INVALID_ARG, "pbicgstab_solve_noalloc: nnz = %lld above %lld (static scratch limit)",
                       (long long)A->nnz, kMaxVals);
    A64.fmt = 0;
    A64.row_ptr = A->row_ptr;
    A64.col = A->col;
  } else if (A->format == PBCG_FMT_DIA) {
    if (A->ndiag < 1 || A->ndiag > kMaxDiag || !A->offsets) return set_error(PBCG_INVALID_ARG, "bad DIA description");
    bool has0 = false;
    for (int d = 0; d < A->ndiag; ++d) {
      if ((d > 0 && A->offsets[d] <= A->offsets[d - 1]) || A->offsets[d] <= -n || A->offsets[d] >= n)
        return set_error(PBCG_INVALID_ARG, "DIA offsets must increase and lie in (-n, n)");
      has0 |= A->offsets[d] == 0;
      A64.off[d] = A->offsets[d];
    }
    if (!has0) return set_error(PBCG_INVALID_ARG, "DIA offsets must contain 0");
    if ((long long)A->ndiag * n > kMaxVals) return set_error(PBCG_INVALID_ARG, "DIA values above the static limit");
    A64.fmt = 1;
    A64.ndiag = A->ndiag;
  } else {
    return set_error(PBCG_INVALID_ARG, "unknown matrix format");
  }
  void* base = nullptr;
  pbcg_status st = scratch_address(&base);
  if (st != PBCG_OK) return st;
  unsigned char* sb = (unsigned char*)base;
  NoAllocState* state = (NoAllocState*)(sb + kOffState);
  double* part = (double*)(sb + kOffPart);
  double* diag = (double*)(sb + kOffDiag);
  double* dinv = (double*)(sb + kOffDinv);
  double* fold = (double*)(sb + kOffFold);
  double* vecs = (double*)(sb + kOffVecs);
  cudaStream_t s = (cudaStream_t)stream;
  const bool jac = M->kind == PBCG_PREC_JACOBI;
  // the solver state must start at zero (barrier counter, error flag, result)
  NCK(cudaMemsetAsync(state, 0, sizeof(NoAllocState), s), "memset scratch state");
  const int nb = (n + 255) / 256;
  if (A64.fmt == 0)
    na_validate_csr<<<nb, 256, 0, s>>>(n, A->nnz, A->row_ptr, A->col, A64.val, jac, &state->flags, diag,
                                        &state->reserved);
  else
    na_validate_dia<<<nb, 256, 0, s>>>(A64, jac, &state->flags, diag);
  NCK(cudaGetLastError(), "validation launch");
  NoAllocState h;
  NCK(cudaMemcpyAsync(&h, state, sizeof h, cudaMemcpyDeviceToHost, s), "copy flags");
  NCK(cudaStreamSynchronize(s), "validation");
  if (h.flags & 1) return set_error(PBCG_INVALID_ARG, "CSR row_ptr is not monotone from 0 to nnz");
  if (h.flags & 2) return set_error(PBCG_INVALID_ARG, "CSR column index out of range or not increasing");
  if (h.flags & 4) return set_error(PBCG_INVALID_ARG, "matrix has a non-finite value");
  if (h.flags & 8) return set_error(PBCG_INVALID_ARG, "Jacobi needs a non-zero diagonal");
  bool dconst = false;
  double dconst_inv = 0.0;
  if (jac) {
    na_fold<<<nb, 256, 0, s>>>(A64, diag, dinv, fold);
    NCK(cudaGetLastError(), "fold launch");
    const unsigned long long init[2] = {~0ull, 0ull};
    NCK(cudaMemcpyAsync(state->drange, init, sizeof init, cudaMemcpyHostToDevice, s), "copy");
    na_diag_range<<<nb, 256, 0, s>>>(n, diag, state->drange);
    NCK(cudaGetLastError(), "diagonal range launch");
    unsigned long long hr[2];
    NCK(cudaMemcpyAsync(hr, state->drange, sizeof hr, cudaMemcpyDeviceToHost, s), "copy");
    NCK(cudaStreamSynchronize(s), "diagonal range");
    if (hr[0] == hr[1]) {
      const unsigned long long u = (hr[0] >> 63) ? (hr[0] & 0x7fffffffffffffffull) : ~hr[0];
      double d;
      memcpy(&d, &u, sizeof d);
      dconst = true;
      dconst_inv = 1.0 / d;
    }
  }
  // launch shape: the context-based solver's default rule (one 1024-thread block per SM,
  // every co-resident block slot busy but at least 32 rows per block), so that a call with
  // default options sums its dot products in the same order as pbicgstab_solve
  const void* kern = pipelined_kernel_f64(false, jac && dconst, false);
  const int nt = opt->block_threads ? opt->block_threads : pbcg::SolverLaunch<double, false>::kThreads;
  cudaFuncAttributes fa;
  NCK(cudaFuncGetAttributes(&fa, kern), "kernel attributes");
  if (nt > fa.maxThreadsPerBlock)
    return set_error(PBCG_INVALID_ARG, "block_threads %d above this solver's limit of %d", nt, fa.maxThreadsPerBlock);
  int per_sm = 0;
  NCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, 0), "occupancy");
  if (per_sm <= 0) return set_error(PBCG_INVALID_ARG, "kernel cannot be resident with %d threads per block", nt);
  const int max_co = std::min(per_sm * sm_count(), kMaxGrid);
  int grid = opt->grid_blocks;
  if (grid == 0) grid = (int)std::min<long long>(std::max<long long>(1, (n + 31) / 32), (long long)max_co);
  if (grid < 1 || grid > max_co) return set_error(PBCG_INVALID_ARG, "grid_blocks %d above %d", grid, max_co);
  {
    const pbcg_status bs = check_barrier_budget(opt->max_it, opt->max_restarts, 0, grid, opt->restart_period,
                                                opt->stag_window);
    if (bs != PBCG_OK) return bs;
  }
  SolverParams<double> p;
  memset(&p, 0, sizeof p);
  p.n = n;
  p.chunk = (n + grid - 1) / grid;
  p.A64 = A64;
  p.Au = A64;
  if (jac) {
    p.At = A64;
    p.At.val = fold;
    if (A64.fmt == 1) {
      int dd = 0;
      for (int d = 0; d < A64.ndiag; ++d)
        if (A64.off[d] != 0) p.At.off[dd++] = A64.off[d];
      p.At.ndiag = dd;
      p.At.unit_diag = 1;
    }
  } else {
    p.At = A64;
  }
  p.dinv = jac ? dinv : nullptr;
  p.dinv_x = (jac && dconst) ? dconst_inv : 1.0;
  p.prec = M->kind;
  p.b = b;
  p.x = x;
  double** slots[] = {&p.r, &p.rh, &p.k, &p.w, &p.g, &p.s, &p.l, &p.z, &p.v, &p.t, &p.nb, &p.m, &p.nn, &p.tmpa, &p.tmpb};
  for (int j = 0; j < 15; ++j) *slots[j] = vecs + (size_t)j * n;
  p.part = part;
  p.bar = &state->bar;
  p.err = &state->err;
  p.res = &state->res;
  p.hist_x = opt->hist_x;
  p.K = opt->record_iterates;
  p.hist_s = opt->hist_scalars;
  p.hist_len = opt->hist_len;
  p.tol = opt->tol;
  p.max_it = opt->max_it;
  p.rr_period = opt->rr_period;
  p.rr_theta = opt->rr_theta;
  const double tms = opt->timeout_ms > 0 ? opt->timeout_ms : 2000.0;
  p.timeout_ns = (unsigned long long)(tms * 1e6);
  p.max_restarts = opt->max_restarts;
  p.restart_period = opt->restart_period;
  p.stag_window = opt->stag_window;
  p.xbest = p.tmpa;   // FP64 and no Neumann sweeps here: the sweep temporary is free
  p.rr_cutoff = opt->rr_cutoff > 0.0 ? opt->rr_cutoff : 1.4901161193847656e-08;   // sqrt(2^-52)
  // row order: the same rule as the context-based solver
  int bandwidth = 0;
  if (A64.fmt == 0) bandwidth = h.reserved;
  else for (int d = 0; d < A64.ndiag; ++d) bandwidth = std::max(bandwidth, std::abs(A64.off[d]));
  p.strided = bandwidth > p.chunk / 2 ? 1 : 0;
  void* args[] = {&p};
  NCK(cudaLaunchCooperativeKernel(kern, grid, nt, args, 0, s), "cooperative launch");
  na_true_res<<<1, 1024, 0, s>>>(A64, b, x, &state->true_rel);
  NCK(cudaGetLastError(), "true residual launch");
  NCK(cudaMemcpyAsync(&h, state, sizeof h, cudaMemcpyDeviceToHost, s), "copy result");
  NCK(cudaStreamSynchronize(s), "solve");
  memset(res, 0, sizeof *res);
  res->status = h.err ? PBCG_TIMEOUT : h.res.status;
  res->iterations = h.res.iterations;
  res->n_replacements = h.res.nrep;
  res->n_restarts = h.res.nrestart;
  res->rel_res_recursive = h.res.rn_rel;
  res->rel_res_true = h.true_rel;
  res->time_ms = -1.0;
  if (res->status == PBCG_TIMEOUT) return set_error(PBCG_TIMEOUT, "a grid-wide wait exceeded timeout_ms");
  return (pbcg_status)res->status;
}
