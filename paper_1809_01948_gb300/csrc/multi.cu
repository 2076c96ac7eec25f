// Many right-hand sides with one matrix, the transposed-matrix context for the
// adjoint solve, and the gradient with respect to the CSR values.
#include <algorithm>
#include <new>
#include <vector>

#include "capi_internal.h"

using namespace pbcg;

namespace {

#define MCK(call, what)                                  \
  do {                                                   \
    pbcg_status s__ = cuda_status((call), (what));       \
    if (s__ != PBCG_OK) return s__;                      \
  } while (0)

// ---------------------------------------------------------------- transpose (CSR)
__global__ void count_cols_kernel(long long nnz, const int* col, int* cnt) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e < nnz) atomicAdd(cnt + col[e], 1);
}

// Exclusive scan of n+1 counts (cnt[n] = 0) in one block: each thread scans a
// contiguous chunk sequentially, then the chunk totals are scanned in shared memory.
__global__ void scan_kernel(int n, const int* cnt, int* out) {
  __shared__ long long tot[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  const int m = n + 1;
  const int per = (m + nt - 1) / nt;
  const int a = min(m, t * per), b = min(m, a + per);
  long long s = 0;
  for (int i = a; i < b; ++i) s += (i < n ? cnt[i] : 0);
  tot[t] = s;
  __syncthreads();
  if (t == 0) {
    long long run = 0;
    for (int i = 0; i < nt; ++i) { const long long v = tot[i]; tot[i] = run; run += v; }
  }
  __syncthreads();
  long long run = tot[t];
  for (int i = a; i < b; ++i) { out[i] = (int)run; run += (i < n ? cnt[i] : 0); }
}

__global__ void scatter_kernel(int n, const int* row_ptr, const int* col, const double* val, const int* rpT,
                               int* fill, int* colT, double* valT, int* perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    const int j = col[e];
    const int pos = rpT[j] + atomicAdd(fill + j, 1);
    colT[pos] = i;
    valT[pos] = val[e];
    perm[pos] = e;
  }
}

// Insertion sort of each transposed row by column: makes the result independent of
// the atomic order above (rows of A^T are short for the stencil-type matrices here).
// perm follows the entries, so valT[k] = val[perm[k]] afterwards.
__global__ void sort_rows_kernel(int n, const int* rp, int* col, double* val, int* perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int e0 = rp[i], e1 = rp[i + 1];
  for (int e = e0 + 1; e < e1; ++e) {
    const int c = col[e];
    const double v = val[e];
    const int pe = perm[e];
    int f = e - 1;
    while (f >= e0 && col[f] > c) { col[f + 1] = col[f]; val[f + 1] = val[f]; perm[f + 1] = perm[f]; --f; }
    col[f + 1] = c;
    val[f + 1] = v;
    perm[f + 1] = pe;
  }
}

// dst[k] = src[perm[k]]
__global__ void gather_kernel(long long m, const int* perm, const double* src, double* dst) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < m) dst[k] = src[perm[k]];
}

// ---------------------------------------------------------------- value gradient
// grad[e] = -sum_c Lam[row_e + c*n] * X[col_e + c*n]  (dL/dA_e of a linear solve)
__global__ void value_grad_kernel(int n, const int* row_ptr, const int* col, int nrhs, const double* Lam,
                                  const double* X, double* grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
    const int j = col[e];
    double g = 0.0;
    for (int c = 0; c < nrhs; ++c) g = fma(Lam[i + (size_t)c * n], X[j + (size_t)c * n], g);
    grad[e] = -g;
  }
}

template <typename T>
const void* multi_kernel_ptr() { return (const void*)pbicgstab_multi_kernel<T>; }

}  // namespace

static pbcg_status ensure_multi(pbcg_ctx* c, int teams, int bpt) {
  const size_t es = elem_size(c->precision);
  const size_t psz = c->precision == PBCG_MIXED ? sizeof(SolverParams<float>) : sizeof(SolverParams<double>);
  if (teams <= c->multi_cap && c->multi_part && bpt * teams <= c->max_blocks) return PBCG_OK;
  void* ptrs[] = {c->multi_vecs, c->multi_part, c->multi_state, c->multi_params};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->multi_hstate) cudaFreeHost(c->multi_hstate);
  if (c->multi_hparams) cudaFreeHost(c->multi_hparams);
  c->multi_vecs = c->multi_part = nullptr;
  c->multi_state = c->multi_hstate = nullptr;
  c->multi_params = c->multi_hparams = nullptr;
  c->multi_cap = 0;
  MCK(cudaMalloc(&c->multi_vecs, es * 15 * (size_t)c->n * teams), "cudaMalloc multi workspace");
  MCK(cudaMalloc(&c->multi_part, sizeof(double) * 3 * kMaxDots * (size_t)c->max_blocks), "cudaMalloc partials");
  MCK(cudaMalloc(&c->multi_state, sizeof(DevState) * teams), "cudaMalloc state");
  MCK(cudaMallocHost(&c->multi_hstate, sizeof(DevState) * teams), "cudaMallocHost state");
  MCK(cudaMalloc(&c->multi_params, psz * teams), "cudaMalloc params");
  MCK(cudaMallocHost(&c->multi_hparams, psz * teams), "cudaMallocHost params");
  c->multi_cap = teams;
  return PBCG_OK;
}

template <typename T>
static pbcg_status launch_wave(pbcg_ctx* c, int teams, int bpt, int nt, const double* B, double* X) {
  SolverParams<T>* hp = (SolverParams<T>*)c->multi_hparams;
  const size_t n = (size_t)c->n;
  // the teams stream their own vectors side by side: prefetch when together they exceed L2
  const int prefetch = (c->stencil && teams * hot_bytes(c) > (double)l2_bytes()) ? 1 : 0;
  for (int t = 0; t < teams; ++t) {
    SolverParams<T> p = make_params<T>(c, B + t * n, X + t * n, bpt);
    p.prefetch = prefetch;
    T* v = (T*)c->multi_vecs + (size_t)t * 15 * n;
    T** slots[] = {&p.r, &p.rh, &p.k, &p.w, &p.g, &p.s, &p.l, &p.z, &p.v, &p.t, &p.nb, &p.m, &p.nn, &p.tmpa, &p.tmpb};
    for (int j = 0; j < 15; ++j) *slots[j] = v + (size_t)j * n;
    p.part = c->multi_part + (size_t)t * 3 * kMaxDots * bpt;
    p.bar = &c->multi_state[t].bar;
    p.err = &c->multi_state[t].err;
    p.res = &c->multi_state[t].res;
    p.hist_x = nullptr;
    p.K = 0;
    p.hist_s = nullptr;
    p.hist_len = 0;
    p.xbest = nullptr;   // stagnation is detected per column, but the last iterate is returned
    p.overlap = 0;       // the teams run plain barriers
    hp[t] = p;
  }
  MCK(cudaMemcpyAsync(c->multi_params, hp, sizeof(SolverParams<T>) * teams, cudaMemcpyHostToDevice, c->stream),
      "copy params");
  MCK(cudaMemsetAsync(c->multi_state, 0, sizeof(DevState) * teams, c->stream), "memset state");
  const SolverParams<T>* dp = (const SolverParams<T>*)c->multi_params;
  void* args[] = {&dp, &bpt};
  MCK(cudaLaunchCooperativeKernel(multi_kernel_ptr<T>(), teams * bpt, nt, args, 0, c->stream), "cooperative launch");
  return PBCG_OK;
}

extern "C" pbcg_status pbicgstab_solve_multi(pbcg_ctx* c, int32_t nrhs, const double* B, double* X,
                                             pbcg_result* res) {
  if (!c || !B || !X || nrhs < 1) return set_error(PBCG_INVALID_ARG, "pbicgstab_solve_multi needs ctx, B, X, nrhs >= 1");
  if (c->opt.rr_auto) return set_error(PBCG_INVALID_ARG, "pbicgstab_solve_multi does not support rr_auto");
  if (c->opt.method != PBCG_PIPELINED) return set_error(PBCG_INVALID_ARG, "pbicgstab_solve_multi runs Algorithm 2 only");
  const int nt = c->opt.block_threads ? c->opt.block_threads : 512;
  int per_sm = 0;
  const void* k = c->precision == PBCG_MIXED ? multi_kernel_ptr<float>() : multi_kernel_ptr<double>();
  MCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, nt, 0), "occupancy");
  const int max_co = std::min(per_sm * sm_count(), c->max_blocks);
  if (max_co < 1) return set_error(PBCG_INVALID_ARG, "multi kernel cannot be resident with %d threads", nt);
  int G = c->opt.grid_blocks ? std::min(c->opt.grid_blocks, max_co) : std::min(max_co, 2 * sm_count());
  const int teams = std::min(nrhs, G);
  // blocks per team: share the grid, at least 32 rows per block
  int bpt = std::max(1, G / teams);
  bpt = (int)std::min<long long>(bpt, std::max<long long>(1, (c->n + 31) / 32));
  pbcg_status st = check_barrier_budget(c->opt.max_it, c->opt.max_restarts, c->degree, bpt, c->opt.restart_period,
                                        c->opt.stag_window);
  if (st != PBCG_OK) return st;
  st = ensure_multi(c, teams, bpt);
  if (st != PBCG_OK) return st;
  float ms_total = 0.f;
  const size_t n = (size_t)c->n;
  for (int w0 = 0; w0 < nrhs; w0 += teams) {
    const int tw = std::min(teams, nrhs - w0);
    MCK(cudaEventRecord(c->ev0, c->stream), "event");
    st = c->precision == PBCG_MIXED ? launch_wave<float>(c, tw, bpt, nt, B + w0 * n, X + w0 * n)
                                    : launch_wave<double>(c, tw, bpt, nt, B + w0 * n, X + w0 * n);
    if (st != PBCG_OK) return st;
    MCK(cudaEventRecord(c->ev1, c->stream), "event");
    for (int t = 0; t < tw; ++t) {
      st = enqueue_true_residual(c, B + (w0 + t) * n, X + (w0 + t) * n, &c->multi_state[t].true_rel);
      if (st != PBCG_OK) return st;
    }
    MCK(cudaMemcpyAsync(c->multi_hstate, c->multi_state, sizeof(DevState) * tw, cudaMemcpyDeviceToHost, c->stream),
        "copy state");
    MCK(cudaStreamSynchronize(c->stream), "multi solve");
    float ms = 0.f;
    MCK(cudaEventElapsedTime(&ms, c->ev0, c->ev1), "event timing");
    ms_total += ms;
    for (int t = 0; t < tw; ++t) {
      const DevState& h = c->multi_hstate[t];
      if (h.err) return set_error(PBCG_TIMEOUT, "a team barrier exceeded timeout_ms");
      if (res) {
        pbcg_result& r = res[w0 + t];
        memset(&r, 0, sizeof r);
        r.status = h.res.status;
        r.iterations = h.res.iterations;
        r.n_replacements = h.res.nrep;
        r.n_restarts = h.res.nrestart;
        r.rel_res_recursive = h.res.rn_rel;
        r.rel_res_true = h.true_rel;
      }
    }
  }
  pbcg_status worst = PBCG_OK;
  if (res) {
    for (int j = 0; j < nrhs; ++j) {
      res[j].time_ms = ms_total;
      if (res[j].status != PBCG_OK && worst == PBCG_OK) worst = (pbcg_status)res[j].status;
    }
  }
  return worst;
}

extern "C" pbcg_status pbicgstab_create_transpose(pbcg_ctx** out, const pbcg_ctx* src) {
  if (!out || !src) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_create_transpose");
  *out = nullptr;
  if (src->fmt != PBCG_FMT_CSR) return set_error(PBCG_INVALID_ARG, "pbicgstab_create_transpose needs a CSR matrix");
  const int n = src->n;
  const long long nnz = src->nnz;
  cudaStream_t s = src->stream;
  int *cnt = nullptr, *rpT = nullptr, *colT = nullptr, *perm = nullptr;
  double* valT = nullptr;
  pbcg_status st = PBCG_OK;
  auto fail = [&](pbcg_status e) {
    if (cnt) cudaFree(cnt);
    if (rpT) cudaFree(rpT);
    if (colT) cudaFree(colT);
    if (valT) cudaFree(valT);
    if (perm) cudaFree(perm);
    return e;
  };
  if ((st = cuda_status(cudaMalloc(&cnt, sizeof(int) * (n + 1)), "cudaMalloc")) != PBCG_OK) return fail(st);
  if ((st = cuda_status(cudaMalloc(&rpT, sizeof(int) * (n + 1)), "cudaMalloc")) != PBCG_OK) return fail(st);
  if ((st = cuda_status(cudaMalloc(&colT, sizeof(int) * std::max<long long>(1, nnz)), "cudaMalloc")) != PBCG_OK) return fail(st);
  if ((st = cuda_status(cudaMalloc(&valT, sizeof(double) * std::max<long long>(1, nnz)), "cudaMalloc")) != PBCG_OK) return fail(st);
  if ((st = cuda_status(cudaMalloc(&perm, sizeof(int) * std::max<long long>(1, nnz)), "cudaMalloc")) != PBCG_OK) return fail(st);
  cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), s);
  const unsigned nbe = (unsigned)((nnz + 255) / 256), nbr = (unsigned)((n + 255) / 256);
  if (nnz) count_cols_kernel<<<nbe, 256, 0, s>>>(nnz, src->col, cnt);
  scan_kernel<<<1, 1024, 0, s>>>(n, cnt, rpT);
  cudaMemsetAsync(cnt, 0, sizeof(int) * (n + 1), s);
  scatter_kernel<<<nbr, 256, 0, s>>>(n, src->row_ptr, src->col, src->val64, rpT, cnt, colT, valT, perm);
  sort_rows_kernel<<<nbr, 256, 0, s>>>(n, rpT, colT, valT, perm);
  if ((st = cuda_status(cudaGetLastError(), "transpose kernels")) != PBCG_OK) return fail(st);
  pbcg_matrix m;
  memset(&m, 0, sizeof m);
  m.format = PBCG_FMT_CSR;
  m.val_dtype = PBCG_F64;
  m.n = n;
  m.nnz = nnz;
  m.row_ptr = rpT;
  m.col = colT;
  m.val = valT;
  pbcg_precond M;
  M.kind = src->prec_kind;
  M.degree = src->degree;
  st = pbicgstab_create(out, &m, &M, &src->opt, (void*)s);
  if (st == PBCG_OK) {   // the permutation stays with the transpose context (value updates)
    (*out)->tperm = perm;
    perm = nullptr;
  }
  return fail(st);   // the new context holds its own copies
}

extern "C" pbcg_status pbicgstab_update_transpose(pbcg_ctx* t, const pbcg_ctx* src) {
  if (!t || !src) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_update_transpose");
  if (!t->tperm || t->n != src->n || t->nnz != src->nnz || src->fmt != PBCG_FMT_CSR)
    return set_error(PBCG_INVALID_ARG, "pbicgstab_update_transpose needs a context made by pbicgstab_create_transpose "
                                       "from a matrix with the source's pattern");
  double* valT = nullptr;
  MCK(cudaMalloc(&valT, sizeof(double) * std::max<long long>(1, t->nnz)), "cudaMalloc");
  const long long m = t->nnz;
  if (m) gather_kernel<<<(unsigned)((m + 255) / 256), 256, 0, src->stream>>>(m, t->tperm, src->val64, valT);
  pbcg_status st = cuda_status(cudaGetLastError(), "gather kernel");
  if (st == PBCG_OK) st = cuda_status(cudaStreamSynchronize(src->stream), "gather");
  if (st == PBCG_OK) st = pbicgstab_update_values(t, valT, PBCG_F64);
  cudaFree(valT);
  return st;
}

extern "C" pbcg_status pbicgstab_csr_value_grad(pbcg_ctx* c, int32_t nrhs, const double* Lam, const double* X,
                                                double* grad) {
  if (!c || !Lam || !X || !grad || nrhs < 1) return set_error(PBCG_INVALID_ARG, "bad arguments to pbicgstab_csr_value_grad");
  if (c->fmt != PBCG_FMT_CSR) return set_error(PBCG_INVALID_ARG, "pbicgstab_csr_value_grad needs a CSR matrix");
  value_grad_kernel<<<(c->n + 255) / 256, 256, 0, c->stream>>>(c->n, c->row_ptr, c->col, nrhs, Lam, X, grad);
  MCK(cudaGetLastError(), "value gradient kernel");
  return PBCG_OK;
}
