// Batched p-BiCGStab: many independent systems in one persistent launch.  Each
// thread block repeatedly takes the next system from a device queue (largest
// first) and runs the same algorithm body as the single-system solver with a
// block-scope team (__syncthreads barriers, shared-memory reductions).
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <type_traits>
#include <vector>

#include "../../include/pbicgstab.h"
#include "capi_internal.h"
#include "solver.cuh"

using namespace pbcg;

namespace {

struct BatchDev {
  int n_sys;
  const long long* row_off;   // n_sys + 1
  const long long* nnz_off;   // n_sys + 1
  const int* order;           // system ids, largest first
  const int* row_ptr;
  const int* col;
  const void* valAt;          // A D^{-1} (or A) in T
  const void* valAu;          // A in T
  const void* valR;           // A in VR (stored values)
  const void* dinv;           // D^{-1} in T, or nullptr
  const double* b;
  double* x;
  void* vecs;                 // 15 * total_rows values of T
  long long total_rows;
  DevResult* res;             // n_sys
  unsigned* counter;
  int prec;
  int degree;                 // Neumann degree (prec == PBCG_PREC_NEUMANN)
  double tol;
  int max_it;
  int rr_period;
  double rr_theta;
  int max_restarts;
  int restart_period;
  int stag_window;
  double rr_cutoff;
  int lanes;                  // threads per row in the SpMVs of passes A and B
};

template <typename V>
__device__ __forceinline__ MatView<V> csr_view(int n, const int* rp, const int* col, const V* val) {
  MatView<V> m;
  m.fmt = 0;
  m.n = n;
  m.row_ptr = rp;
  m.col = col;
  m.val = val;
  m.ndiag = 0;
  m.unit_diag = 0;
  m.pattern = 0;
  return m;
}

// Parameters of system k for the algorithm body (built by one thread into shared memory).
template <typename T, typename VR>
__device__ void build_params(const BatchDev& d, int k, SolverParams<T, VR>& p) {
  const long long r0 = d.row_off[k], e0 = d.nnz_off[k];
  const int n = (int)(d.row_off[k + 1] - r0);
  const int* rp = d.row_ptr + r0 + k;
  const int* col = d.col + e0;
  p.n = n;
  p.chunk = n;
  p.At = csr_view<T>(n, rp, col, (const T*)d.valAt + e0);
  p.Au = csr_view<T>(n, rp, col, (const T*)d.valAu + e0);
  p.A64 = csr_view<VR>(n, rp, col, (const VR*)d.valR + e0);
  p.dinv = d.dinv ? (const T*)d.dinv + r0 : nullptr;
  p.dinv_c = T(0);
  p.dinv_x = 1.0;
  p.prefetch = 0;
  p.prec = d.prec;
  p.degree = d.degree;
  p.b = d.b + r0;
  p.x = d.x + r0;
  T* v = (T*)d.vecs + r0;
  const size_t R = (size_t)d.total_rows;
  p.r = v;          p.rh = v + R;      p.k = v + 2 * R;   p.w = v + 3 * R;   p.g = v + 4 * R;
  p.s = v + 5 * R;  p.l = v + 6 * R;   p.z = v + 7 * R;   p.v = v + 8 * R;   p.t = v + 9 * R;
  p.nb = v + 10 * R; p.m = v + 11 * R; p.nn = v + 12 * R; p.tmpa = v + 13 * R; p.tmpb = v + 14 * R;
  p.part = nullptr;
  p.bar = nullptr;
  p.err = nullptr;
  p.res = d.res + k;
  p.hist_x = nullptr;
  p.K = 0;
  p.hist_s = nullptr;
  p.hist_len = 0;
  p.tol = d.tol;
  p.max_it = d.max_it;
  p.rr_period = d.rr_period;
  p.rr_theta = d.rr_theta;
  p.timeout_ns = 0;
  p.max_restarts = d.max_restarts;
  p.restart_period = d.restart_period;
  p.stag_window = d.stag_window;
  p.xbest = nullptr;   // stagnation is detected per system, but the last iterate is returned
  p.rr_cutoff = d.rr_cutoff;
  p.strided = 0;
  p.overlap = 0;   // block and cluster teams: no grid barrier to overlap
  p.halo = 0;
  p.staged = 0;
}

template <typename T, typename VR>
__global__ void __launch_bounds__(kMaxThreads, 1) batched_kernel(const BatchDev d) {
  __shared__ double smem[kWork + 3 * kMaxDots];
  __shared__ double scal[8];
  __shared__ int s_sys;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned q = atomicAdd(d.counter, 1u);
      s_sys = q < (unsigned)d.n_sys ? d.order[q] : -1;
    }
    __syncthreads();
    const int k = s_sys;
    if (k < 0) return;
    __shared__ SolverParams<T, VR> p;   // per-system parameters, built by thread 0
    const int n = (int)(d.row_off[k + 1] - d.row_off[k]);
    if (threadIdx.x == 0) build_params(d, k, p);
    __syncthreads();
    BlockTeam team;
    team.first = 0;
    team.stride = blockDim.x;
    team.end = n;
    team.lanes = d.lanes;
    team.smem = smem;
    team.scal = scal;
    solve_body<false, false>(p, team);
    __syncthreads();
    // final FP64 true residual of this system
    double a[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double bi = p.b[i];
      const double r = bi - row_dot<double>(p.A64, p.x, i);
      a[0] = fma(r, r, a[0]);
      a[1] = fma(bi, bi, a[1]);
    }
    block_reduce<2>(a, smem, smem + kWork);
    if (threadIdx.x == 0) {
      const double rr = smem[kWork], bb = smem[kWork + 1];
      p.res->true_rel = bb > 0.0 ? sqrt(rr) / sqrt(bb) : sqrt(rr);
    }
  }
}

// One thread-block cluster per system: the cluster's blocks share the rows (block rank
// r takes rows r*blockDim + t, stepping by the cluster's threads), synchronise with the
// hardware cluster barrier and sum their partials through distributed shared memory.
// Large systems then run on several SMs while small ones still fill the GPU.  Every block
// of a cluster takes the same control-flow decisions (the totals are identical), so all
// reach every cluster barrier.  STREAM: the mixed solver's streaming register budget
// (SolverLaunch<float, true>: 40 registers, six 256-thread blocks per SM instead of four);
// on the 512-system banded batch the extra resident warps cut the solve by 12%.
template <typename T, typename VR, bool STREAM = false>
__global__ void __launch_bounds__(SolverLaunch<T, STREAM>::kThreads, SolverLaunch<T, STREAM>::kBlocksPerSM)
    batched_cluster_kernel(const BatchDev d) {
  __shared__ double smem[kWork + 5 * kMaxDots];
  __shared__ double scal[8];
  __shared__ int s_sys;      // rank 0: the system the cluster works on
  __shared__ int s_local;    // every block: its copy of it
  __shared__ SolverParams<T, VR> p;
  unsigned rank, nrank;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(nrank));
  ClusterTeam team;
  team.lanes = d.lanes;
  team.rank = rank;
  team.nrank = nrank;
  team.smem = smem;
  team.scal = scal;
  for (;;) {
    team.sync();   // every block is done with the previous system and its s_sys
    if (rank == 0 && threadIdx.x == 0) {
      const unsigned q = atomicAdd(d.counter, 1u);
      s_sys = q < (unsigned)d.n_sys ? d.order[q] : -1;
    }
    team.sync();
    if (threadIdx.x == 0) {
      const unsigned laddr = (unsigned)__cvta_generic_to_shared(&s_sys);
      unsigned raddr;
      int k;
      asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(0u));
      asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(k) : "r"(raddr) : "memory");
      s_local = k;
      if (k >= 0) build_params(d, k, p);
    }
    __syncthreads();
    const int k = s_local;
    if (k < 0) break;
    const int n = (int)(d.row_off[k + 1] - d.row_off[k]);
    team.first = (int)rank * blockDim.x;
    team.stride = (int)nrank * blockDim.x;
    team.end = n;
    solve_body<false, false>(p, team);
    team.sync();
    // final FP64 true residual of this system
    double a[2] = {0.0, 0.0};
    for (int i = team.first + threadIdx.x; i < n; i += team.stride) {
      const double bi = p.b[i];
      const double r = bi - row_dot<double>(p.A64, p.x, i);
      a[0] = fma(r, r, a[0]);
      a[1] = fma(bi, bi, a[1]);
    }
    team.template publish<2>(a, 0);
    team.sync();
    double t2[2];
    team.template combine<2>(0, t2);
    if (team.leader()) p.res->true_rel = t2[1] > 0.0 ? sqrt(t2[0]) / sqrt(t2[1]) : sqrt(t2[0]);
  }
  team.sync();   // no block leaves while a peer may still read its shared memory
}

__global__ void batch_validate_kernel(int n_sys, const long long* row_off, const long long* nnz_off,
                                      const int* row_ptr, const int* col, const void* val, int f32,
                                      int need_diag, int* flags, double* diag) {
  // one thread per global row; find its system by binary search
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= row_off[n_sys]) return;
  int lo = 0, hi = n_sys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row_off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const int k = lo;
  const int n = (int)(row_off[k + 1] - row_off[k]);
  const int i = (int)(g - row_off[k]);
  const int* rp = row_ptr + row_off[k] + k;
  const long long nnz = nnz_off[k + 1] - nnz_off[k];
  int f = 0;
  const int e0 = rp[i], e1 = rp[i + 1];
  if (i == 0 && e0 != 0) f |= 1;
  if (i == n - 1 && (long long)e1 != nnz) f |= 1;
  if (e1 < e0 || e0 < 0 || (long long)e1 > nnz) { atomicOr(flags, f | 1); return; }
  double dg = 0.0;
  int prev = -1;
  for (int e = e0; e < e1; ++e) {
    const long long ge = nnz_off[k] + e;
    const int c = col[ge];
    if (c < 0 || c >= n || c <= prev) f |= 2;
    prev = c;
    const double v = f32 ? (double)((const float*)val)[ge] : ((const double*)val)[ge];
    if (!isfinite(v)) f |= 4;
    if (c == i) dg = v;
  }
  if (need_diag && dg == 0.0) f |= 8;
  diag[g] = dg;
  if (f) atomicOr(flags, f);
}

template <typename T, typename VR>
__global__ void batch_prepare_kernel(int n_sys, const long long* row_off, const long long* nnz_off,
                                     const int* row_ptr, const int* col, const VR* val, const double* diag,
                                     int jacobi, T* valAt, T* valAu, T* dinvT) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= row_off[n_sys]) return;
  int lo = 0, hi = n_sys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row_off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  const int k = lo;
  const long long r0 = row_off[k];
  const int i = (int)(g - r0);
  const int* rp = row_ptr + r0 + k;
  if (jacobi) dinvT[g] = T(1.0 / diag[g]);
  for (int e = rp[i]; e < rp[i + 1]; ++e) {
    const long long ge = nnz_off[k] + e;
    const double a = (double)val[ge];
    if (valAu) valAu[ge] = T(a);
    if (jacobi) valAt[ge] = T(a * (1.0 / diag[r0 + col[ge]]));
  }
}

}  // namespace

struct pbcg_batch_ctx {
  int n_sys = 0;
  long long total_rows = 0, total_nnz = 0;
  int precision = 0, vr_f32 = 0, prec = 0, degree = 0;
  pbcg_options opt{};
  cudaStream_t stream = nullptr, cap_stream = nullptr;
  long long *row_off = nullptr, *nnz_off = nullptr;
  int* order = nullptr;
  int *row_ptr = nullptr, *col = nullptr;
  void* valR = nullptr;
  void* valAu = nullptr;
  void* valAt = nullptr;
  void* dinv = nullptr;
  double* diag = nullptr;
  void* vecs = nullptr;
  DevResult* dres = nullptr;
  DevResult* hres = nullptr;
  unsigned* counter = nullptr;
  int* flags = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaGraphExec_t exec = nullptr;
  const double* g_b = nullptr;
  double* g_x = nullptr;
  int g_grid = 0, g_threads = 0, g_cluster = 0, g_lanes = 0;
  bool g_stream = false;
  int tuned_grid = 0, tuned_threads = 0, tuned_cluster = 0, tuned_lanes = 0;
  bool tuned_stream = false;
};

static void batch_free(pbcg_batch_ctx* c) {
  if (!c) return;
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->valAu == c->valR) c->valAu = nullptr;   // aliases the stored values
  void* ptrs[] = {c->row_off, c->nnz_off, c->order, c->row_ptr, c->col, c->valR, c->valAu, c->valAt, c->dinv,
                  c->diag, c->vecs, c->dres, c->counter, c->flags};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->hres) cudaFreeHost(c->hres);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

template <typename T, typename VR>
static const void* bkernel(bool cluster, bool stream) {
  if constexpr (std::is_same<T, float>::value) {
    if (stream && cluster) return (const void*)batched_cluster_kernel<T, VR, true>;
  }
  return cluster ? (const void*)batched_cluster_kernel<T, VR> : (const void*)batched_kernel<T, VR>;
}

// The one-block-per-system kernel, or (cluster = true) the cluster-per-system kernel
// (stream: its streaming build, mixed precision only).
static const void* pick_kernel(const pbcg_batch_ctx* c, bool cluster = false, bool stream = false) {
  const bool mixed = c->precision == PBCG_MIXED;
  if (mixed) return c->vr_f32 ? bkernel<float, float>(cluster, stream) : bkernel<float, double>(cluster, stream);
  return c->vr_f32 ? bkernel<double, float>(cluster, false) : bkernel<double, double>(cluster, false);
}

static BatchDev make_dev(pbcg_batch_ctx* c, const double* b, double* x, int lanes) {
  BatchDev d;
  memset(&d, 0, sizeof d);
  d.n_sys = c->n_sys;
  d.row_off = c->row_off;
  d.nnz_off = c->nnz_off;
  d.order = c->order;
  d.row_ptr = c->row_ptr;
  d.col = c->col;
  d.valAt = c->valAt ? c->valAt : c->valAu;
  d.valAu = c->valAu;
  d.valR = c->valR;
  d.dinv = c->dinv;
  d.b = b;
  d.x = x;
  d.vecs = c->vecs;
  d.total_rows = c->total_rows;
  d.res = c->dres;
  d.counter = c->counter;
  d.prec = c->prec;
  d.degree = c->degree;
  d.tol = c->opt.tol;
  d.max_it = c->opt.max_it;
  d.rr_period = c->opt.rr_period;
  d.rr_theta = c->opt.rr_theta;
  d.max_restarts = c->opt.max_restarts;
  d.restart_period = c->opt.restart_period;
  d.stag_window = c->opt.stag_window;
  d.rr_cutoff = c->opt.rr_cutoff > 0.0 ? c->opt.rr_cutoff : 1.4901161193847656e-08;   // sqrt(2^-52)
  d.lanes = lanes;
  return d;
}

#define BCK(call, what)                                  \
  do {                                                   \
    pbcg_status s__ = cuda_status((call), (what));       \
    if (s__ != PBCG_OK) return s__;                      \
  } while (0)

static void cluster_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute& attr, int grid, int threads, int cluster,
                           cudaStream_t s) {
  memset(&cfg, 0, sizeof cfg);
  memset(&attr, 0, sizeof attr);
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = (unsigned)cluster;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
}

static pbcg_status launch_direct(pbcg_batch_ctx* c, const double* b, double* x, int grid, int threads, int cluster,
                                 int lanes, bool stream, cudaStream_t s) {
  BCK(cudaMemsetAsync(c->counter, 0, sizeof(unsigned), s), "memset");
  BatchDev d = make_dev(c, b, x, lanes);
  void* args[] = {&d};
  if (cluster <= 1) {
    BCK(cudaLaunchKernel(pick_kernel(c), grid, threads, args, 0, s), "batched launch");
  } else {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr;
    cluster_config(cfg, attr, grid, threads, cluster, s);
    BCK(cudaLaunchKernelExC(&cfg, pick_kernel(c, true, stream), args), "batched cluster launch");
  }
  return PBCG_OK;
}

struct BatchShape {
  int grid, threads, cluster, lanes;
  bool stream;
};

// Clusters of `cluster` blocks that can be resident at once for this block size (0: none).
static pbcg_status active_clusters(const pbcg_batch_ctx* c, int threads, int cluster, int* n, bool stream = false) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr;
  cluster_config(cfg, attr, cluster, threads, cluster, c->stream);
  *n = 0;
  BCK(cudaOccupancyMaxActiveClusters(n, pick_kernel(c, true, stream), &cfg), "cluster occupancy");
  return PBCG_OK;
}

// Candidate launch shapes: one block per system at 256/512/1024 threads and 1-4 blocks per
// SM, and clusters of 2, 4 or 8 blocks per system at every resident cluster count; in mixed
// precision also the streaming cluster build where it fits more clusters (options.batch_build
// restricts the list to one build).
static pbcg_status candidate_shapes(const pbcg_batch_ctx* c, std::vector<BatchShape>& out, int only_cluster) {
  const int sms = sm_count();
  const int tlist[] = {256, 512, 1024};
  const int build = c->opt.batch_build;   // 0: both builds, 1: 64 registers only, 2: streaming only
  const bool want64 = build != 2;
  const bool want_stream = c->precision == PBCG_MIXED && build != 1;
  for (int t : tlist) {
    if (only_cluster <= 1 && want64) {
      int per = 0;
      BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pick_kernel(c), t, 0), "occupancy");
      for (int bps = 1; bps <= std::min(per, 4); ++bps) out.push_back({sms * bps, t, 1, 1, false});
    }
    for (int cl = 2; cl <= 8; cl *= 2) {
      if (only_cluster > 1 && cl != only_cluster) continue;
      if (only_cluster == 1) continue;
      int nc = 0;
      pbcg_status st = active_clusters(c, t, cl, &nc);
      if (st != PBCG_OK) return st;
      if (want64 && nc > 0) out.push_back({nc * cl, t, cl, 1, false});
      if (want_stream && t <= SolverLaunch<float, true>::kThreads) {   // only where it adds residency
        int ns = 0;
        st = active_clusters(c, t, cl, &ns, true);
        if (st != PBCG_OK) return st;
        if (ns > (want64 ? nc : 0)) out.push_back({ns * cl, t, cl, 1, true});
      }
    }
  }
  return PBCG_OK;
}

// Times one batch solve per candidate on a scratch copy of x: first the launch shapes with
// one thread per row, then 2, 4 and 8 threads per row in the SpMVs on the best shape
// (options.lanes_per_row fixes that choice).
static pbcg_status autotune(pbcg_batch_ctx* c, const double* b, double* x) {
  std::vector<BatchShape> cands;
  pbcg_status st = candidate_shapes(c, cands, c->opt.cluster_blocks);
  if (st != PBCG_OK) return st;
  double* xs = nullptr;
  BCK(cudaMallocAsync((void**)&xs, sizeof(double) * c->total_rows, c->stream), "autotune scratch");
  float best = 1e30f;
  auto trial = [&](const BatchShape& sh) -> pbcg_status {
    pbcg_status s2 = cuda_status(cudaMemcpyAsync(xs, x, sizeof(double) * c->total_rows, cudaMemcpyDeviceToDevice,
                                                 c->stream), "autotune copy");
    if (s2 == PBCG_OK) s2 = cuda_status(cudaEventRecord(c->ev0, c->stream), "event");
    if (s2 == PBCG_OK) s2 = launch_direct(c, b, xs, sh.grid, sh.threads, sh.cluster, sh.lanes, sh.stream, c->stream);
    if (s2 == PBCG_OK) s2 = cuda_status(cudaEventRecord(c->ev1, c->stream), "event");
    if (s2 == PBCG_OK) s2 = cuda_status(cudaEventSynchronize(c->ev1), "autotune");
    float ms = 0.f;
    if (s2 == PBCG_OK) s2 = cuda_status(cudaEventElapsedTime(&ms, c->ev0, c->ev1), "event timing");
    if (s2 != PBCG_OK) return s2;
    if (ms < best) {
      best = ms;
      c->tuned_grid = sh.grid; c->tuned_threads = sh.threads; c->tuned_cluster = sh.cluster; c->tuned_lanes = sh.lanes;
      c->tuned_stream = sh.stream;
    }
    return PBCG_OK;
  };
  const int fixed_lanes = c->opt.lanes_per_row;
  for (auto& sh : cands) {
    BatchShape s1 = sh;
    s1.lanes = fixed_lanes ? fixed_lanes : 1;
    if ((st = trial(s1)) != PBCG_OK) break;
  }
  if (st == PBCG_OK && !fixed_lanes) {
    const BatchShape base{c->tuned_grid, c->tuned_threads, c->tuned_cluster, 1, c->tuned_stream};
    for (int L = 2; L <= 8 && st == PBCG_OK; L *= 2) {
      BatchShape s2 = base;
      s2.lanes = L;
      st = trial(s2);
    }
  }
  cudaFreeAsync(xs, c->stream);
  if (st == PBCG_OK && !c->tuned_grid) return set_error(PBCG_CUDA_ERROR, "autotune found no launch shape that fits");
  return st;
}

extern "C" pbcg_status pbicgstab_batch_create(pbcg_batch_ctx** out, const pbcg_batch* B, const pbcg_options* opt,
                                              void* stream) {
  if (!out || !B || !opt) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_batch_create");
  *out = nullptr;
  if (B->n_sys < 1 || !B->row_off || !B->nnz_off || !B->row_ptr || !B->col || !B->val)
    return set_error(PBCG_INVALID_ARG, "batch needs n_sys >= 1 and all arrays");
  if (B->val_dtype != PBCG_F64 && B->val_dtype != PBCG_F32) return set_error(PBCG_INVALID_ARG, "unknown dtype");
  if (B->precond != PBCG_PREC_NONE && B->precond != PBCG_PREC_JACOBI && B->precond != PBCG_PREC_NEUMANN)
    return set_error(PBCG_INVALID_ARG, "batched solves support NONE, JACOBI and NEUMANN preconditioners");
  if (B->precond == PBCG_PREC_NEUMANN && (B->degree < 1 || B->degree > 8))
    return set_error(PBCG_INVALID_ARG, "Neumann degree must be in [1, 8]");
  if (opt->precision != PBCG_FP64 && opt->precision != PBCG_MIXED) return set_error(PBCG_INVALID_ARG, "bad precision");
  if (opt->max_it < 0 || !(opt->tol >= 0.0) || opt->rr_period < 0 || !(opt->rr_theta >= 0.0 && opt->rr_theta < 1.0) ||
      opt->rr_auto != 0)
    return set_error(PBCG_INVALID_ARG, "bad solver options");
  if (opt->method != PBCG_PIPELINED) return set_error(PBCG_INVALID_ARG, "batched solves run Algorithm 2 only (PBCG_PIPELINED)");
  if (opt->block_threads != 0 && (opt->block_threads < 32 || opt->block_threads > kMaxThreads || opt->block_threads % 32))
    return set_error(PBCG_INVALID_ARG, "block_threads must be 0 or a multiple of 32 in [32, 1024]");
  if (opt->max_restarts < 0 || opt->max_restarts > 1000) return set_error(PBCG_INVALID_ARG, "max_restarts must be in [0, 1000]");
  if (opt->restart_period < 0 || opt->stag_window < 0 || !(opt->rr_cutoff >= 0.0 && opt->rr_cutoff < 1.0))
    return set_error(PBCG_INVALID_ARG, "restart_period and stag_window must be >= 0, rr_cutoff in [0, 1)");
  if (opt->cluster_blocks != 0 && opt->cluster_blocks != 1 && opt->cluster_blocks != 2 && opt->cluster_blocks != 4 &&
      opt->cluster_blocks != 8)
    return set_error(PBCG_INVALID_ARG, "cluster_blocks must be 0, 1, 2, 4 or 8");
  if (opt->lanes_per_row != 0 && opt->lanes_per_row != 1 && opt->lanes_per_row != 2 && opt->lanes_per_row != 4 &&
      opt->lanes_per_row != 8)
    return set_error(PBCG_INVALID_ARG, "lanes_per_row must be 0, 1, 2, 4 or 8");
  if (opt->batch_build < 0 || opt->batch_build > 2) return set_error(PBCG_INVALID_ARG, "batch_build must be 0, 1 or 2");
  if (opt->batch_build == 2 && (opt->precision != PBCG_MIXED || opt->cluster_blocks == 1 ||
                                opt->block_threads > SolverLaunch<float, true>::kThreads))
    return set_error(PBCG_INVALID_ARG, "the streaming build (batch_build 2) runs mixed precision in clusters of "
                                       "2, 4 or 8 blocks of at most %d threads", SolverLaunch<float, true>::kThreads);
  const int ns = B->n_sys;
  if (B->row_off[0] != 0 || B->nnz_off[0] != 0) return set_error(PBCG_INVALID_ARG, "offsets must start at 0");
  for (int k = 0; k < ns; ++k) {
    const long long nk = B->row_off[k + 1] - B->row_off[k];
    if (nk < 1 || nk > PBCG_MAX_ROWS) return set_error(PBCG_INVALID_ARG, "system %d has an invalid size", k);
    if (B->nnz_off[k + 1] < B->nnz_off[k]) return set_error(PBCG_INVALID_ARG, "nnz offsets must not decrease");
  }
  pbcg_batch_ctx* c = new (std::nothrow) pbcg_batch_ctx();
  if (!c) return set_error(PBCG_OUT_OF_MEMORY, "host allocation failed");
#define CKB(call, what)                                  \
  do {                                                   \
    pbcg_status s__ = cuda_status((call), (what));       \
    if (s__ != PBCG_OK) { batch_free(c); return s__; }   \
  } while (0)
  c->n_sys = ns;
  c->total_rows = B->row_off[ns];
  c->total_nnz = B->nnz_off[ns];
  c->precision = opt->precision;
  c->vr_f32 = B->val_dtype == PBCG_F32;
  c->prec = B->precond;
  c->degree = B->precond == PBCG_PREC_NEUMANN ? B->degree : 0;
  c->opt = *opt;
  c->stream = (cudaStream_t)stream;
  const size_t es = c->precision == PBCG_MIXED ? 4 : 8;
  const size_t vs = c->vr_f32 ? 4 : 8;
  const long long R = c->total_rows, E = std::max<long long>(1, c->total_nnz);
  CKB(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "stream");
  CKB(cudaEventCreate(&c->ev0), "event");
  CKB(cudaEventCreate(&c->ev1), "event");
  CKB(cudaMalloc(&c->row_off, sizeof(long long) * (ns + 1)), "cudaMalloc");
  CKB(cudaMalloc(&c->nnz_off, sizeof(long long) * (ns + 1)), "cudaMalloc");
  CKB(cudaMalloc(&c->order, sizeof(int) * ns), "cudaMalloc");
  CKB(cudaMalloc(&c->row_ptr, sizeof(int) * (R + ns)), "cudaMalloc");
  CKB(cudaMalloc(&c->col, sizeof(int) * E), "cudaMalloc");
  CKB(cudaMalloc(&c->valR, vs * E), "cudaMalloc");
  CKB(cudaMalloc(&c->diag, sizeof(double) * R), "cudaMalloc");
  CKB(cudaMalloc(&c->flags, sizeof(int)), "cudaMalloc");
  CKB(cudaMalloc(&c->counter, sizeof(unsigned)), "cudaMalloc");
  CKB(cudaMalloc(&c->dres, sizeof(DevResult) * ns), "cudaMalloc");
  CKB(cudaMallocHost(&c->hres, sizeof(DevResult) * ns), "cudaMallocHost");
  CKB(cudaMalloc(&c->vecs, es * 15 * (size_t)R), "cudaMalloc workspace");
  std::vector<int> order(ns);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (B->row_off[a + 1] - B->row_off[a]) > (B->row_off[b + 1] - B->row_off[b]);
  });
  cudaStream_t s = c->stream;
  CKB(cudaMemcpyAsync(c->row_off, B->row_off, sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice, s), "copy");
  CKB(cudaMemcpyAsync(c->nnz_off, B->nnz_off, sizeof(long long) * (ns + 1), cudaMemcpyHostToDevice, s), "copy");
  CKB(cudaMemcpyAsync(c->order, order.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s), "copy");
  CKB(cudaMemcpyAsync(c->row_ptr, B->row_ptr, sizeof(int) * (R + ns), cudaMemcpyDeviceToDevice, s), "copy");
  if (c->total_nnz) {
    CKB(cudaMemcpyAsync(c->col, B->col, sizeof(int) * c->total_nnz, cudaMemcpyDeviceToDevice, s), "copy");
    CKB(cudaMemcpyAsync(c->valR, B->val, vs * c->total_nnz, cudaMemcpyDeviceToDevice, s), "copy");
  }
  CKB(cudaMemsetAsync(c->flags, 0, sizeof(int), s), "memset");
  const unsigned nb = (unsigned)((R + 255) / 256);
  // Jacobi and Neumann both need D^{-1} and the folded A D^{-1} (the first Neumann sweep)
  const int jac = c->prec != PBCG_PREC_NONE;
  batch_validate_kernel<<<nb, 256, 0, s>>>(ns, c->row_off, c->nnz_off, c->row_ptr, c->col, c->valR, c->vr_f32, jac,
                                           c->flags, c->diag);
  CKB(cudaGetLastError(), "batch validation launch");
  int hflags = 0;
  CKB(cudaMemcpyAsync(&hflags, c->flags, sizeof(int), cudaMemcpyDeviceToHost, s), "copy flags");
  CKB(cudaStreamSynchronize(s), "batch validation");
  if (hflags) {
    batch_free(c);
    if (hflags & 1) return set_error(PBCG_INVALID_ARG, "a system's row_ptr is not monotone from 0 to its nnz");
    if (hflags & 2) return set_error(PBCG_INVALID_ARG, "a column index is out of range or not increasing");
    if (hflags & 4) return set_error(PBCG_INVALID_ARG, "a matrix value is not finite");
    return set_error(PBCG_INVALID_ARG, "Jacobi and Neumann need a non-zero diagonal in every row");
  }
  // values in T: the unfolded copy (mixed with FP64 input, or FP64 with FP32 input) and A D^{-1}
  const bool need_au = (c->precision == PBCG_MIXED) != (bool)c->vr_f32;
  if (need_au) CKB(cudaMalloc(&c->valAu, es * E), "cudaMalloc");
  else c->valAu = nullptr;
  if (jac) {
    CKB(cudaMalloc(&c->valAt, es * E), "cudaMalloc");
    CKB(cudaMalloc(&c->dinv, es * R), "cudaMalloc");
  }
  if (c->precision == PBCG_MIXED) {
    if (c->vr_f32)
      batch_prepare_kernel<float, float><<<nb, 256, 0, s>>>(ns, c->row_off, c->nnz_off, c->row_ptr, c->col,
          (const float*)c->valR, c->diag, jac, (float*)c->valAt, (float*)nullptr, (float*)c->dinv);
    else
      batch_prepare_kernel<float, double><<<nb, 256, 0, s>>>(ns, c->row_off, c->nnz_off, c->row_ptr, c->col,
          (const double*)c->valR, c->diag, jac, (float*)c->valAt, (float*)c->valAu, (float*)c->dinv);
  } else {
    if (c->vr_f32)
      batch_prepare_kernel<double, float><<<nb, 256, 0, s>>>(ns, c->row_off, c->nnz_off, c->row_ptr, c->col,
          (const float*)c->valR, c->diag, jac, (double*)c->valAt, (double*)c->valAu, (double*)c->dinv);
    else
      batch_prepare_kernel<double, double><<<nb, 256, 0, s>>>(ns, c->row_off, c->nnz_off, c->row_ptr, c->col,
          (const double*)c->valR, c->diag, jac, (double*)c->valAt, (double*)nullptr, (double*)c->dinv);
  }
  if (!need_au) c->valAu = nullptr;
  CKB(cudaGetLastError(), "batch prepare");
  CKB(cudaStreamSynchronize(s), "batch prepare");
  if (!c->valAu) c->valAu = c->valR;   // same precision: the stored values serve directly
  *out = c;
  return PBCG_OK;
#undef CKB
}

static pbcg_status ensure_graph(pbcg_batch_ctx* c, const double* b, double* x, int grid, int threads, int cluster,
                                int lanes, bool stream) {
  if (c->exec && c->g_b == b && c->g_x == x && c->g_grid == grid && c->g_threads == threads && c->g_cluster == cluster &&
      c->g_lanes == lanes && c->g_stream == stream)
    return PBCG_OK;
  if (c->exec) { cudaGraphExecDestroy(c->exec); c->exec = nullptr; }
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  pbcg_status st = launch_direct(c, b, x, grid, threads, cluster, lanes, stream, c->cap_stream);
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
  if (st != PBCG_OK) { if (graph) cudaGraphDestroy(graph); return st; }
  BCK(e, "end capture");
  e = cudaGraphInstantiate(&c->exec, graph, 0);
  cudaGraphDestroy(graph);
  BCK(e, "graph instantiate");
  c->g_b = b;
  c->g_x = x;
  c->g_grid = grid;
  c->g_threads = threads;
  c->g_cluster = cluster;
  c->g_lanes = lanes;
  c->g_stream = stream;
  return PBCG_OK;
}

extern "C" pbcg_status pbicgstab_batch_solve(pbcg_batch_ctx* c, const double* b, double* x, pbcg_batch_result* res) {
  if (!c || !b || !x) return set_error(PBCG_INVALID_ARG, "NULL argument to pbicgstab_batch_solve");
  int grid = c->opt.grid_blocks, threads = c->opt.block_threads, cluster = std::max(1, c->opt.cluster_blocks);
  int lanes = std::max(1, c->opt.lanes_per_row);
  bool stream = c->opt.batch_build == 2;   // caller-fixed shapes: the 64-register builds unless asked
  if (grid == 0 || threads == 0) {
    if (!c->tuned_grid) {
      pbcg_status st = autotune(c, b, x);
      if (st != PBCG_OK) return st;
    }
    grid = c->tuned_grid;
    threads = c->tuned_threads;
    cluster = c->tuned_cluster;
    lanes = c->tuned_lanes;
    stream = c->tuned_stream;
  } else if (stream && cluster <= 1) {
    return set_error(PBCG_INVALID_ARG, "the streaming build runs clusters: cluster_blocks must be 2, 4 or 8");
  } else if (cluster > 1) {
    int nc = 0;
    pbcg_status st = active_clusters(c, threads, cluster, &nc, stream);
    if (st != PBCG_OK) return st;
    if (grid % cluster || grid / cluster > nc)
      return set_error(PBCG_INVALID_ARG, "grid_blocks must be a multiple of the cluster size and fit on the GPU");
  }
  pbcg_status st = ensure_graph(c, b, x, grid, threads, cluster, lanes, stream);
  if (st != PBCG_OK) return st;
  BCK(cudaEventRecord(c->ev0, c->stream), "event");
  BCK(cudaGraphLaunch(c->exec, c->stream), "graph launch");
  BCK(cudaEventRecord(c->ev1, c->stream), "event");
  if (!res) return PBCG_OK;
  BCK(cudaMemcpyAsync(c->hres, c->dres, sizeof(DevResult) * c->n_sys, cudaMemcpyDeviceToHost, c->stream), "copy");
  BCK(cudaStreamSynchronize(c->stream), "batched solve");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  res->time_ms = ms;
  res->block_threads = threads;
  res->grid_blocks = grid;
  res->cluster_blocks = cluster;
  res->lanes_per_row = lanes;
  res->batch_build = stream ? 2 : 1;
  int nok = 0;
  pbcg_status first_bad = PBCG_OK;
  for (int k = 0; k < c->n_sys; ++k) {
    const DevResult& r = c->hres[k];
    if (res->status) res->status[k] = r.status;
    if (res->iterations) res->iterations[k] = r.iterations;
    if (res->n_replacements) res->n_replacements[k] = r.nrep;
    if (res->rel_res_true) res->rel_res_true[k] = r.true_rel;
    if (r.status == PBCG_OK) ++nok;
    else if (first_bad == PBCG_OK) first_bad = (pbcg_status)r.status;
  }
  res->n_ok = nok;
  return first_bad;
}

extern "C" pbcg_status pbicgstab_batch_destroy(pbcg_batch_ctx* c) {
  if (!c) return PBCG_OK;
  cudaStreamSynchronize(c->stream);
  batch_free(c);
  return PBCG_OK;
}

extern "C" pbcg_status pbicgstab_solve_batched(const pbcg_batch* B, const pbcg_options* opt, void* stream,
                                               const double* b, double* x, pbcg_batch_result* res) {
  pbcg_batch_ctx* c = nullptr;
  pbcg_status st = pbicgstab_batch_create(&c, B, opt, stream);
  if (st != PBCG_OK) return st;
  st = pbicgstab_batch_solve(c, b, x, res);
  if (!res) cudaStreamSynchronize((cudaStream_t)stream);
  pbicgstab_batch_destroy(c);
  return st;
}
