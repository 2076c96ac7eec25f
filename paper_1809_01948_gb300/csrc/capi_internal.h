// Internal declarations shared by the host translation units of libpbicgstab.
#pragma once
#include <cstdarg>
#include <algorithm>
#include <type_traits>
#include <cuda_runtime.h>
#include <cmath>
#include <cstring>
#include "../../include/pbicgstab.h"
#include "solver.cuh"

namespace pbcg {
// Entry points of the persistent solver kernels (kernels_f64.cu, kernels_f32.cu,
// kernels_vec.cu; compiled as separate translation units).  automated: Eq. (criterion)
// policy; scalar: scaled-form Jacobi of a constant diagonal; stream: the 40-register mixed
// build; vec: four rows per thread in the hot passes.
const void* pipelined_kernel_f64(bool automated, bool scalar, bool vec);
const void* pipelined_kernel_f32(bool automated, bool stream, bool scalar, bool vec);
const void* classic_kernel_f64(bool scalar);
const void* pipelined_kernel_f64_vec(bool scalar);
const void* pipelined_kernel_f32_vec(bool scalar, bool stream);
pbcg_status set_error(pbcg_status st, const char* fmt, ...);
pbcg_status cuda_status(cudaError_t e, const char* what);
int sm_count();
}  // namespace pbcg

using pbcg::MatView;
using pbcg::SolverParams;
using pbcg::DevResult;
using pbcg::kMaxDiag;
using pbcg::kMaxDots;
using pbcg::kMaxThreads;

struct DevState {
  DevResult res;
  unsigned bar;
  int err;
  double true_rel;
  int flags;
  int reserved;                   // validation: max |col - row|
  int maxnnz;                     // validation: max stored entries in a row
  int reserved2;
  unsigned long long maxabs_bits; // bit patterns of non-negative doubles order like the values
  unsigned long long rowsum_bits;
  unsigned long long colsum_max;  // max column sum in fixed point
  unsigned long long dinv_bits;
};

struct pbcg_ctx {
  int n = 0;
  long long nnz = 0;
  int fmt = 0;
  int precision = 0;
  int prec_kind = 0;
  int degree = 0;
  cudaStream_t stream = nullptr;
  pbcg_options opt{};
  // matrix (device, owned)
  int* row_ptr = nullptr;
  int* col = nullptr;
  double* val64 = nullptr;   // FP64 values (CSR nnz, DIA ndiag*n)
  void* valAt = nullptr;     // hot operator values in T
  void* valAu = nullptr;     // A in T (mixed: FP32 copy; FP64: aliases val64)
  double* diag64 = nullptr;
  double* dinv64 = nullptr;
  void* dinvT = nullptr;
  int ndiag = 0;
  int offsets[kMaxDiag] = {0};
  int ndiag_t = 0;           // diagonals stored in valAt (DIA fold drops the main one)
  int offsets_t[kMaxDiag] = {0};
  int at_unit_diag = 0;
  int bandwidth = 0;         // max |col - row| over the stored entries
  int maxnnz = 0;            // max stored entries in a row
  // constant-coefficient stencil form of A (options.operator_storage auto, when every
  // offset carries one value and the diagonal is constant): views use these instead of
  // the stored values
  int stencil = 0;
  int st_n = 0;                          // offsets, ascending
  int st_off[kMaxDiag] = {0};
  double st_val[kMaxDiag] = {0};         // A's value at each offset
  double st_dinv = 0.0;                  // 1 / (the constant diagonal)
  unsigned short* st_mask = nullptr;     // per row: bit d set when the entry at st_off[d] is present
  int dconst = 0;            // the diagonal is one value d (every row, non-zero)
  double dconst_inv = 0.0;   // 1 / d
  double norm_bound = 0.0;   // sqrt(||A||_1 ||A||_inf) (upper bound of ||A||_2)
  double dinv_max = 1.0;     // max |d_inv| in the working precision (1 without preconditioner)
  // vectors + reductions
  void* vecs = nullptr;
  int nvec = 15;
  double* part = nullptr;
  int max_blocks = 0;
  DevState* dstate = nullptr;
  DevState* hstate = nullptr;  // pinned
  double* xbest = nullptr;     // best (re)start iterate of options.stag_window (n doubles)
  int launch[4] = {0, 0, 0, 0};  // last solve: grid, threads, rows per thread, prefetch distance
  int valid = 1;               // 0 after a failed pbicgstab_update_values: solves are refused
  int* tperm = nullptr;        // transpose contexts: entry e of A^T is entry tperm[e] of the source
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // multi-RHS workspace (grown on demand by pbicgstab_solve_multi)
  int multi_cap = 0;           // right-hand sides the buffers below hold
  void* multi_vecs = nullptr;  // multi_cap * 15 * n values of T
  double* multi_part = nullptr;
  DevState* multi_state = nullptr;
  DevState* multi_hstate = nullptr;   // pinned
  void* multi_params = nullptr;       // multi_cap SolverParams<T>
  void* multi_hparams = nullptr;      // pinned staging copy
};

inline size_t elem_size(int precision) { return precision == PBCG_MIXED ? sizeof(float) : sizeof(double); }

// Stencil view of A (hot = false: values of A rounded to V) or of the Jacobi-folded
// operator A D^{-1} (hot = true: a_ij * d_inv rounded once to V, as the fold kernels
// compute it; the DIA fold's unit main diagonal is implicit, the CSR fold keeps it).
template <typename V>
inline MatView<V> make_stencil_view(const pbcg_ctx* c, bool hot) {
  MatView<V> m;
  memset(&m, 0, sizeof m);
  m.fmt = 2;
  m.n = c->n;
  m.mask = c->st_mask;
  int k = 0;
  for (int d = 0; d < c->st_n; ++d) {
    if (hot && c->fmt == PBCG_FMT_DIA && c->st_off[d] == 0) continue;
    m.off[k] = c->st_off[d];
    m.cval[k] = hot ? V(c->st_val[d] * c->st_dinv) : V(c->st_val[d]);
    m.mbit[k] = (unsigned char)d;
    ++k;
  }
  m.ndiag = k;
  m.unit_diag = (hot && c->fmt == PBCG_FMT_DIA) ? 1 : 0;
  m.pattern = pbcg::stencil_pattern(m.off, m.ndiag);
  return m;
}

template <typename V>
inline MatView<V> make_view(const pbcg_ctx* c, const V* val, bool hot) {
  if (c->stencil) return make_stencil_view<V>(c, hot);
  MatView<V> m;
  memset(&m, 0, sizeof m);
  m.fmt = c->fmt;
  m.n = c->n;
  m.row_ptr = c->row_ptr;
  m.col = c->col;
  m.val = val;
  if (c->fmt == PBCG_FMT_DIA) {
    if (hot) {
      m.ndiag = c->ndiag_t;
      m.unit_diag = c->at_unit_diag;
      for (int d = 0; d < c->ndiag_t; ++d) m.off[d] = c->offsets_t[d];
    } else {
      m.ndiag = c->ndiag;
      for (int d = 0; d < c->ndiag; ++d) m.off[d] = c->offsets[d];
    }
  }
  return m;
}

inline MatView<double> pbcg_view64(const pbcg_ctx* c) { return make_view<double>(c, c->val64, false); }


pbcg_status check_options(const pbcg_options* o, long long n);
pbcg_status build_stencil(pbcg_ctx* c);
pbcg_status launch_shape(const pbcg_ctx* c, int* grid, int* threads, bool vec);
bool quad_rows(const pbcg_ctx* c, const double* b, const double* x);
pbcg_status enqueue_true_residual(pbcg_ctx* c, const double* b, const double* x, double* out_dev);

int l2_bytes();   // L2 size of the current device in bytes

// Bytes an iteration streams repeatedly: the work vectors it touches (about 12), x, and
// the operator (the stencil mask, or the stored values and indices).
// Jacobi with a constant diagonal runs in scaled form (the SCALAR kernel builds).
inline bool scalar_jacobi(const pbcg_ctx* c) {
  return c->prec_kind == PBCG_PREC_JACOBI && c->dconst && !c->opt.rr_auto;
}

// The grid barrier counts arrivals in 32 bits (barrier index x blocks).  An iteration
// crosses at most 4d + 6 barriers (d = Neumann degree: two preconditioner applications,
// passes A and B, a replacement and a failed stop test), a (re)start d + 2; keep the
// solve's total times the blocks below 2^31 so the count cannot wrap.  With a restart
// policy every iteration may end in a restart (a failed stop-test verification restarts).
inline pbcg_status check_barrier_budget(int max_it, int max_restarts, int degree, int blocks,
                                        int restart_period = 0, int stag_window = 0) {
  const long long start = 4 + 2LL * degree;
  const long long per_it = 8 + 4LL * degree + (restart_period > 0 ? start : 0);
  const long long fixed = start * ((long long)max_restarts + 1 + (restart_period > 0 ? 1 : 0)) +
                          (stag_window > 0 ? 2 : 0);
  const long long budget = ((1LL << 31) - 1) / blocks;       // barriers the counter allows
  if (((long long)max_it + 1) * per_it + fixed > budget)
    return pbcg::set_error(PBCG_INVALID_ARG, "max_it %d is too large for %d blocks per barrier (at most %lld)",
                           max_it, blocks, (budget - fixed) / per_it - 1);
  return PBCG_OK;
}

inline double hot_bytes(const pbcg_ctx* c) {
  const double es = (double)elem_size(c->precision);
  double op;
  if (c->stencil) op = 2.0;
  else if (c->fmt == PBCG_FMT_DIA) op = c->ndiag * es;
  else op = (double)c->nnz / std::max(1, c->n) * (es + 4.0) + 4.0;
  return (double)c->n * (12.0 * es + 16.0 + op);
}

// vec: the four-row kernels, whose per-block chunks start at multiples of 4.
template <typename T>
inline SolverParams<T> make_params(pbcg_ctx* c, const double* b, double* x, int grid, bool vec = false) {
  SolverParams<T> p;
  memset(&p, 0, sizeof p);
  const int n = c->n;
  p.n = n;
  p.chunk = (n + grid - 1) / grid;
  if (vec) p.chunk = (p.chunk + 3) / 4 * 4;
  const T* at = c->valAt ? (const T*)c->valAt : (const T*)c->valAu;
  p.At = make_view<T>(c, at, c->valAt != nullptr);
  if (!c->valAt && c->fmt == PBCG_FMT_DIA) p.At = make_view<T>(c, at, false);
  p.Au = make_view<T>(c, (const T*)c->valAu, false);
  p.A64 = make_view<double>(c, c->val64, false);
  p.dinv = (c->prec_kind == PBCG_PREC_NONE || c->stencil) ? nullptr
           : (std::is_same<T, float>::value ? (const T*)c->dinvT : (const T*)c->dinv64);
  p.dinv_c = T(c->st_dinv);
  p.dinv_x = c->dconst ? c->dconst_inv : 1.0;
  p.prec = c->prec_kind;
  p.degree = c->degree;
  p.b = b;
  p.x = x;
  T* v = (T*)c->vecs;
  T** slots[] = {&p.r, &p.rh, &p.k, &p.w, &p.g, &p.s, &p.l, &p.z, &p.v, &p.t, &p.nb, &p.m, &p.nn, &p.tmpa, &p.tmpb};
  for (int j = 0; j < 15; ++j) *slots[j] = v + (size_t)j * n;
  p.part = c->part;
  p.bar = &c->dstate->bar;
  p.err = &c->dstate->err;
  p.res = &c->dstate->res;
  p.hist_x = c->opt.hist_x;
  p.K = c->opt.record_iterates;
  p.hist_s = c->opt.hist_scalars;
  p.hist_len = c->opt.hist_len;
  p.tol = c->opt.tol;
  p.max_it = c->opt.max_it;
  p.rr_period = c->opt.rr_period;
  p.rr_theta = c->opt.rr_theta;
  const double tms = c->opt.timeout_ms > 0 ? c->opt.timeout_ms : 2000.0;
  p.timeout_ns = (unsigned long long)(tms * 1e6);
  p.max_restarts = c->opt.max_restarts;
  p.restart_period = c->opt.restart_period;
  p.stag_window = c->opt.stag_window;
  p.xbest = c->xbest;
  p.rr_cutoff = c->opt.rr_cutoff > 0.0 ? c->opt.rr_cutoff : 1.4901161193847656e-08;   // sqrt(2^-52)
  p.strided = c->bandwidth > p.chunk / 2 ? 1 : 0;
  p.halo = c->bandwidth;
  p.overlap = (c->opt.barrier_overlap >= 0 && !p.strided && c->prec_kind != PBCG_PREC_NEUMANN &&
               c->opt.method == PBCG_PIPELINED && !c->opt.rr_auto && grid > 1 && p.chunk > 2 * c->bandwidth) ? 1 : 0;
  // stencil storage only: with CSR / DIA values the row products already keep several
  // loads per row in flight (measured slower with the prefetch on the 3D CSR operator)
  // automatic: the one-row kernels of a stencil system whose working set exceeds L2 (the
  // four-row kernels keep enough loads in flight without it: measured no faster with it)
  p.prefetch = (c->stencil && !vec && hot_bytes(c) > (double)l2_bytes()) ? 1 : 0;
  if (c->opt.prefetch_trips != 0) p.prefetch = c->opt.prefetch_trips > 0 ? c->opt.prefetch_trips : 0;
  p.rr_tau = c->opt.rr_tau > 0.0 ? c->opt.rr_tau : 1.4901161193847656e-08;
  p.bnd_msn = (double)c->maxnnz * sqrt((double)n);
  p.bnd_tmsn = sqrt((double)n);
  p.bnd_nA = c->norm_bound;
  p.bnd_nM = c->dinv_max;
  p.bnd_eps = std::is_same<T, float>::value ? 1.1920928955078125e-07 : 2.220446049250313e-16;
  return p;
}


