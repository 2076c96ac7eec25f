// Persistent, cooperatively launched p-BiCGStab kernel (Algorithm 2 of arXiv
// 1809.01948 with the residual replacement step of Eq. (rr)).
//
// One launch runs the whole solve.  Rows are split into one contiguous chunk per
// block.  Each iteration is two fused passes separated by grid barriers; each pass
// is an SPMV fused with the AXPY recurrences and the partial dot products of one
// global reduction phase, so the paper's overlap of each global reduction with an SPMV
// and a preconditioner application becomes: the reduction completes at the barrier
// the next SPMV needs anyway.
//
//   pass A: t_i = A m_i (the product the paper forms during the previous iteration's
//          second reduction), then g, s, l, z, q, u, y and partials of (q,y), (y,y)
//   pass B: v_i = A n_i, omega_i, then x, r, k, w (q, u, y recomputed
//          bit-identically instead of stored) and partials of (r0,r_{i+1}),
//          (r0,w_{i+1}), (r0,s_i), (r0,z_i), (r_{i+1},r_{i+1})
//
// Jacobi / no preconditioner: m = D^{-1} w and n = D^{-1} z are formed on the fly and
// the SPMVs use the folded operator A D^{-1} (t = A D^{-1} w = A m), so each
// iteration has exactly two grid barriers.  Neumann(d): m and n are stored and each
// M^{-1} application adds d barrier-separated Jacobi-sweep passes.
//
// Every block computes the scalars alpha, beta, omega from the same partials in the
// same order, so all blocks take identical control-flow decisions without any
// extra synchronisation.
#pragma once
#include <type_traits>
#include "common.cuh"

namespace pbcg {

struct DevResult {
  int status;
  int iterations;
  int nrep;
  int nrestart;
  double rn_rel;   // ||r_last|| / ||b||
  double bnorm;
  double rn0;
  double true_rel; // set when the in-kernel true residual was evaluated (else -1)
};

template <typename T, typename VR = double>
struct SolverParams {
  int n, chunk;
  MatView<T> At;        // hot operator: A D^{-1} (Jacobi, and Neumann's first sweep) or A (none)
  MatView<T> Au;        // A in the vector precision (Neumann sweeps, t = A m, v = A n)
  MatView<VR> A64;      // A with its stored values (FP64, or FP32 widened exactly): initial
                        // and replacement residuals, evaluated in FP64
  const T* dinv;        // D^{-1} (nullptr without preconditioner or when D is constant)
  T dinv_c;             // D^{-1} of a constant diagonal (used when dinv is nullptr)
  double dinv_x;        // 1/d of a constant diagonal, for the scaled-form (SCALAR) kernels
  int prec;             // 0 none, 1 Jacobi, 2 Neumann
  int degree;
  const double* b;
  double* x;
  T *r, *rh, *k, *w, *g, *s, *l, *z, *v, *t, *nb, *m, *nn, *tmpa, *tmpb;
  double* part;         // grid team: 3 partial sets of (team blocks) * kMaxDots doubles
  unsigned* bar;
  int* err;
  DevResult* res;
  double* hist_x;
  int K;
  double* hist_s;
  int hist_len;
  double tol;
  int max_it;
  int rr_period;
  double rr_theta;
  unsigned long long timeout_ns;
  int max_restarts;     // restarts from the current iterate allowed after a breakdown
  int strided;          // grid team row order: 1 grid-stride, 0 one contiguous chunk per block
  int prefetch;         // > 0: request the operands of the row sweep this many trips ahead into L2
  int staged;           // > 0: the four-row FP32 Neumann sweeps stage their operands in dynamic
                        // shared memory (the kernel's launch provides two stages)
  int overlap;          // 1: compute the next SpMV on a block's interior rows inside each grid
                        // barrier (chunked row order, no Neumann); 0: plain barriers
  int halo;             // max |col - row| of A: rows farther than this from a block's chunk
                        // ends have all their SpMV operands in the block's own rows
  int restart_period;   // > 0: restart from the current iterate every P iterations (reading R20)
  int stag_window;      // > 0: progress-based stagnation (reading R21)
  double* xbest;        // FP64 n-vector for R21's best iterate, or nullptr (no fallback)
  double rr_cutoff;     // periodic replacements stop once ||r_i|| < rr_cutoff ||r_0||
  // automated replacement, Eq. (criterion) with the gap bound f^r of Eq. (DDr_bound)
  // (read only by kernels instantiated with AUTO = true)
  double rr_tau;
  double bnd_msn;       // mu sqrt(N), mu = max stored entries in a row of A
  double bnd_tmsn;      // mu~ sqrt(N), mu~ = max entries in a row of M^{-1} (1: Jacobi / none)
  double bnd_nA;        // upper bound of ||A||_2: sqrt(||A||_1 ||A||_inf)
  double bnd_nM;        // ||M^{-1}||_2 = max |d_inv| (Jacobi) or 1
  double bnd_eps;       // 2^-52, or 2^-23 for the FP32 recurrences of mixed mode
};

// ---------------------------------------------------------------------------
// Run-time gap bound f^r for the automated replacement policy (Section 3.6):
// Eq. (DDr_bound) with the local-error norms replaced by their bounds
// Eq. (errbounds1)-(errbounds4) and the gaps of s, w, z by the triangle-inequality
// bounds F^s, F^w, F^z of Eqs. (Ds), (Dw), (Dz).  Only thread 0 of a team runs these
// (scalar FP64 work); the decision is broadcast.
struct GapBound {
  double f, Fz, Fs, Fw, f_pending, f_prev, rn_prev, rn_cur;
  double pg, ps, pl, pz, pn, pv;   // norms of g, s, l, z, n, v of the previous iteration
  int first, have_prev;
};

// indices of the 15 iteration-i norms handed to gb_step
enum { NX = 0, NR, NK, NW, NG, NS, NL, NZ, NQ, NU, NY, NM, NT, NN, NV, NNORMS };

template <typename T, typename VR>
__device__ void gb_start(GapBound& S, const SolverParams<T, VR>& p, double xnorm, double bn, double rn) {
  S.f = ((p.bnd_msn + 1.0) * p.bnd_nA * xnorm + bn) * p.bnd_eps;   // initial gap of r_0 = fl(b - A x0)
  S.Fz = S.Fs = S.Fw = 0.0;
  S.pg = S.ps = S.pl = S.pz = S.pn = S.pv = 0.0;
  S.first = 1;
  S.have_prev = 0;
  S.rn_cur = rn;
}

// Eq. (criterion): replace in iteration i when f_{i-1} <= tau ||r_{i-1}|| and f_i > tau ||r_i||.
__device__ __forceinline__ bool gb_criterion(const GapBound& S, double tau) {
  return S.have_prev && S.f_prev <= tau * S.rn_prev && S.f > tau * S.rn_cur;
}

template <typename T, typename VR>
__device__ void gb_step(GapBound& S, const SolverParams<T, VR>& p, const double* c, double alpha, double beta,
                        double omega, double omega_prev) {
  const double msn = p.bnd_msn, tmsn = p.bnd_tmsn, nA = p.bnd_nA, nM = p.bnd_nM, eps = p.bnd_eps;
  const double a = fabs(alpha), b = fabs(beta), o = fabs(omega), op = fabs(omega_prev);
  const double bo = b * op, oa = o * a;
  const double Pg = S.first ? 0.0 : S.pg, Ps = S.first ? 0.0 : S.ps, Pl = S.first ? 0.0 : S.pl;
  const double Pz = S.first ? 0.0 : S.pz, Pn = S.first ? 0.0 : S.pn, Pv = S.first ? 0.0 : S.pv;
  // Eq. (errbounds1)-(errbounds4)
  const double dg = (c[NK] + 3 * b * Pg + 4 * bo * Pl) * eps;
  const double dx = (2 * c[NX] + 3 * a * c[NG] + 2 * o * c[NU]) * eps;
  const double ds = (c[NW] + 3 * b * Ps + 4 * bo * Pz) * eps;
  const double dr = (c[NQ] + 2 * o * c[NY]) * eps;
  const double dl = (c[NM] + tmsn * nM * c[NW] + 3 * b * Pl + 4 * bo * Pn + tmsn * nM * bo * Pz) * eps;
  const double dz = (c[NT] + msn * nA * c[NM] + tmsn * nA * nM * c[NW] + 3 * b * Pz + 4 * bo * Pv +
                     msn * nA * bo * Pn + tmsn * nA * nM * bo * Pz) * eps;
  const double dk = (c[NU] + 3 * o * c[NM] + tmsn * nM * o * c[NW] + 4 * oa * c[NN] + tmsn * nM * oa * c[NZ]) * eps;
  const double dw = (c[NY] + 3 * o * c[NT] + msn * nA * o * c[NM] + tmsn * nA * nM * o * c[NW] + 4 * oa * c[NV] +
                     msn * nA * oa * c[NN] + tmsn * nA * nM * oa * c[NZ]) * eps;
  const double dq = (c[NR] + 2 * a * c[NS]) * eps;
  const double du = (c[NK] + 2 * a * c[NL]) * eps;
  const double dy = (c[NW] + 2 * a * c[NZ]) * eps;
  if (S.first) {   // z_0 = t_0, s_0 = w_0, g_0 = k_0: round-off of explicit products
    S.Fz = msn * nA * c[NL] * eps;
    S.Fw = msn * nA * c[NK] * eps;
    S.Fs = msn * nA * c[NG] * eps;
    S.first = 0;
  } else {
    const double Fz = b * S.Fz + nA * dl + dz;                                   // Eq. (Dz)
    const double Fs = S.Fw + b * S.Fs + bo * S.Fz + nA * dg + ds;                // Eq. (Ds)
    S.Fz = Fz;
    S.Fs = Fs;
  }
  S.f_pending = S.f;
  S.f = S.f + a * S.Fs + o * S.Fw + oa * S.Fz + nA * dx + dr + o * nA * du + dq + o * dy;   // Eq. (Dr)
  S.Fw = S.Fw + a * S.Fz + nA * (dk + du) + dw + dy;                                       // Eq. (Dw)
  S.pg = c[NG]; S.ps = c[NS]; S.pl = c[NL]; S.pz = c[NZ]; S.pn = c[NN]; S.pv = c[NV];
}

// After Eq. (rr): every gap restarts from the round-off of the explicit recomputation.
template <typename T, typename VR>
__device__ void gb_reset(GapBound& S, const SolverParams<T, VR>& p, double xn, double kn, double gn, double sn,
                         double ln, double zn, double bn) {
  const double msn = p.bnd_msn, nA = p.bnd_nA, eps = p.bnd_eps;
  S.f = ((msn + 1.0) * nA * xn + bn) * eps;
  S.Fw = msn * nA * kn * eps;
  S.Fs = msn * nA * gn * eps;
  S.Fz = msn * nA * ln * eps;
  S.ps = sn;
  S.pl = ln;
  S.pz = zn;
}

__device__ __forceinline__ void gb_end_iteration(GapBound& S, double rn) {
  S.f_prev = S.f_pending;
  S.rn_prev = S.rn_cur;
  S.rn_cur = rn;
  S.have_prev = 1;
}

// ---------------------------------------------------------------------------
// Synchronisation scopes.  The algorithm body is written once against a "team":
//  GridTeam  -- the whole cooperative grid solves one system; sync() is the
//               grid barrier with timeout, dot partials go through global memory.
//  BlockTeam -- one thread block solves one system (batched solver); sync() is
//               __syncthreads and the partials stay in shared memory.
// Both give every thread of the team bit-identical reduction results.
struct GridTeam {
  int lanes = 1;  // one thread per row
  // Rows of this block: first, first + stride, ... below end.  Either one contiguous
  // chunk per block (neighbours within about a chunk are re-read from L1/L2 by the same
  // block), or grid-stride order: the whole grid sweeps a window of gridDim*blockDim
  // consecutive rows together, so neighbours farther away than a chunk (the +-plane
  // couplings of a 3D stencil) are read from L2 while the window still holds them.
  int first, stride, end;
  int first4, stride4;   // four-row (VEC) passes: first row of this thread's first quad is
                         // first4 + 4 * threadIdx.x, then every stride4 rows, below end
  int bid;        // this block's index within the team
  int nblk;       // blocks in the team (the whole grid, or one sub-grid of a multi solve)
  unsigned epoch;
  unsigned* bar;
  int* err;
  unsigned long long timeout_ns;
  double* part;
  double* smem;   // >= kWork + kMaxDots doubles
  double* scal;   // >= 8 doubles of shared memory for scalar broadcasts
  __device__ __forceinline__ bool sync() { return grid_barrier(bar, ++epoch, (unsigned)nblk, err, timeout_ns); }
  __device__ __forceinline__ void arrive() { grid_arrive(bar); ++epoch; }
  __device__ __forceinline__ bool wait() { return grid_wait(bar, epoch, (unsigned)nblk, err, timeout_ns); }
  template <int ND>
  __device__ __forceinline__ void publish(double (&v)[ND], int set) {
    block_publish<ND>(v, smem, part + (size_t)set * nblk * kMaxDots, bid);
  }
  template <int ND>
  __device__ __forceinline__ void combine(int set, double (&out)[ND]) {
    grid_combine<ND>(part + (size_t)set * nblk * kMaxDots, nblk, out, smem);
  }
  __device__ __forceinline__ bool leader() const { return bid == 0 && threadIdx.x == 0; }
};

struct BlockTeam {
  int first, stride, end;
  int lanes = 1;  // threads per row in the SpMVs of passes A and B (CSR; a power of two)
  double* smem;   // >= kWork + 3*kMaxDots doubles
  double* scal;   // >= 8 doubles of shared memory for scalar broadcasts
  __device__ __forceinline__ bool sync() { __syncthreads(); return true; }
  template <int ND>
  __device__ __forceinline__ void publish(double (&v)[ND], int set) {
    block_reduce<ND>(v, smem, smem + kWork + set * kMaxDots);
  }
  template <int ND>
  __device__ __forceinline__ void combine(int set, double (&out)[ND]) {
#pragma unroll
    for (int d = 0; d < ND; ++d) out[d] = smem[kWork + set * kMaxDots + d];
  }
  __device__ __forceinline__ bool leader() const { return threadIdx.x == 0; }
};

// A thread-block cluster solves one system (batched solver): rows are dealt to the
// cluster's blocks in turn, sync() is the hardware cluster barrier, and each block's
// partials stay in its own shared memory, from which every block sums all ranks' values
// in rank order through distributed shared memory -- identical totals in every block.
struct ClusterTeam {
  int first, stride, end;
  int lanes = 1;  // threads per row in the SpMVs of passes A and B (CSR; a power of two)
  unsigned rank, nrank;
  double* smem;   // >= kWork + 5*kMaxDots doubles
  double* scal;   // >= 8 doubles
  __device__ __forceinline__ bool sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    return true;
  }
  template <int ND>
  __device__ __forceinline__ void publish(double (&v)[ND], int set) {
    block_reduce<ND>(v, smem, smem + kWork + set * kMaxDots);
  }
  // Valid after the sync() that follows every rank's publish of `set`; a rank publishes
  // the same set again only after a later sync(), so the reads below never race with it.
  template <int ND>
  __device__ __forceinline__ void combine(int set, double (&out)[ND]) {
    double* tot = smem + kWork + 4 * kMaxDots;   // this block's copy of the totals
    if (threadIdx.x < ND) {
      const unsigned laddr = (unsigned)__cvta_generic_to_shared(smem + kWork + set * kMaxDots + threadIdx.x);
      double acc = 0.0;
      for (unsigned q = 0; q < nrank; ++q) {   // rank order: the same sum in every block
        unsigned raddr;
        double v;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(q));
        asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(raddr) : "memory");
        acc += v;
      }
      tot[threadIdx.x] = acc;
    }
    __syncthreads();
#pragma unroll
    for (int d = 0; d < ND; ++d) out[d] = tot[d];
    __syncthreads();
  }
  __device__ __forceinline__ bool leader() const { return rank == 0 && threadIdx.x == 0; }
};

// d_inv of row i: the stored vector, or the one value of a constant diagonal.
template <typename T, typename VR>
__device__ __forceinline__ T dinv_at(const SolverParams<T, VR>& p, int i) {
  return p.dinv ? __ldg(p.dinv + i) : p.dinv_c;
}

// M^{-1} v at row i.  With a constant diagonal d (SCALAR kernels) the Jacobi preconditioner
// is the scalar 1/d, and Algorithm 2 with M^{-1} = I/d equals Algorithm 2 with M^{-1} = I
// on every vector the reductions and the stop test see (r, w, s, z, t, v, q, y; alpha,
// beta, omega unchanged), while its preconditioned vectors are the identity version's
// divided by d.  The solver therefore keeps those vectors multiplied by d -- this function
// is then the identity -- and applies the 1/d where they leave the recurrences: in the
// x update (x += (alpha/d) g + (omega/d) u) and in the replacement's s = A g.  Exact
// arithmetic is unchanged; two FP64 multiplications per row and pass disappear.
template <bool SCALAR, typename T, typename VR>
__device__ __forceinline__ T minv_local(const SolverParams<T, VR>& p, T v, int i) {
  return (p.prec == 1 && !SCALAR) ? T(dinv_at(p, i) * v) : v;
}

// One Jacobi sweep of the Neumann polynomial on two quads of four rows per thread with the
// operands staged in shared memory: out = D^{-1}src + D^{-1}(src - V src) (j = 1,
// V = A D^{-1}) or out = prev + D^{-1}(src - V prev) (j > 1, V = A), the same per-row
// products in the same order as the register form.  Each block walks its trips (rows
// base .. base+R-1, R = 8 x threads) through an S-stage pipeline: thread 0 moves the windows
// of trip k+S-1 with bulk copies (TMA, one instruction per contiguous window, completing on
// the stage's mbarrier) while the block computes trip k from shared memory, so the loads
// wait in the copy engine rather than in registers; two quads per thread halve the per-trip
// waits and barriers.  128-bit shared reads at a 16-byte thread stride are conflict-free; the
// couplings within +-3 rows come from the own quad and the neighbouring lanes' quads
// (shuffles), the lanes at a warp's ends read the one value beyond it from shared memory.
// A stage wait that runs past timeout_ns sets the error flag; the block then waits (bounded)
// for its copies in flight and returns, and the grid barrier that follows reports it.
template <int S, typename VR, typename Team>
__device__ void staged_sweep(const SolverParams<float, VR>& p, const Team& team, float* buf, int j, const float* src,
                             const float* prev, float* out) {
  const MatView<float>& V = j == 1 ? p.At : p.Au;
  const float* gin = j == 1 ? src : prev;        // the gathered vector
  const int n = p.n, row1 = team.end;
  const int tid = threadIdx.x;
  const int nmask = ((n + 7) & ~7) + 8;          // padded length of the mask array
  __shared__ StageLayout s_lay;
  __shared__ int s_base[kMaxDiag];
  __shared__ __align__(8) unsigned long long s_bar[S];
  __shared__ int s_fail;
  if (tid == 0) {
    stage_layout(s_lay, p.Au.off, p.Au.ndiag, 8 * (int)blockDim.x);
    for (int q = 0; q < S; ++q) mbar_init(&s_bar[q], 1);
    fence_proxy_async_smem();
    fence_proxy_async_global();   // the previous sweep's plain stores, before bulk reads
    s_fail = 0;
  }
  __syncthreads();
  const int R = s_lay.R, H = s_lay.H, nearw = R + 2 * s_lay.H;
  if (tid < V.ndiag) {   // where offset d's neighbours of the thread's rows sit in a stage
    const int off = V.off[tid];
    int base = H + off;
    if (off < -R || off > R) {
      int f = 0;
      while (f < s_lay.nfar - 1 && s_lay.far[f] != off) ++f;
      base = nearw + f * R;
    }
    s_base[tid] = base;
  }
  // two quads per thread per trip: rows base + q*4*blockDim + 4*tid, q = 0, 1
  const int tfirst = p.strided ? 8 * (int)blockIdx.x * (int)blockDim.x : team.first;
  const int tstride = p.strided ? 8 * (int)gridDim.x * (int)blockDim.x : 8 * (int)blockDim.x;
  int ntrips = 0;
  for (int b = tfirst; b < row1; b += tstride) ++ntrips;
  // V's offsets in one of the stencil patterns: the products of a trip then carry no
  // offset tests
  const int pat = V.pattern;

  // thread 0: the windows of trip k into stage k % S, clipped to the vectors' rows
  auto issue = [&](int k) {
    float* st = buf + (size_t)(k % S) * s_lay.stage_f;
    unsigned long long* bar = &s_bar[k % S];
    const int base = tfirst + k * tstride;
    const int mlo = base & ~7;
    const int mhi = min(mlo + R + 8, nmask);
    unsigned bytes = 0;
    for (int go = 0; go < 2; ++go) {
      if (go) mbar_arrive_expect_tx(bar, bytes);
      auto win = [&](float* dst, const float* v, int lo, int cnt) {
        const int a0 = max(lo, 0), a1 = min(lo + cnt, n);   // multiples of 4
        if (a1 <= a0) return;
        if (go) bulk_copy_g2s(dst + (a0 - lo), v + a0, (unsigned)(a1 - a0) * 4u, bar);
        else bytes += (unsigned)(a1 - a0) * 4u;
      };
      win(st, gin, base - H, nearw);
      for (int f = 0; f < s_lay.nfar; ++f) win(st + nearw + f * R, gin, base + s_lay.far[f], R);
      if (go && j > 1) {   // the source rows, read from global memory by the trip: into L2 now
        const int a1 = min(base + R, n);
        if (a1 > base) bulk_prefetch_l2(src + base, (unsigned)(a1 - base) * 4u);
      }
      if (go) bulk_copy_g2s(st + s_lay.mask_f, p.Au.mask + mlo, (unsigned)(mhi - mlo) * 2u, bar);
      else bytes += (unsigned)(mhi - mlo) * 2u;
    }
  };
  if (tid == 0)
    for (int k = 0; k < S - 1 && k < ntrips; ++k) issue(k);
  const unsigned lane = tid & 31u;
  int k = 0;
  for (; k < ntrips; ++k) {
    if (tid == 0 && k + S - 1 < ntrips) issue(k + S - 1);
    bool ok = mbar_wait(&s_bar[k % S], (unsigned)(k / S) & 1u, p.timeout_ns);
    ok = __all_sync(kFull, ok);
    if (!ok) s_fail = 1;
    if (ok) {
      const float* st = buf + (size_t)(k % S) * s_lay.stage_f;
      const int base = tfirst + k * tstride;
      for (int qd = 0; qd < 2; ++qd) {
      const int qo = qd * 4 * (int)blockDim.x;
      const int i0 = base + qo + 4 * tid;
      const float* ownp = st + H + qo + 4 * tid;
      const float4 own4 = *reinterpret_cast<const float4*>(ownp);
      const float prv3 = __shfl_up_sync(kFull, own4.w, 1);
      const float nxt0 = __shfl_down_sync(kFull, own4.x, 1);
      float prv1 = 0.f, prv2 = 0.f, nxt1 = 0.f, nxt2 = 0.f;   // the +-2, +-3 couplings: general offsets only
      if (pat == 0) {
        prv1 = __shfl_up_sync(kFull, own4.y, 1);
        prv2 = __shfl_up_sync(kFull, own4.z, 1);
        nxt1 = __shfl_down_sync(kFull, own4.y, 1);
        nxt2 = __shfl_down_sync(kFull, own4.z, 1);
      }
      if (i0 < row1) {
        const unsigned short* mrow =
            reinterpret_cast<const unsigned short*>(st + s_lay.mask_f) + (base - (base & ~7)) + qo + 4 * tid;
        const uint2 mu = *reinterpret_cast<const uint2*>(mrow);
        const unsigned m0 = mu.x & 0xffffu, m1 = mu.x >> 16, m2 = mu.y & 0xffffu, m3 = mu.y >> 16;
        // x[i0 + t] for t = -3 .. 6
        // x[i0 - 1] and x[i0 + 4]: the neighbouring lanes' quads, or shared memory at a warp's ends
        float wm1 = prv3, w4 = nxt0;
        if (lane == 0) wm1 = ownp[-1];
        if (lane == 31) w4 = ownp[4];
        const float w0 = own4.x, w1 = own4.y, w2 = own4.z, w3 = own4.w;
        auto pick = [&](int t) {   // x[i0 + t], -3 <= t <= 6 (general offsets)
          return t == -3 ? (lane ? prv1 : ownp[-3]) : t == -2 ? (lane ? prv2 : ownp[-2]) : t == -1 ? wm1
               : t == 0 ? w0 : t == 1 ? w1 : t == 2 ? w2 : t == 3 ? w3 : t == 4 ? w4
               : t == 5 ? (lane != 31 ? nxt1 : ownp[5]) : (lane != 31 ? nxt2 : ownp[6]);
        };
        float4 sv = own4;
        if (j > 1) sv = *reinterpret_cast<const float4*>(src + i0);   // own rows: one coalesced load
        float a0 = V.unit_diag ? w0 : 0.f, a1 = V.unit_diag ? w1 : 0.f;
        float a2 = V.unit_diag ? w2 : 0.f, a3 = V.unit_diag ? w3 : 0.f;
        // offset d's products; with the offset count known at compile time (5: 2D, 7: 3D
        // stencils) the loop unrolls, the offsets become constant-bank operands and their
        // tests loop-invariant, which is most of a sweep's instruction count
        auto product = [&](int d) {
          const int off = V.off[d];
          const unsigned bit = V.mbit[d];
          const float c = V.cval[d];
          float e0, e1, e2, e3;
          if (off == -1) { e0 = wm1; e1 = w0; e2 = w1; e3 = w2; }
          else if (off == 1) { e0 = w1; e1 = w2; e2 = w3; e3 = w4; }
          else if (off == 0) { e0 = w0; e1 = w1; e2 = w2; e3 = w3; }
          else if (off >= -3 && off <= 3) { e0 = pick(off); e1 = pick(off + 1); e2 = pick(off + 2); e3 = pick(off + 3); }
          else if ((off & 3) == 0) {
            const float4 v4 = *reinterpret_cast<const float4*>(st + s_base[d] + qo + 4 * tid);
            e0 = v4.x; e1 = v4.y; e2 = v4.z; e3 = v4.w;
          } else {
            const float* ep = st + s_base[d] + qo + 4 * tid;
            e0 = ep[0]; e1 = ep[1]; e2 = ep[2]; e3 = ep[3];
          }
          if ((m0 >> bit) & 1u) a0 = fma(c, e0, a0);
          if ((m1 >> bit) & 1u) a1 = fma(c, e1, a1);
          if ((m2 >> bit) & 1u) a2 = fma(c, e2, a2);
          if ((m3 >> bit) & 1u) a3 = fma(c, e3, a3);
        };
        // the same products with the offset kinds fixed at compile time
        auto product_k = [&](int d, auto kc) {
          constexpr int K = decltype(kc)::value;
          const unsigned bit = V.mbit[d];
          const float c = V.cval[d];
          float e0, e1, e2, e3;
          if constexpr (K == 1) { e0 = wm1; e1 = w0; e2 = w1; e3 = w2; }
          else if constexpr (K == 2) { e0 = w0; e1 = w1; e2 = w2; e3 = w3; }
          else if constexpr (K == 3) { e0 = w1; e1 = w2; e2 = w3; e3 = w4; }
          else {
            const float4 v4 = *reinterpret_cast<const float4*>(st + s_base[d] + qo + 4 * tid);
            e0 = v4.x; e1 = v4.y; e2 = v4.z; e3 = v4.w;
          }
          if ((m0 >> bit) & 1u) a0 = fma(c, e0, a0);
          if ((m1 >> bit) & 1u) a1 = fma(c, e1, a1);
          if ((m2 >> bit) & 1u) a2 = fma(c, e2, a2);
          if ((m3 >> bit) & 1u) a3 = fma(c, e3, a3);
        };
        if (pat == 7) {
          for_pattern<7>(product_k);
        } else if (pat == 6) {
          for_pattern<6>(product_k);
        } else if (pat == 5) {
          for_pattern<5>(product_k);
        } else if (pat == 4) {
          for_pattern<4>(product_k);
        } else if (V.ndiag == 7) {
#pragma unroll
          for (int d = 0; d < 7; ++d) product(d);
        } else if (V.ndiag == 5) {
#pragma unroll
          for (int d = 0; d < 5; ++d) product(d);
        } else {
#pragma unroll 1
          for (int d = 0; d < V.ndiag; ++d) product(d);
        }
        const float di = p.dinv_c;
        Quad<float> o;
        if (j == 1) {
          o.v[0] = fma(di, sv.x - a0, di * sv.x); o.v[1] = fma(di, sv.y - a1, di * sv.y);
          o.v[2] = fma(di, sv.z - a2, di * sv.z); o.v[3] = fma(di, sv.w - a3, di * sv.w);
        } else {
          o.v[0] = fma(di, sv.x - a0, w0); o.v[1] = fma(di, sv.y - a1, w1);
          o.v[2] = fma(di, sv.z - a2, w2); o.v[3] = fma(di, sv.w - a3, w3);
        }
        st4(out, i0, o);
      }
      }   // qd
    }
    __syncthreads();   // the stage is refilled for trip k + S; s_fail is settled
    if (s_fail) break;
  }
  if (tid == 0) {
    if (s_fail) {
      atomicCAS(p.err, 0, (int)kTimeout);
      const int issued = min(ntrips, k + S);   // trips 0 .. k + S - 1 were issued
      for (int q = k; q < issued; ++q) mbar_wait(&s_bar[q % S], (unsigned)(q / S) & 1u, p.timeout_ns);
    }
    for (int q = 0; q < S; ++q) mbar_inval(&s_bar[q]);
  }
}

// Neumann polynomial M^{-1} src = sum_{j<=d} (I - D^{-1}A)^j D^{-1} src by d
// Jacobi sweeps y_1 = D^{-1}src + D^{-1}(src - (A D^{-1}) src),
// y_j = y_{j-1} + D^{-1}(src - A y_{j-1}); one or two vectors at once.
// Returns false if the grid must stop.
template <bool VEC = false, typename T, typename VR, typename Team>
__device__ bool neumann_apply(const SolverParams<T, VR>& p, Team& team, const T* src0, T* dst0, const T* src1,
                              T* dst1) {
  const int row0 = team.first, rstride = team.stride, row1 = team.end;
  const int d = p.degree;
  const T* prev0 = nullptr;
  const T* prev1 = nullptr;
  for (int j = 1; j <= d; ++j) {
    T* out0 = ((d - j) % 2 == 0) ? dst0 : p.tmpa;
    T* out1 = ((d - j) % 2 == 0) ? dst1 : p.tmpb;
    if constexpr (VEC && std::is_same<T, float>::value) {
      if (p.staged && !src1) {
        extern __shared__ __align__(16) float pbcg_stage_smem[];
        staged_sweep<2>(p, team, pbcg_stage_smem, j, src0, prev0, out0);
        if (!team.sync()) return false;
        prev0 = out0;
        continue;
      }
    }
    if constexpr (VEC) {
      // four rows per thread; the stencil storage has one diagonal value (dinv_c)
      const T di = p.dinv_c;
      for (int i0 = team.first4 + 4 * threadIdx.x; i0 < row1; i0 += team.stride4) {
        if (p.prefetch && (threadIdx.x & 3) == 0 && i0 + p.prefetch * team.stride4 < row1) {
          const int jn = i0 + p.prefetch * team.stride4;
          prefetch_l2(src0 + jn);
          if (j > 1) prefetch_l2(prev0 + jn);
          if (src1) { prefetch_l2(src1 + jn); if (j > 1) prefetch_l2(prev1 + jn); }
        }
        unsigned mk[4];
        ld_mask4(p.Au.mask, i0, mk);
        {
          const Quad<T> sv = ld4(src0, i0);
          Quad<T> o;
          if (j == 1) {
            const Quad<T> as = quad_dot<T>(p.At, src0, i0, mk);
#pragma unroll
            for (int q = 0; q < 4; ++q) o.v[q] = fma(di, sv.v[q] - as.v[q], di * sv.v[q]);
          } else {
            const Quad<T> ap = quad_dot<T>(p.Au, prev0, i0, mk);
            const Quad<T> pv = ld4(prev0, i0);
#pragma unroll
            for (int q = 0; q < 4; ++q) o.v[q] = fma(di, sv.v[q] - ap.v[q], pv.v[q]);
          }
          st4(out0, i0, o);
        }
        if (src1) {
          const Quad<T> sv = ld4(src1, i0);
          Quad<T> o;
          if (j == 1) {
            const Quad<T> as = quad_dot<T>(p.At, src1, i0, mk);
#pragma unroll
            for (int q = 0; q < 4; ++q) o.v[q] = fma(di, sv.v[q] - as.v[q], di * sv.v[q]);
          } else {
            const Quad<T> ap = quad_dot<T>(p.Au, prev1, i0, mk);
            const Quad<T> pv = ld4(prev1, i0);
#pragma unroll
            for (int q = 0; q < 4; ++q) o.v[q] = fma(di, sv.v[q] - ap.v[q], pv.v[q]);
          }
          st4(out1, i0, o);
        }
      }
      if (!team.sync()) return false;
      prev0 = out0;
      prev1 = out1;
      continue;
    }
    for (int i = row0 + threadIdx.x; i < row1; i += rstride) {
      if (p.prefetch && i + p.prefetch * rstride < row1) {
        const int jn = i + p.prefetch * rstride;
        prefetch_l2(src0 + jn);
        if (j > 1) prefetch_l2(prev0 + jn);
        if (src1) { prefetch_l2(src1 + jn); if (j > 1) prefetch_l2(prev1 + jn); }
      }
      const T di = dinv_at(p, i);
      {
        const T sv = src0[i];
        if (j == 1) out0[i] = fma(di, sv - row_dot<T>(p.At, src0, i), di * sv);
        else out0[i] = fma(di, sv - row_dot<T>(p.Au, prev0, i), prev0[i]);
      }
      if (src1) {
        const T sv = src1[i];
        if (j == 1) out1[i] = fma(di, sv - row_dot<T>(p.At, src1, i), di * sv);
        else out1[i] = fma(di, sv - row_dot<T>(p.Au, prev1, i), prev1[i]);
      }
    }
    if (!team.sync()) return false;
    prev0 = out0;
    prev1 = out1;
  }
  return true;
}

#define PBCG_HS 8

// Eq. (rr), first half: r = b - A x in FP64 (FP64 values), s = A g with FP64 values,
// and with Jacobi / no preconditioner also k = D^{-1} r, l = D^{-1} s and
// nb = D^{-1} z_i (n_i stays the one computed from the old z_i, reading R6).
// Publishes the partial ||b - A x||^2 to P2.  With write == false only the norm
// is computed (stopping-test verification).
template <bool AUTO, bool SCALAR, typename T, typename VR, typename Team>
__device__ void replace_r1(const SolverParams<T, VR>& p, Team& team, bool write) {
  using Acc = typename AccOf<T>::type;
  const int row0 = team.first, rstride = team.stride, row1 = team.end;
  DAcc a_tr, a_x;
  Acc a_g, a_k, a_s, a_l;
  const bool neu = p.prec == 2;
  for (int i = row0 + threadIdx.x; i < row1; i += rstride) {
    const double r64 = p.b[i] - row_dot<double>(p.A64, p.x, i);
    if (write) {
      const T ri = T(r64);
      const double ag = row_dot<double>(p.A64, p.g, i);
      const T si = T(SCALAR ? ag * p.dinv_x : ag);
      p.r[i] = ri;
      p.s[i] = si;
      if (!neu) {
        const T ki = minv_local<SCALAR>(p, ri, i), li = minv_local<SCALAR>(p, si, i);
        p.k[i] = ki;
        p.l[i] = li;
        p.nb[i] = minv_local<SCALAR>(p, p.z[i], i);
        if (AUTO) { a_k.add(ki, ki); a_l.add(li, li); }
      }
      if (AUTO) {
        const double xi = p.x[i];
        const T gi = p.g[i];
        a_x.add(xi, xi); a_g.add(gi, gi); a_s.add(si, si);
      }
    }
    a_tr.add(r64, r64);
  }
  if (AUTO) {
    // ||b - A x||^2 and the norms the gap bound restarts from: x, g, k, s, l
    double v6[6] = {a_tr.value(), a_x.value(), a_g.value(), a_k.value(), a_s.value(), a_l.value()};
    team.template publish<6>(v6, 2);
  } else {
    double v1[1] = {a_tr.value()};
    team.template publish<1>(v1, 2);
  }
}

// Eq. (rr), second half (after a grid barrier): Neumann k = M^{-1} r, l = M^{-1} s;
// then w = A k, z = A l and the line-21 partials of the replaced vectors into P1.
template <bool AUTO, typename T, typename VR, typename Team>
__device__ bool replace_r2(const SolverParams<T, VR>& p, Team& team) {
  using Acc = typename AccOf<T>::type;
  const int row0 = team.first, rstride = team.stride, row1 = team.end;
  const bool neu = p.prec == 2;
  if (neu && !neumann_apply(p, team, p.r, p.k, p.s, p.l)) return false;
  Acc a_rr, a_rw, a_rs, a_rz, a_r2, a_z;
  for (int i = row0 + threadIdx.x; i < row1; i += rstride) {
    const T wi = neu ? row_dot<T>(p.Au, p.k, i) : row_dot<T>(p.At, p.r, i);
    const T zi = neu ? row_dot<T>(p.Au, p.l, i) : row_dot<T>(p.At, p.s, i);
    p.w[i] = wi;
    p.z[i] = zi;
    const T rh = p.rh[i], ri = p.r[i], si = p.s[i];
    a_rr.add(rh, ri); a_rw.add(rh, wi); a_rs.add(rh, si); a_rz.add(rh, zi); a_r2.add(ri, ri);
    if (AUTO) a_z.add(zi, zi);
  }
  if (AUTO) {
    double v6[6] = {a_rr.value(), a_rw.value(), a_rs.value(), a_rz.value(), a_r2.value(), a_z.value()};
    team.template publish<6>(v6, 1);
  } else {
    double v5[5] = {a_rr.value(), a_rw.value(), a_rs.value(), a_rz.value(), a_r2.value()};
    team.template publish<5>(v5, 1);
  }
  return true;
}

// y_i = (A x)_i for this block's rows with L threads per row (L = team.lanes): the block's
// rows first + k*stride + [0, blockDim) are dealt to blockDim/L lane groups, so each
// thread follows a chain of nnz/L dependent loads instead of nnz.  The block then reads
// y at its own rows (one __syncthreads: no other block touches them).
template <typename T, typename Team>
__device__ void spmv_lanes(const Team& team, const MatView<T>& A, const T* x, T* y) {
  const int L = team.lanes, G = blockDim.x / L, g = threadIdx.x / L, sub = threadIdx.x % L;
  for (int base = team.first; base < team.end; base += team.stride)
    for (int h = 0; h < L; ++h) {
      const int i = base + g + h * G;
      if (i < team.end) {
        const T v = row_dot_lanes<T>(A, x, i, sub, L);
        if (sub == 0) y[i] = v;
      }
    }
  __syncthreads();
}

// Interior of a block's chunk (chunked row order): rows [lo, hi) whose SpMV operands, rows
// within +-halo, all belong to the block.  Their products need no other block's writes, so
// the block computes them between arriving at a grid barrier and waiting on it.  The quad
// passes use the quads inside [lo, hi): first row a multiple of 4 from lo4 = lo rounded up.
struct Interior {
  int lo, hi, lo4;
  __device__ __forceinline__ bool row(int i) const { return i >= lo && i < hi; }
  __device__ __forceinline__ bool quad(int i0) const { return i0 >= lo4 && i0 + 3 < hi; }
};

template <typename T, typename VR, typename Team>
__device__ __forceinline__ Interior interior_of(const SolverParams<T, VR>& p, const Team& team) {
  Interior in;
  in.lo = team.first + p.halo;
  in.hi = team.end - p.halo;
  in.lo4 = (in.lo + 3) & ~3;
  if (!p.overlap || in.hi <= in.lo) in.lo = in.hi = in.lo4 = 0;   // empty
  return in;
}

// y = At x on the interior rows (the row mapping need not match the passes': the grid_wait
// after it synchronises the block).
template <bool VEC, typename T, typename VR, typename Team>
__device__ __forceinline__ void interior_product(const SolverParams<T, VR>& p, const Team& team, const Interior& in,
                                                 const T* x, T* y) {
  if constexpr (VEC) {
    for (int i0 = in.lo4 + 4 * threadIdx.x; i0 + 3 < in.hi; i0 += 4 * blockDim.x) {
      unsigned mk[4];
      ld_mask4(p.At.mask, i0, mk);
      st4(y, i0, quad_dot<T>(p.At, x, i0, mk));
    }
  } else {
    for (int i = in.lo + threadIdx.x; i < in.hi; i += blockDim.x) y[i] = row_dot<T>(p.At, x, i);
  }
}

// Pass A on four rows per thread (stencil storage, VEC kernels): the same per-row
// arithmetic as the one-row loop in solve_body, rows taken a quad at a time.
template <bool SCALAR, typename T, typename VR, typename Team, typename Acc>
__device__ __forceinline__ void pass_a_quads(const SolverParams<T, VR>& p, const Team& team, T aT, T bT, T opT,
                                             bool rep_last, const Interior& pre, Acc& a_qy, Acc& a_yy) {
  const bool neu = p.prec == 2;
  const int row1 = team.end;
  for (int i0 = team.first4 + 4 * threadIdx.x; i0 < row1; i0 += team.stride4) {
    if (p.prefetch && (threadIdx.x & 3) == 0 && i0 + p.prefetch * team.stride4 < row1) {   // later quads, into L2
      const int j = i0 + p.prefetch * team.stride4;
      prefetch_l2(p.w + j); prefetch_l2(p.z + j); prefetch_l2(p.k + j); prefetch_l2(p.g + j);
      prefetch_l2(p.l + j); prefetch_l2(p.s + j); prefetch_l2(p.v + j); prefetch_l2(p.r + j);
      if (neu) { prefetch_l2(p.m + j); prefetch_l2(p.nn + j); }
    }
    unsigned mk[4];
    ld_mask4(p.Au.mask, i0, mk);
    const Quad<T> W = ld4(p.w, i0), Z = ld4(p.z, i0), K = ld4(p.k, i0), G = ld4(p.g, i0);
    const Quad<T> L = ld4(p.l, i0), S = ld4(p.s, i0), V = ld4(p.v, i0), R = ld4(p.r, i0);
    Quad<T> M, NP;
    if (neu) {
      M = ld4(p.m, i0);
      NP = ld4(p.nn, i0);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) M.v[q] = minv_local<SCALAR>(p, W.v[q], i0 + q);
      if (rep_last) NP = ld4(p.nb, i0);
      else {
#pragma unroll
        for (int q = 0; q < 4; ++q) NP.v[q] = minv_local<SCALAR>(p, Z.v[q], i0 + q);
      }
    }
    const Quad<T> Tq = pre.quad(i0) ? ld4(p.t, i0)                      // t_i = A m_i (inside the last barrier)
                       : neu ? quad_dot<T>(p.Au, p.m, i0, mk) : quad_dot<T>(p.At, p.w, i0, mk);
    Quad<T> Gn, Sn, Ln, Zn;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Gn.v[q] = fma(bT, fma(-opT, L.v[q], G.v[q]), K.v[q]);    // g_i
      Sn.v[q] = fma(bT, fma(-opT, Z.v[q], S.v[q]), W.v[q]);    // s_i
      Ln.v[q] = fma(bT, fma(-opT, NP.v[q], L.v[q]), M.v[q]);   // l_i
      Zn.v[q] = fma(bT, fma(-opT, V.v[q], Z.v[q]), Tq.v[q]);   // z_i
      const T qq = fma(-aT, Sn.v[q], R.v[q]);                  // q_i
      const T y = fma(-aT, Zn.v[q], W.v[q]);                   // y_i
      a_qy.add(qq, y);
      a_yy.add(y, y);
    }
    st4(p.g, i0, Gn); st4(p.s, i0, Sn); st4(p.l, i0, Ln); st4(p.z, i0, Zn); st4(p.t, i0, Tq);
  }
}

// Pass B on four rows per thread (see pass_a_quads).
template <bool SCALAR, typename T, typename VR, typename Team, typename Acc>
__device__ __forceinline__ void pass_b_quads(const SolverParams<T, VR>& p, const Team& team, T aT, T oT, double ax,
                                             double ox, bool hist, int it, bool do_rr, const Interior& pre,
                                             Acc& a_rr, Acc& a_rw, Acc& a_rs, Acc& a_rz, Acc& a_r2) {
  const bool neu = p.prec == 2;
  const int row1 = team.end;
  const size_t n = (size_t)p.n;
  for (int i0 = team.first4 + 4 * threadIdx.x; i0 < row1; i0 += team.stride4) {
    if (p.prefetch && (threadIdx.x & 3) == 0 && i0 + p.prefetch * team.stride4 < row1) {
      const int j = i0 + p.prefetch * team.stride4;
      prefetch_l2(p.z + j); prefetch_l2(p.w + j); prefetch_l2(p.r + j); prefetch_l2(p.s + j);
      prefetch_l2(p.k + j); prefetch_l2(p.l + j); prefetch_l2(p.g + j); prefetch_l2(p.t + j);
      prefetch_l2(p.x + j); prefetch_l2(p.rh + j);
      if (neu) { prefetch_l2(p.m + j); prefetch_l2(p.nn + j); }
    }
    unsigned mk[4];
    ld_mask4(p.Au.mask, i0, mk);
    const Quad<T> Z = ld4(p.z, i0), W = ld4(p.w, i0), R = ld4(p.r, i0), S = ld4(p.s, i0);
    const Quad<T> K = ld4(p.k, i0), L = ld4(p.l, i0), G = ld4(p.g, i0), Tt = ld4(p.t, i0);
    const Quad<double> X = ld4(p.x, i0);
    Quad<T> N, M;
    if (neu) {
      N = ld4(p.nn, i0);
      M = ld4(p.m, i0);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        N.v[q] = minv_local<SCALAR>(p, Z.v[q], i0 + q);
        M.v[q] = minv_local<SCALAR>(p, W.v[q], i0 + q);
      }
    }
    const Quad<T> Vq = pre.quad(i0) ? ld4(p.v, i0)                      // v_i = A n_i (inside the last barrier)
                       : neu ? quad_dot<T>(p.Au, p.nn, i0, mk) : quad_dot<T>(p.At, p.z, i0, mk);
    Quad<double> Xn;
    Quad<T> Rn, Kn, Wn;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T qq = fma(-aT, S.v[q], R.v[q]);
      const T u = fma(-aT, L.v[q], K.v[q]);
      const T y = fma(-aT, Z.v[q], W.v[q]);
      Xn.v[q] = fma(ox, (double)u, fma(ax, (double)G.v[q], X.v[q]));   // x_{i+1}
      Rn.v[q] = fma(-oT, y, qq);                                          // r_{i+1}
      Kn.v[q] = fma(-oT, fma(-aT, N.v[q], M.v[q]), u);                   // k_{i+1}
      Wn.v[q] = fma(-oT, fma(-aT, Vq.v[q], Tt.v[q]), y);                 // w_{i+1}
    }
    st4(p.x, i0, Xn); st4(p.v, i0, Vq); st4(p.r, i0, Rn); st4(p.k, i0, Kn); st4(p.w, i0, Wn);
    if (hist) {
#pragma unroll
      for (int q = 0; q < 4; ++q) p.hist_x[(size_t)it * n + i0 + q] = Xn.v[q];
    }
    if (!do_rr) {
      const Quad<T> RH = ld4(p.rh, i0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a_rr.add(RH.v[q], Rn.v[q]); a_rw.add(RH.v[q], Wn.v[q]); a_rs.add(RH.v[q], S.v[q]);
        a_rz.add(RH.v[q], Z.v[q]); a_r2.add(Rn.v[q], Rn.v[q]);
      }
    }
  }
}

// The whole solve (Algorithm 2 + Eq. rr) for one system, executed by a team.
template <bool AUTO, bool SCALAR, bool VEC = false, typename T, typename VR, typename Team>
__device__ __forceinline__ void solve_body(const SolverParams<T, VR>& p, Team& team) {
  static_assert(!(VEC && AUTO), "the four-row passes run without the automated policy");
  using Acc = typename AccOf<T>::type;
  const int n = p.n;
  // automated replacement state, used by thread 0 only (AUTO kernels)
  __shared__ GapBound gb;
  __shared__ double gnorm[NNORMS];
  const int row0 = team.first, rstride = team.stride, row1 = team.end;
  const bool neu = p.prec == 2;
  const bool leader = team.leader();
  int nrep = 0;
  int nrestart = 0;           // restarts after breakdowns (bounded by max_restarts)
  int nperiodic = 0;          // periodic restarts (reading R20)
  int it = 0;                 // completed iterations, across restarts
  bool first = true;
  double rn0 = 0.0;
  // reading R21: reference true residual, the iteration it was set, best true residual
  double ref_true = INFINITY, best_true = INFINITY;
  int ref_it = 0;

#define PBCG_SYNC() \
  do { if (!team.sync()) return; } while (0)
#define PBCG_ROWS for (int i = row0 + threadIdx.x; i < row1; i += rstride)
  // FP64 division and square root are multi-instruction sequences on the scarce FP64
  // pipe: thread 0 evaluates them and the block reads the results from shared memory.
  double* const sc = team.scal;
#define PBCG_BCAST_BEGIN if (threadIdx.x == 0) {
#define PBCG_BCAST_END \
  }                    \
  __syncthreads();
#define PBCG_BCAST_DONE __syncthreads();
#define PBCG_FINISH(st, its, rnv)                                                        \
  do {                                                                                   \
    if (leader) {                                                                        \
      p.res->status = (st); p.res->iterations = (its); p.res->nrep = nrep;               \
      p.res->nrestart = nrestart + nperiodic; p.res->rn_rel = (rnv) / bn;                \
    }                                                                                    \
    return;                                                                              \
  } while (0)

  // A breakdown (a zero or non-finite omega, (r0, r_i), beta or alpha denominator) can,
  // if the options allow it, restart the method from the current iterate: the initialisation
  // again with x as the initial guess and the new r as the shadow vector.
  for (;;) {
  // ---------------- initialisation of Algorithm 2
  {
    Acc a_rr;
    DAcc a_bb, a_xx, a_tr;
    PBCG_ROWS {
      const double bi = p.b[i];
      if (AUTO) { const double xi = p.x[i]; a_xx.add(xi, xi); }
      const double r64 = bi - row_dot<double>(p.A64, p.x, i);
      const T ri = T(r64);
      p.r[i] = ri;
      p.rh[i] = ri;
      if (!neu) p.k[i] = minv_local<SCALAR>(p, ri, i);
      p.g[i] = T(0); p.s[i] = T(0); p.l[i] = T(0); p.z[i] = T(0); p.v[i] = T(0);
      if (neu) p.nn[i] = T(0);
      a_rr.add(ri, ri);
      a_bb.add(bi, bi);
      if constexpr (!std::is_same<T, double>::value) a_tr.add(r64, r64);   // FP64 ||b - A x||^2
    }
    double v4[4] = {a_rr.value(), a_bb.value(), std::is_same<T, double>::value ? a_rr.value() : a_tr.value(),
                    a_xx.value()};
    if (AUTO) team.template publish<4>(v4, 0);
    else team.template publish<3>(*reinterpret_cast<double(*)[3]>(v4), 0);
  }
  PBCG_SYNC();
  if (neu && !neumann_apply(p, team, p.r, p.k, (const T*)nullptr, (T*)nullptr)) return;
  {
    Acc a_rw;
    PBCG_ROWS {
      const T wi = neu ? row_dot<T>(p.Au, p.k, i) : row_dot<T>(p.At, p.r, i);  // w_0 = A k_0
      p.w[i] = wi;
      a_rw.add(p.rh[i], wi);
    }
    double v1[1] = {a_rw.value()};
    team.template publish<1>(v1, 1);
  }
  PBCG_SYNC();
  double rho, rw0, bn, rn, alpha, tolb, rtrue;
  {
    double t4[4] = {0.0, 0.0, 0.0, 0.0};
    if (AUTO) team.template combine<4>(0, t4);
    else team.template combine<3>(0, *reinterpret_cast<double(*)[3]>(t4));
    double t1[1];
    team.template combine<1>(1, t1);
    rho = t4[0];
    rw0 = t1[0];
    PBCG_BCAST_BEGIN
      sc[0] = sqrt(t4[1]);
      sc[1] = sqrt(rho);
      sc[2] = rw0 != 0.0 ? rho / rw0 : INFINITY;
      sc[3] = p.tol * sc[0];
      sc[4] = sqrt(t4[2]);
      if (AUTO) gb_start(gb, p, sqrt(t4[3]), sc[0], sc[1]);
    PBCG_BCAST_END
    bn = sc[0];
    rn = sc[1];
    alpha = sc[2];
    tolb = sc[3];
    rtrue = sc[4];
    PBCG_BCAST_DONE
  }
  if (first) {
    if (leader) { p.res->bnorm = bn; p.res->rn0 = rn; p.res->true_rel = -1.0; }
    if (bn == 0.0) {            // b = 0: x = 0
      PBCG_ROWS { p.x[i] = 0.0; }
      if (leader) {
        p.res->status = kOK; p.res->iterations = 0; p.res->nrep = 0; p.res->nrestart = 0; p.res->rn_rel = 0.0;
      }
      return;
    }
    rn0 = rn;
    first = false;
  }
  if (rtrue <= tolb) PBCG_FINISH(kOK, it, rn);
  if (p.stag_window > 0) {
    // reading R21: progress of the FP64 true residual between (re)starts
    if (rtrue <= 0.5 * ref_true) {
      ref_true = rtrue;
      ref_it = it;
    } else if (it - ref_it >= p.stag_window) {
      if (p.xbest && best_true < rtrue) PBCG_ROWS { p.x[i] = p.xbest[i]; }
      PBCG_FINISH(kStagnated, it, rn);
    }
    if (rtrue < best_true) {   // each thread copies the rows it alone updates
      best_true = rtrue;
      if (p.xbest) PBCG_ROWS { p.xbest[i] = p.x[i]; }
    }
  }
  if (rw0 == 0.0 || !isfinite(alpha)) PBCG_FINISH(kBreakdown, it, rn);
  const int it_start = it;
  double beta = 0.0, omega_prev = 0.0;
  bool rep_last = false;
  bool restart = false;
  // interior rows of this block, and whether t = A m was computed on them inside the last
  // barrier (never right after a (re)start or a replacement forced by the stop test)
  const Interior inner = interior_of(p, team);
  const Interior none{0, 0, 0};
  bool t_pre = false;
  const double rr_cutoff = p.rr_cutoff * rn0;       // periodic replacements stop below this
  double rr_theta_thr = p.rr_theta * rn;            // relative trigger threshold

  for (; it < p.max_it; ++it) {
    // ---------------- m_i = M^{-1} w_i (Neumann only; on the fly otherwise)
    if (neu && !neumann_apply<VEC>(p, team, p.w, p.m, (const T*)nullptr, (T*)nullptr)) return;
    // ---------------- pass A: t_i = A m_i; g, s, l, z, q, u, y; partials of (q, y), (y, y)
    const bool split = team.lanes > 1 && !neu && p.At.fmt == 0;   // lane-split SpMVs (batched CSR)
    if (split) spmv_lanes(team, p.At, p.w, p.t);
    {
      const T aT = T(alpha), bT = T(beta), opT = T(omega_prev);
      Acc a_qy, a_yy;
      Acc an[12];   // AUTO: squared norms of r k w g s l z q u y m t (iteration i)
      const Interior& tin = t_pre ? inner : none;
      if constexpr (VEC) pass_a_quads<SCALAR>(p, team, aT, bT, opT, rep_last, tin, a_qy, a_yy);
      else PBCG_ROWS {
        if (p.prefetch && i + p.prefetch * rstride < row1) {   // operands of a later row, into L2
          const int j = i + p.prefetch * rstride;
          prefetch_l2(p.w + j); prefetch_l2(p.z + j); prefetch_l2(p.k + j); prefetch_l2(p.g + j);
          prefetch_l2(p.l + j); prefetch_l2(p.s + j); prefetch_l2(p.v + j); prefetch_l2(p.r + j);
          if (neu) { prefetch_l2(p.m + j); prefetch_l2(p.nn + j); }
        }
        const T wi = p.w[i];
        const T mi = neu ? p.m[i] : minv_local<SCALAR>(p, wi, i);
        const T ti = (split || tin.row(i)) ? p.t[i] : neu ? row_dot<T>(p.Au, p.m, i) : row_dot<T>(p.At, p.w, i);
        const T zo = p.z[i];
        const T np = neu ? p.nn[i] : (rep_last ? p.nb[i] : minv_local<SCALAR>(p, zo, i));   // n_{i-1}
        const T kk = p.k[i], gg = p.g[i], ll = p.l[i], ss = p.s[i], vv = p.v[i], rr = p.r[i];
        const T gn = fma(bT, fma(-opT, ll, gg), kk);   // g_i = k_i + beta_i (g_{i-1} - omega_{i-1} l_{i-1})
        const T sn = fma(bT, fma(-opT, zo, ss), wi);   // s_i = w_i + beta_i (s_{i-1} - omega_{i-1} z_{i-1})
        const T ln = fma(bT, fma(-opT, np, ll), mi);   // l_i = m_i + beta_i (l_{i-1} - omega_{i-1} n_{i-1})
        const T zn = fma(bT, fma(-opT, vv, zo), ti);   // z_i = t_i + beta_i (z_{i-1} - omega_{i-1} v_{i-1})
        const T q = fma(-aT, sn, rr);                  // q_i = r_i - alpha_i s_i
        const T y = fma(-aT, zn, wi);                  // y_i = w_i - alpha_i z_i
        p.g[i] = gn; p.s[i] = sn; p.l[i] = ln; p.z[i] = zn; p.t[i] = ti;
        a_qy.add(q, y);
        a_yy.add(y, y);
        if (AUTO) {
          const T u = fma(-aT, ln, kk);
          an[0].add(rr, rr); an[1].add(kk, kk); an[2].add(wi, wi); an[3].add(gn, gn); an[4].add(sn, sn);
          an[5].add(ln, ln); an[6].add(zn, zn); an[7].add(q, q); an[8].add(u, u); an[9].add(y, y);
          an[10].add(mi, mi); an[11].add(ti, ti);
        }
      }
      if (AUTO) {
        double v14[14];
        v14[0] = a_qy.value();
        v14[1] = a_yy.value();
#pragma unroll
        for (int j = 0; j < 12; ++j) v14[2 + j] = an[j].value();
        team.template publish<14>(v14, 0);
      } else {
        double v2[2] = {a_qy.value(), a_yy.value()};
        team.template publish<2>(v2, 0);
      }
    }
    if constexpr (std::is_same<Team, GridTeam>::value) {
      if (p.overlap) {   // v_i = A n_i on the interior rows while the first reduction completes
        team.arrive();
        interior_product<VEC>(p, team, inner, p.z, p.v);
        if (!team.wait()) return;
      } else {
        PBCG_SYNC();
      }
    } else {
      PBCG_SYNC();
    }
    // ---------------- n_i = M^{-1} z_i (Neumann only), overlapping the reduction
    if (neu && !neumann_apply<VEC>(p, team, p.z, p.nn, (const T*)nullptr, (T*)nullptr)) return;
    double omega;
    bool do_auto = false;
    {
      double t14[14];
      if (AUTO) team.template combine<14>(0, t14);
      else team.template combine<2>(0, *reinterpret_cast<double(*)[2]>(t14));
      PBCG_BCAST_BEGIN
        sc[0] = t14[1] == 0.0 ? 0.0 : t14[0] / t14[1];   // omega_i
        if (AUTO) {
          for (int j = 1; j <= 12; ++j) gnorm[j] = sqrt(t14[j + 1]);   // r..t of iteration i
          sc[1] = gb_criterion(gb, p.rr_tau) ? 1.0 : 0.0;               // Eq. (criterion)
        }
      PBCG_BCAST_END
      omega = sc[0];
      if (AUTO) do_auto = sc[1] != 0.0;
      PBCG_BCAST_DONE
    }
    if (!isfinite(omega)) {
      if (nrestart < p.max_restarts) { ++nrestart; ++it; restart = true; break; }
      PBCG_FINISH(kBreakdown, it, rn);
    }
    bool do_rr = false;
    if (p.rr_period > 0 && it > 0 && it % p.rr_period == 0 && rn >= rr_cutoff) do_rr = true;
    if (p.rr_theta > 0.0 && rn <= rr_theta_thr) do_rr = true;
    if (do_auto) do_rr = true;
    // ---------------- pass B: v_i = A n_i; x, r, k, w; partials of the second reduction
    if (split) spmv_lanes(team, p.At, p.z, p.v);
    {
      const T aT = T(alpha), oT = T(omega);
      const double ax = SCALAR ? alpha * p.dinv_x : alpha;   // x update (see minv_local)
      const double ox = SCALAR ? omega * p.dinv_x : omega;
      Acc a_rr, a_rw, a_rs, a_rz, a_r2;
      DAcc a_xn;
      Acc a_nn, a_vn;   // AUTO: squared norms of x_i, n_i, v_i
      const bool hist = it < p.K;
      if constexpr (VEC)
        pass_b_quads<SCALAR>(p, team, aT, oT, ax, ox, hist, it, do_rr, inner, a_rr, a_rw, a_rs, a_rz, a_r2);
      else PBCG_ROWS {
        if (p.prefetch && i + p.prefetch * rstride < row1) {
          const int j = i + p.prefetch * rstride;
          prefetch_l2(p.z + j); prefetch_l2(p.w + j); prefetch_l2(p.r + j); prefetch_l2(p.s + j);
          prefetch_l2(p.k + j); prefetch_l2(p.l + j); prefetch_l2(p.g + j); prefetch_l2(p.t + j);
          prefetch_l2(p.x + j); prefetch_l2(p.rh + j);
          if (neu) { prefetch_l2(p.m + j); prefetch_l2(p.nn + j); }
        }
        const T zi = p.z[i];
        const T ni = neu ? p.nn[i] : minv_local<SCALAR>(p, zi, i);
        const T vi = (split || inner.row(i)) ? p.v[i] : neu ? row_dot<T>(p.Au, p.nn, i) : row_dot<T>(p.At, p.z, i);
        const T wi = p.w[i];
        const T mi = neu ? p.m[i] : minv_local<SCALAR>(p, wi, i);
        const T rr = p.r[i], ss = p.s[i], kk = p.k[i], ll = p.l[i], gg = p.g[i], ti = p.t[i];
        const T q = fma(-aT, ss, rr);
        const T u = fma(-aT, ll, kk);
        const T y = fma(-aT, zi, wi);
        const double xo = p.x[i];
        if (AUTO) { a_xn.add(xo, xo); a_nn.add(ni, ni); a_vn.add(vi, vi); }
        const double xn = fma(ox, (double)u, fma(ax, (double)gg, xo));  // x_{i+1}
        const T rn1 = fma(-oT, y, q);                    // r_{i+1} = q_i - omega_i y_i
        const T kn = fma(-oT, fma(-aT, ni, mi), u);      // k_{i+1} = u_i - omega_i (m_i - alpha_i n_i)
        const T wn = fma(-oT, fma(-aT, vi, ti), y);      // w_{i+1} = y_i - omega_i (t_i - alpha_i v_i)
        p.x[i] = xn; p.v[i] = vi; p.r[i] = rn1; p.k[i] = kn; p.w[i] = wn;
        if (hist) p.hist_x[(size_t)it * n + i] = xn;
        if (!do_rr) {
          const T rh = p.rh[i];
          a_rr.add(rh, rn1); a_rw.add(rh, wn); a_rs.add(rh, ss); a_rz.add(rh, zi); a_r2.add(rn1, rn1);
        }
      }
      if (!do_rr) {
        double v5[5] = {a_rr.value(), a_rw.value(), a_rs.value(), a_rz.value(), a_r2.value()};
        team.template publish<5>(v5, 1);
      }
      if (AUTO) {
        double v3[3] = {a_xn.value(), a_nn.value(), a_vn.value()};
        team.template publish<3>(v3, 3);
      }
    }
    // ---------------- residual replacement, Eq. (rr), right after the w update (reading R6)
    if (do_rr) {
      PBCG_SYNC();
      replace_r1<AUTO, SCALAR>(p, team, true);
      PBCG_SYNC();
      if (!replace_r2<AUTO>(p, team)) return;
      ++nrep;
    }
    rep_last = do_rr;
    t_pre = false;
    if constexpr (std::is_same<Team, GridTeam>::value) {
      if (p.overlap) {   // t_{i+1} = A m_{i+1} on the interior rows while the second reduction completes
        team.arrive();
        interior_product<VEC>(p, team, inner, p.w, p.t);
        if (!team.wait()) return;
        t_pre = true;
      } else {
        PBCG_SYNC();
      }
    } else {
      PBCG_SYNC();
    }
    // ---------------- second reduction, stopping test, beta_{i+1}, alpha_{i+1}
    double t5[6];
    if (AUTO && do_rr) team.template combine<6>(1, t5);
    else team.template combine<5>(1, *reinterpret_cast<double(*)[5]>(t5));
    double rho_new = t5[0], rw = t5[1], rs = t5[2], rz = t5[3];
    if (AUTO) {
      // gap bound: step with the iteration-i norms, then restart it after a replacement
      double t3[3], t6[6];
      team.template combine<3>(3, t3);
      if (do_rr) team.template combine<6>(2, t6);
      if (threadIdx.x == 0) {
        gnorm[NX] = sqrt(t3[0]);
        gnorm[NN] = sqrt(t3[1]);
        gnorm[NV] = sqrt(t3[2]);
        gb_step(gb, p, gnorm, alpha, beta, omega, omega_prev);
        if (do_rr) gb_reset(gb, p, sqrt(t6[1]), sqrt(t6[3]), sqrt(t6[2]), sqrt(t6[4]), sqrt(t6[5]), sqrt(t5[5]), bn);
      }
    }
    PBCG_BCAST_BEGIN
      sc[0] = sqrt(t5[4]);
    PBCG_BCAST_END
    rn = sc[0];
    PBCG_BCAST_DONE
    if (rn <= tolb) {
      // reading R5: verify with the FP64 true residual; with a replacement policy a
      // failed check forces a replacement, without one the solve has stagnated.
      const bool any_rr = p.rr_period > 0 || p.rr_theta > 0.0 || AUTO;
      replace_r1<AUTO, SCALAR>(p, team, any_rr);
      PBCG_SYNC();
      double t1[6];
      if (AUTO) team.template combine<6>(2, t1);
      else team.template combine<1>(2, *reinterpret_cast<double(*)[1]>(t1));
      PBCG_BCAST_BEGIN
        sc[0] = sqrt(t1[0]);
        p.res->true_rel = sc[0] / bn;
      PBCG_BCAST_END
      const double true_rn = sc[0];
      PBCG_BCAST_DONE
      if (true_rn <= tolb || !any_rr) {
        if (leader && it < p.hist_len) {
          double* h = p.hist_s + (size_t)it * PBCG_HS;
          h[0] = alpha; h[1] = omega; h[2] = NAN; h[3] = rn / bn; h[4] = do_rr ? 1.0 : 0.0;
        }
        if (true_rn > tolb && p.restart_period > 0) {   // reading R20: restart from x instead
          ++nperiodic; ++it; restart = true; break;
        }
        PBCG_FINISH(true_rn <= tolb ? kOK : kStagnated, it + 1, rn);
      }
      if (!replace_r2<AUTO>(p, team)) return;
      ++nrep;
      rep_last = true;
      do_rr = true;
      t_pre = false;   // w was replaced after t was computed from it
      PBCG_SYNC();
      if (AUTO) team.template combine<6>(1, t5);
      else team.template combine<5>(1, *reinterpret_cast<double(*)[5]>(t5));
      rho_new = t5[0]; rw = t5[1]; rs = t5[2]; rz = t5[3];
      if (AUTO && threadIdx.x == 0)
        gb_reset(gb, p, sqrt(t1[1]), sqrt(t1[3]), sqrt(t1[2]), sqrt(t1[4]), sqrt(t1[5]), sqrt(t5[5]), bn);
      PBCG_BCAST_BEGIN
        sc[0] = sqrt(t5[4]);
      PBCG_BCAST_END
      rn = sc[0];
      PBCG_BCAST_DONE
    }
    double beta_new, alpha_new, den;
    PBCG_BCAST_BEGIN
      if (AUTO) gb_end_iteration(gb, rn);
      if (do_rr) sc[3] = p.rr_theta * rn;
      sc[0] = __dmul_rn(__ddiv_rn(alpha, omega), __ddiv_rn(rho_new, rho));                               // beta_{i+1}
      sc[1] = __dsub_rn(__dadd_rn(rw, __dmul_rn(sc[0], rs)), __dmul_rn(__dmul_rn(sc[0], omega), rz));   // its alpha denominator
      sc[2] = sc[1] != 0.0 ? __ddiv_rn(rho_new, sc[1]) : INFINITY;
    PBCG_BCAST_END
    beta_new = sc[0];
    den = sc[1];
    alpha_new = sc[2];
    if (do_rr) rr_theta_thr = sc[3];
    PBCG_BCAST_DONE
    if (omega == 0.0 || rho == 0.0) {
      if (nrestart < p.max_restarts) { ++nrestart; ++it; restart = true; break; }
      PBCG_FINISH(kBreakdown, it + 1, rn);
    }
    if (leader && it < p.hist_len) {
      double* h = p.hist_s + (size_t)it * PBCG_HS;
      h[0] = alpha; h[1] = omega; h[2] = beta_new; h[3] = rn / bn; h[4] = do_rr ? 1.0 : 0.0;
    }
    if (!(isfinite(beta_new) && den != 0.0 && isfinite(alpha_new))) {
      if (nrestart < p.max_restarts) { ++nrestart; ++it; restart = true; break; }
      PBCG_FINISH(kBreakdown, it + 1, rn);
    }
    if (p.restart_period > 0 && it + 1 - it_start >= p.restart_period) {   // reading R20
      ++nperiodic; ++it; restart = true; break;
    }
    alpha = alpha_new;
    beta = beta_new;
    omega_prev = omega;
    rho = rho_new;
  }
  if (!restart) {
    if (p.stag_window > 0 && p.xbest && best_true < INFINITY) {
      // reading R21: return the best (re)start iterate when the last one is worse
      replace_r1<AUTO, SCALAR>(p, team, false);
      PBCG_SYNC();
      double t6[6];
      if (AUTO) team.template combine<6>(2, t6);
      else team.template combine<1>(2, *reinterpret_cast<double(*)[1]>(t6));
      PBCG_BCAST_BEGIN
        sc[0] = sqrt(t6[0]);
      PBCG_BCAST_END
      const double last_true = sc[0];
      PBCG_BCAST_DONE
      if (best_true < last_true) PBCG_ROWS { p.x[i] = p.xbest[i]; }
    }
    PBCG_FINISH(kNotConverged, p.max_it, rn);
  }
  }  // restarts
#undef PBCG_SYNC
#undef PBCG_ROWS
#undef PBCG_FINISH
#undef PBCG_BCAST_BEGIN
#undef PBCG_BCAST_END
#undef PBCG_BCAST_DONE
}

// Register budget of the persistent solver.  FP64 is bound by the FP64 pipe and keeps 64
// registers (one 1024-thread block per SM).  The FP32 recurrences of the mixed solver come
// in two builds: where the working set stays in L2 the same 64-register shape is fastest
// (2D mixed: 46 vs 64 us per iteration), where it streams from DRAM the iteration is bound
// by memory-level parallelism, so STREAM trades registers (40, with some spilling) for 48
// resident warps per SM (three 512-thread blocks): 1173 vs 1301 us per iteration on the
// 256^3 Neumann system (FP64 at that budget loses 12%).
// The four-row (VEC) kernels: 512-thread blocks, one per SM (128 registers, no spills), and
// for a mixed solve whose working set exceeds L2 a streaming build of 768-thread blocks (80
// registers, some spilling): 24 instead of 16 resident warps per SM, 806 vs 941 us per
// iteration on the 256^3 Neumann system (on the L2-resident 2D system and in FP64 the
// 512-thread build is faster: 36 vs 39 and 88 vs 105 us).  The build parameters below let a
// build trade registers for resident warps differently.
#ifndef PBCG_VEC_THREADS
#define PBCG_VEC_THREADS 512
#endif
#ifndef PBCG_VEC_STREAM_THREADS
#define PBCG_VEC_STREAM_THREADS 768
#endif
#ifndef PBCG_VEC_BLOCKS_PER_SM
#define PBCG_VEC_BLOCKS_PER_SM 1
#endif
template <typename T, bool STREAM, bool VEC = false>
struct SolverLaunch {
  static constexpr int kThreads = VEC ? (STREAM ? PBCG_VEC_STREAM_THREADS : PBCG_VEC_THREADS)
                                      : STREAM ? 512 : kMaxThreads;
  static constexpr int kBlocksPerSM = VEC ? PBCG_VEC_BLOCKS_PER_SM : STREAM ? 3 : 1;
};

// One cooperative grid solves one system.  AUTO adds the automated replacement policy
// (extra norms in the reductions and the gap bound in thread 0).
// VEC: the hot passes take four rows per thread (structured-stencil storage, n a multiple
// of 4, 16-byte aligned vectors, p.chunk a multiple of 4); the other passes keep one row
// per thread -- every pass is separated from the next by a barrier, so the two row
// mappings never meet inside one.
template <typename T, bool AUTO, bool STREAM = false, bool SCALAR = false, bool VEC = false>
__global__ void __launch_bounds__(SolverLaunch<T, STREAM, VEC>::kThreads, SolverLaunch<T, STREAM, VEC>::kBlocksPerSM)
    pbicgstab_kernel(const SolverParams<T> p) {
  __shared__ double smem[kWork + 3 * kMaxDots];
  __shared__ double scal[8];
  GridTeam team;
  team.bid = blockIdx.x;
  team.nblk = gridDim.x;
  if (p.strided) {
    team.first = blockIdx.x * blockDim.x;
    team.stride = gridDim.x * blockDim.x;
    team.end = p.n;
    team.first4 = 4 * blockIdx.x * blockDim.x;
    team.stride4 = 4 * gridDim.x * blockDim.x;
  } else {
    team.first = (int)min((long long)p.n, (long long)blockIdx.x * p.chunk);
    team.stride = blockDim.x;
    team.end = min(p.n, team.first + p.chunk);
    team.first4 = team.first;
    team.stride4 = 4 * blockDim.x;
  }
  team.epoch = 0;
  team.bar = p.bar;
  team.err = p.err;
  team.timeout_ns = p.timeout_ns;
  team.part = p.part;
  team.smem = smem;
  team.scal = scal;
  solve_body<AUTO, SCALAR, VEC>(p, team);
}

// Several independent solves that share the grid: team t is blocks
// [t*bpt, (t+1)*bpt) and runs the whole algorithm on params[t] (its own b, x,
// work vectors, barrier counter, partials and result) with team-local barriers.
// Used for many right-hand sides with one matrix (the matrix is read by every
// team; at moderate sizes it stays in L2).
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 1) pbicgstab_multi_kernel(const SolverParams<T>* params, int bpt) {
  __shared__ double smem[kWork + 3 * kMaxDots];
  __shared__ double scal[8];
  __shared__ SolverParams<T> sp;
  const int t = blockIdx.x / bpt;
  if (threadIdx.x == 0) sp = params[t];
  __syncthreads();
  GridTeam team;
  team.bid = blockIdx.x - t * bpt;
  team.nblk = bpt;
  if (sp.strided) {
    team.first = team.bid * blockDim.x;
    team.stride = bpt * blockDim.x;
    team.end = sp.n;
  } else {
    team.first = (int)min((long long)sp.n, (long long)team.bid * sp.chunk);
    team.stride = blockDim.x;
    team.end = min(sp.n, team.first + sp.chunk);
  }
  team.epoch = 0;
  team.bar = sp.bar;
  team.err = sp.err;
  team.timeout_ns = sp.timeout_ns;
  team.part = sp.part;
  team.smem = smem;
  team.scal = scal;
  solve_body<false, false>(sp, team);
}

// ---------------------------------------------------------------------------
// Classic preconditioned BiCGStab (Algorithm 1), the paper's reference method, with
// the same team machinery.  Three grid barriers per iteration, one per global
// reduction phase of Algorithm 1 ((r0, s_i); (q_i, y_i) with (y_i, y_i); (r0, r_{i+1})).
// The new search direction p_{i} = r_i + beta (p_{i-1} - omega s_{i-1}) and
// q_i = r_i - alpha s_i are formed on the fly wherever the SpMV gathers them, so they need no pass of
// their own; p and s are double-buffered because a pass reads the old values at
// neighbouring rows while writing the new ones.  No preconditioner or Jacobi (folded
// into A D^{-1}: s = A g = (A D^{-1}) p, y = A u = (A D^{-1}) q); no replacement.
// Vector slots: r, rh, y = w, p = g / l (alternating), s = s / z (alternating).
template <bool SCALAR, typename T, typename VR, typename Team>
__device__ void classic_body(const SolverParams<T, VR>& p, Team& team) {
  using Acc = typename AccOf<T>::type;
  const int n = p.n;
  const int row0 = team.first, rstride = team.stride, row1 = team.end;
  const bool leader = team.leader();
  double* const sc = team.scal;
  T* pbuf[2] = {p.g, p.l};
  T* sbuf[2] = {p.s, p.z};
  T* const y = p.w;
#define CL_SYNC() \
  do { if (!team.sync()) return; } while (0)
#define CL_ROWS for (int i = row0 + threadIdx.x; i < row1; i += rstride)
#define CL_FINISH(st, its, rnv)                                                          \
  do {                                                                                   \
    if (leader) {                                                                        \
      p.res->status = (st); p.res->iterations = (its); p.res->nrep = 0;                  \
      p.res->nrestart = 0; p.res->rn_rel = (rnv) / bn;                                   \
    }                                                                                    \
    return;                                                                              \
  } while (0)
  // r_0 = b - A x_0; p_0 = r_0 (formed on the fly below, with beta = 0)
  {
    Acc a_rr;
    DAcc a_bb;
    CL_ROWS {
      const double bi = p.b[i];
      const double r64 = bi - row_dot<double>(p.A64, p.x, i);
      const T ri = T(r64);
      p.r[i] = ri;
      p.rh[i] = ri;
      pbuf[0][i] = T(0);
      sbuf[0][i] = T(0);
      a_rr.add(ri, ri);
      a_bb.add(bi, bi);
    }
    double v2[2] = {a_rr.value(), a_bb.value()};
    team.template publish<2>(v2, 0);
  }
  CL_SYNC();
  double rho, bn, rn, tolb;
  {
    double t2[2];
    team.template combine<2>(0, t2);
    rho = t2[0];
    if (threadIdx.x == 0) { sc[0] = sqrt(t2[1]); sc[1] = sqrt(rho); sc[2] = p.tol * sc[0]; }
    __syncthreads();
    bn = sc[0]; rn = sc[1]; tolb = sc[2];
    __syncthreads();
  }
  if (leader) { p.res->bnorm = bn; p.res->rn0 = rn; p.res->true_rel = -1.0; }
  if (bn == 0.0) {
    CL_ROWS { p.x[i] = 0.0; }
    if (leader) { p.res->status = kOK; p.res->iterations = 0; p.res->nrep = 0; p.res->nrestart = 0; p.res->rn_rel = 0.0; }
    return;
  }
  if (rn <= tolb) CL_FINISH(kOK, 0, rn);
  double beta = 0.0, omega = 0.0;
  int cur = 0;
  for (int it = 0; it < p.max_it; ++it) {
    const T* p_old = pbuf[cur];
    const T* s_old = sbuf[cur];
    T* p_new = pbuf[cur ^ 1];
    T* s_new = sbuf[cur ^ 1];
    // p_i (from the previous iteration), g_i = M^{-1} p_i, s_i = A g_i, (r0, s_i)
    {
      const T bT = T(beta), oT = T(omega);
      Acc a_rs;
      CL_ROWS {
        const T acc = row_dot_fn<T>(p.At, i, [&](int j) { return fma(bT, fma(-oT, s_old[j], p_old[j]), p.r[j]); });
        const T pi = fma(bT, fma(-oT, s_old[i], p_old[i]), p.r[i]);
        p_new[i] = pi;
        s_new[i] = acc;
        a_rs.add(p.rh[i], acc);
      }
      double v1[1] = {a_rs.value()};
      team.template publish<1>(v1, 0);
    }
    CL_SYNC();
    double alpha;
    {
      double t1[1];
      team.template combine<1>(0, t1);
      if (threadIdx.x == 0) sc[0] = t1[0] != 0.0 ? rho / t1[0] : INFINITY;   // alpha_i
      __syncthreads();
      alpha = sc[0];
      __syncthreads();
      if (!isfinite(alpha)) CL_FINISH(kBreakdown, it, rn);
    }
    // q_i = r_i - alpha s_i, u_i = M^{-1} q_i, y_i = A u_i, (q_i, y_i), (y_i, y_i)
    {
      const T aT = T(alpha);
      Acc a_qy, a_yy;
      CL_ROWS {
        const T acc = row_dot_fn<T>(p.At, i, [&](int j) { return fma(-aT, s_new[j], p.r[j]); });
        const T qi = fma(-aT, s_new[i], p.r[i]);
        y[i] = acc;
        a_qy.add(qi, acc);
        a_yy.add(acc, acc);
      }
      double v2[2] = {a_qy.value(), a_yy.value()};
      team.template publish<2>(v2, 1);
    }
    CL_SYNC();
    {
      double t2[2];
      team.template combine<2>(1, t2);
      if (threadIdx.x == 0) sc[0] = t2[1] == 0.0 ? 0.0 : t2[0] / t2[1];   // omega_i
      __syncthreads();
      omega = sc[0];
      __syncthreads();
      if (!isfinite(omega)) CL_FINISH(kBreakdown, it, rn);
    }
    // x_{i+1} = (x_i + alpha g_i) + omega u_i, r_{i+1} = q_i - omega y_i, (r0, r_{i+1})
    {
      const T aT = T(alpha), oT = T(omega);
      const double ax = SCALAR ? alpha * p.dinv_x : alpha;   // x update (see minv_local)
      const double ox = SCALAR ? omega * p.dinv_x : omega;
      Acc a_rr, a_r2;
      const bool hist = it < p.K;
      CL_ROWS {
        const T qi = fma(-aT, s_new[i], p.r[i]);
        const T gi = minv_local<SCALAR>(p, p_new[i], i);
        const T ui = minv_local<SCALAR>(p, qi, i);
        const double xn = fma(ox, (double)ui, fma(ax, (double)gi, p.x[i]));
        const T rn1 = fma(-oT, y[i], qi);
        p.x[i] = xn;
        p.r[i] = rn1;
        if (hist) p.hist_x[(size_t)it * n + i] = xn;
        a_rr.add(p.rh[i], rn1);
        a_r2.add(rn1, rn1);
      }
      double v2[2] = {a_rr.value(), a_r2.value()};
      team.template publish<2>(v2, 2);
    }
    CL_SYNC();
    double rho_new;
    {
      double t2[2];
      team.template combine<2>(2, t2);
      rho_new = t2[0];
      if (threadIdx.x == 0) {
        sc[0] = sqrt(t2[1]);
        sc[1] = __dmul_rn(__ddiv_rn(alpha, omega), __ddiv_rn(rho_new, rho));   // beta_i
      }
      __syncthreads();
      rn = sc[0];
      const double beta_new = sc[1];
      __syncthreads();
      if (leader && it < p.hist_len) {
        double* h = p.hist_s + (size_t)it * PBCG_HS;
        h[0] = alpha; h[1] = omega; h[2] = beta_new; h[3] = rn / bn; h[4] = 0.0;
      }
      if (rn <= tolb) {   // reading R5 without replacement: verify, else stagnated
        if (leader && it < p.hist_len) p.hist_s[(size_t)it * PBCG_HS + 2] = NAN;
        DAcc a_tr;
        CL_ROWS {
          const double r64 = p.b[i] - row_dot<double>(p.A64, p.x, i);
          a_tr.add(r64, r64);
        }
        double v1[1] = {a_tr.value()};
        team.template publish<1>(v1, 3);
        CL_SYNC();
        double t1[1];
        team.template combine<1>(3, t1);
        if (threadIdx.x == 0) { sc[0] = sqrt(t1[0]); p.res->true_rel = sc[0] / bn; }
        __syncthreads();
        const double true_rn = sc[0];
        __syncthreads();
        CL_FINISH(true_rn <= tolb ? kOK : kStagnated, it + 1, rn);
      }
      if (omega == 0.0 || rho == 0.0 || !isfinite(beta_new)) CL_FINISH(kBreakdown, it + 1, rn);
      beta = beta_new;
      rho = rho_new;
    }
    cur ^= 1;
  }
  CL_FINISH(kNotConverged, p.max_it, rn);
#undef CL_SYNC
#undef CL_ROWS
#undef CL_FINISH
}

template <typename T, bool SCALAR = false>
__global__ void __launch_bounds__(kMaxThreads, 1) classic_kernel(const SolverParams<T> p) {
  __shared__ double smem[kWork + 3 * kMaxDots];
  __shared__ double scal[8];
  GridTeam team;
  team.bid = blockIdx.x;
  team.nblk = gridDim.x;
  if (p.strided) {
    team.first = blockIdx.x * blockDim.x;
    team.stride = gridDim.x * blockDim.x;
    team.end = p.n;
  } else {
    team.first = (int)min((long long)p.n, (long long)blockIdx.x * p.chunk);
    team.stride = blockDim.x;
    team.end = min(p.n, team.first + p.chunk);
  }
  team.epoch = 0;
  team.bar = p.bar;
  team.err = p.err;
  team.timeout_ns = p.timeout_ns;
  team.part = p.part;
  team.smem = smem;
  team.scal = scal;
  classic_body<SCALAR>(p, team);
}

}  // namespace pbcg
