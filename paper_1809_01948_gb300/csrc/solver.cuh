// Persistent, cooperatively launched p-BiCGStab kernel (Algorithm 2 of arXiv
// 1809.01948 with the residual replacement step of Eq. (rr)).
//
// One launch runs the whole solve.  Rows are split into one contiguous chunk per
// block.  Each iteration is two fused passes separated by grid barriers; each pass
// is an SPMV fused with the AXPY recurrences and the partial dot products of one
// global reduction phase, so the paper's "overlap GLRED with SPMV + PREC" becomes:
// the reduction completes at the barrier the next SPMV needs anyway.
//
//   pass A (lines 5-12 + 23 of iteration i-1): t_i = A m_i, then g, s, l, z, q, u, y
//          and partials of (q,y), (y,y)
//   pass B (lines 13-21): v_i = A n_i, omega_i, then x, r, k, w (q, u, y recomputed
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
  const T* dinv;        // D^{-1} (nullptr without preconditioner)
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
};

// ---------------------------------------------------------------------------
// Synchronisation scopes.  The algorithm body is written once against a "team":
//  GridTeam  -- the whole cooperative grid solves one system; sync() is the
//               grid barrier with timeout, dot partials go through global memory.
//  BlockTeam -- one thread block solves one system (batched solver); sync() is
//               __syncthreads and the partials stay in shared memory.
// Both give every thread of the team bit-identical reduction results.
struct GridTeam {
  // Rows of this block: first, first + stride, ... below end.  Either one contiguous
  // chunk per block (neighbours within about a chunk are re-read from L1/L2 by the same
  // block), or grid-stride order: the whole grid sweeps a window of gridDim*blockDim
  // consecutive rows together, so neighbours farther away than a chunk (the +-plane
  // couplings of a 3D stencil) are read from L2 while the window still holds them.
  int first, stride, end;
  int bid;        // this block's index within the team
  int nblk;       // blocks in the team (the whole grid, or one sub-grid of a multi solve)
  unsigned epoch;
  unsigned* bar;
  int* err;
  unsigned long long timeout_ns;
  double* part;
  double* smem;   // >= 32*8 + kMaxDots doubles
  double* scal;   // >= 8 doubles of shared memory for scalar broadcasts
  __device__ __forceinline__ bool sync() { return grid_barrier(bar, ++epoch, (unsigned)nblk, err, timeout_ns); }
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
  double* smem;   // >= 32*8 + 3*kMaxDots doubles
  double* scal;   // >= 8 doubles of shared memory for scalar broadcasts
  __device__ __forceinline__ bool sync() { __syncthreads(); return true; }
  template <int ND>
  __device__ __forceinline__ void publish(double (&v)[ND], int set) {
    block_reduce<ND>(v, smem, smem + 32 * 8 + set * kMaxDots);
  }
  template <int ND>
  __device__ __forceinline__ void combine(int set, double (&out)[ND]) {
#pragma unroll
    for (int d = 0; d < ND; ++d) out[d] = smem[32 * 8 + set * kMaxDots + d];
  }
  __device__ __forceinline__ bool leader() const { return threadIdx.x == 0; }
};

template <typename T, typename VR>
__device__ __forceinline__ T minv_local(const SolverParams<T, VR>& p, T v, int i) {
  return p.prec == 1 ? T(__ldg(p.dinv + i) * v) : v;
}

// Neumann polynomial M^{-1} src = sum_{j<=d} (I - D^{-1}A)^j D^{-1} src by d
// Jacobi sweeps y_1 = D^{-1}src + D^{-1}(src - (A D^{-1}) src),
// y_j = y_{j-1} + D^{-1}(src - A y_{j-1}); one or two vectors at once.
// Returns false if the grid must stop.
template <typename T, typename VR, typename Team>
__device__ bool neumann_apply(const SolverParams<T, VR>& p, Team& team, const T* src0, T* dst0, const T* src1,
                              T* dst1) {
  const int row0 = team.first, rstride = team.stride, row1 = team.end;
  const int d = p.degree;
  const T* prev0 = nullptr;
  const T* prev1 = nullptr;
  for (int j = 1; j <= d; ++j) {
    T* out0 = ((d - j) % 2 == 0) ? dst0 : p.tmpa;
    T* out1 = ((d - j) % 2 == 0) ? dst1 : p.tmpb;
    for (int i = row0 + threadIdx.x; i < row1; i += rstride) {
      const T di = __ldg(p.dinv + i);
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
template <typename T, typename VR, typename Team>
__device__ void replace_r1(const SolverParams<T, VR>& p, Team& team, bool write) {
  const int row0 = team.first, rstride = team.stride, row1 = team.end;
  DAcc a_tr;
  const bool neu = p.prec == 2;
  for (int i = row0 + threadIdx.x; i < row1; i += rstride) {
    const double r64 = p.b[i] - row_dot<double>(p.A64, p.x, i);
    if (write) {
      const T ri = T(r64);
      const T si = T(row_dot<double>(p.A64, p.g, i));
      p.r[i] = ri;
      p.s[i] = si;
      if (!neu) {
        p.k[i] = minv_local(p, ri, i);
        p.l[i] = minv_local(p, si, i);
        p.nb[i] = minv_local(p, p.z[i], i);
      }
    }
    a_tr.add(r64, r64);
  }
  double v1[1] = {a_tr.value()};
  team.template publish<1>(v1, 2);
}

// Eq. (rr), second half (after a grid barrier): Neumann k = M^{-1} r, l = M^{-1} s;
// then w = A k, z = A l and the line-21 partials of the replaced vectors into P1.
template <typename T, typename VR, typename Team>
__device__ bool replace_r2(const SolverParams<T, VR>& p, Team& team) {
  using Acc = typename AccOf<T>::type;
  const int row0 = team.first, rstride = team.stride, row1 = team.end;
  const bool neu = p.prec == 2;
  if (neu && !neumann_apply(p, team, p.r, p.k, p.s, p.l)) return false;
  Acc a_rr, a_rw, a_rs, a_rz, a_r2;
  for (int i = row0 + threadIdx.x; i < row1; i += rstride) {
    const T wi = neu ? row_dot<T>(p.Au, p.k, i) : row_dot<T>(p.At, p.r, i);
    const T zi = neu ? row_dot<T>(p.Au, p.l, i) : row_dot<T>(p.At, p.s, i);
    p.w[i] = wi;
    p.z[i] = zi;
    const T rh = p.rh[i], ri = p.r[i], si = p.s[i];
    a_rr.add(rh, ri); a_rw.add(rh, wi); a_rs.add(rh, si); a_rz.add(rh, zi); a_r2.add(ri, ri);
  }
  double v5[5] = {a_rr.value(), a_rw.value(), a_rs.value(), a_rz.value(), a_r2.value()};
  team.template publish<5>(v5, 1);
  return true;
}

// The whole solve (Algorithm 2 + Eq. rr) for one system, executed by a team.
template <typename T, typename VR, typename Team>
__device__ void solve_body(const SolverParams<T, VR>& p, Team& team) {
  using Acc = typename AccOf<T>::type;
  const int n = p.n;
  const int row0 = team.first, rstride = team.stride, row1 = team.end;
  const bool neu = p.prec == 2;
  const bool leader = team.leader();
  int nrep = 0;
  int nrestart = 0;
  int it = 0;                 // completed iterations, across restarts
  bool first = true;
  double rn0 = 0.0;

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
      p.res->nrestart = nrestart; p.res->rn_rel = (rnv) / bn;                            \
    }                                                                                    \
    return;                                                                              \
  } while (0)

  // A breakdown (a zero or non-finite omega, (r0, r_i), beta or alpha denominator) can,
  // if the options allow it, restart the method from the current iterate: lines 2-3
  // again with x as the initial guess and the new r as the shadow vector.
  for (;;) {
  // ---------------- initialisation (Algorithm 2, lines 2-3)
  {
    Acc a_rr;
    DAcc a_bb;
    PBCG_ROWS {
      const double bi = p.b[i];
      const double r64 = bi - row_dot<double>(p.A64, p.x, i);
      const T ri = T(r64);
      p.r[i] = ri;
      p.rh[i] = ri;
      if (!neu) p.k[i] = minv_local(p, ri, i);
      p.g[i] = T(0); p.s[i] = T(0); p.l[i] = T(0); p.z[i] = T(0); p.v[i] = T(0);
      if (neu) p.nn[i] = T(0);
      a_rr.add(ri, ri);
      a_bb.add(bi, bi);
    }
    double v2[2] = {a_rr.value(), a_bb.value()};
    team.template publish<2>(v2, 0);
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
  double rho, rw0, bn, rn, alpha, tolb;
  {
    double t2[2];
    team.template combine<2>(0, t2);
    double t1[1];
    team.template combine<1>(1, t1);
    rho = t2[0];
    rw0 = t1[0];
    PBCG_BCAST_BEGIN
      sc[0] = sqrt(t2[1]);
      sc[1] = sqrt(rho);
      sc[2] = rw0 != 0.0 ? rho / rw0 : INFINITY;
      sc[3] = p.tol * sc[0];
    PBCG_BCAST_END
    bn = sc[0];
    rn = sc[1];
    alpha = sc[2];
    tolb = sc[3];
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
  if (rn <= tolb) PBCG_FINISH(kOK, it, rn);
  if (rw0 == 0.0 || !isfinite(alpha)) PBCG_FINISH(kBreakdown, it, rn);
  double beta = 0.0, omega_prev = 0.0;
  bool rep_last = false;
  bool restart = false;
  const double sqrt_eps = 1.4901161193847656e-08;  // sqrt(2^-52)
  const double rr_cutoff = sqrt_eps * rn0;          // periodic replacements stop below this
  double rr_theta_thr = p.rr_theta * rn;            // relative trigger threshold

  for (; it < p.max_it; ++it) {
    // ---------------- m_i = M^{-1} w_i (Neumann only; on the fly otherwise)
    if (neu && !neumann_apply(p, team, p.w, p.m, (const T*)nullptr, (T*)nullptr)) return;
    // ---------------- pass A: t_i = A m_i; lines 5-11; partials of line 12
    {
      const T aT = T(alpha), bT = T(beta), opT = T(omega_prev);
      Acc a_qy, a_yy;
      PBCG_ROWS {
        const T wi = p.w[i];
        const T mi = neu ? p.m[i] : minv_local(p, wi, i);
        const T ti = neu ? row_dot<T>(p.Au, p.m, i) : row_dot<T>(p.At, p.w, i);
        const T zo = p.z[i];
        const T np = neu ? p.nn[i] : (rep_last ? p.nb[i] : minv_local(p, zo, i));   // n_{i-1}
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
      }
      double v2[2] = {a_qy.value(), a_yy.value()};
      team.template publish<2>(v2, 0);
    }
    PBCG_SYNC();
    // ---------------- n_i = M^{-1} z_i (Neumann only), overlapping the reduction
    if (neu && !neumann_apply(p, team, p.z, p.nn, (const T*)nullptr, (T*)nullptr)) return;
    double omega;
    {
      double t2[2];
      team.template combine<2>(0, t2);
      PBCG_BCAST_BEGIN
        sc[0] = t2[1] == 0.0 ? 0.0 : t2[0] / t2[1];   // line 16
      PBCG_BCAST_END
      omega = sc[0];
      PBCG_BCAST_DONE
    }
    if (!isfinite(omega)) {
      if (nrestart < p.max_restarts) { ++nrestart; ++it; restart = true; break; }
      PBCG_FINISH(kBreakdown, it, rn);
    }
    bool do_rr = false;
    if (p.rr_period > 0 && it > 0 && it % p.rr_period == 0 && rn >= rr_cutoff) do_rr = true;
    if (p.rr_theta > 0.0 && rn <= rr_theta_thr) do_rr = true;
    // ---------------- pass B: v_i = A n_i; lines 17-20; partials of line 21
    {
      const T aT = T(alpha), oT = T(omega);
      Acc a_rr, a_rw, a_rs, a_rz, a_r2;
      const bool hist = it < p.K;
      PBCG_ROWS {
        const T zi = p.z[i];
        const T ni = neu ? p.nn[i] : minv_local(p, zi, i);
        const T vi = neu ? row_dot<T>(p.Au, p.nn, i) : row_dot<T>(p.At, p.z, i);
        const T wi = p.w[i];
        const T mi = neu ? p.m[i] : minv_local(p, wi, i);
        const T rr = p.r[i], ss = p.s[i], kk = p.k[i], ll = p.l[i], gg = p.g[i], ti = p.t[i];
        const T q = fma(-aT, ss, rr);
        const T u = fma(-aT, ll, kk);
        const T y = fma(-aT, zi, wi);
        const double xn = fma(omega, (double)u, fma(alpha, (double)gg, p.x[i]));  // line 17
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
    }
    // ---------------- residual replacement, Eq. (rr), after line 20 (reading R6)
    if (do_rr) {
      PBCG_SYNC();
      replace_r1(p, team, true);
      PBCG_SYNC();
      if (!replace_r2(p, team)) return;
      ++nrep;
    }
    rep_last = do_rr;
    PBCG_SYNC();
    // ---------------- lines 21-26: second reduction, stopping test, beta, alpha
    double t5[5];
    team.template combine<5>(1, t5);
    double rho_new = t5[0], rw = t5[1], rs = t5[2], rz = t5[3];
    PBCG_BCAST_BEGIN
      sc[0] = sqrt(t5[4]);
    PBCG_BCAST_END
    rn = sc[0];
    PBCG_BCAST_DONE
    if (rn <= tolb) {
      // reading R5: verify with the FP64 true residual; with a replacement policy a
      // failed check forces a replacement, without one the solve has stagnated.
      const bool any_rr = p.rr_period > 0 || p.rr_theta > 0.0;
      replace_r1(p, team, any_rr);
      PBCG_SYNC();
      double t1[1];
      team.template combine<1>(2, t1);
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
        PBCG_FINISH(true_rn <= tolb ? kOK : kStagnated, it + 1, rn);
      }
      if (!replace_r2(p, team)) return;
      ++nrep;
      rep_last = true;
      do_rr = true;
      PBCG_SYNC();
      team.template combine<5>(1, t5);
      rho_new = t5[0]; rw = t5[1]; rs = t5[2]; rz = t5[3];
      PBCG_BCAST_BEGIN
        sc[0] = sqrt(t5[4]);
      PBCG_BCAST_END
      rn = sc[0];
      PBCG_BCAST_DONE
    }
    double beta_new, alpha_new, den;
    PBCG_BCAST_BEGIN
      if (do_rr) sc[3] = p.rr_theta * rn;
      sc[0] = __dmul_rn(__ddiv_rn(alpha, omega), __ddiv_rn(rho_new, rho));                               // line 25
      sc[1] = __dsub_rn(__dadd_rn(rw, __dmul_rn(sc[0], rs)), __dmul_rn(__dmul_rn(sc[0], omega), rz));   // line 26
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
    alpha = alpha_new;
    beta = beta_new;
    omega_prev = omega;
    rho = rho_new;
  }
  if (!restart) PBCG_FINISH(kNotConverged, p.max_it, rn);
  }  // restarts
#undef PBCG_SYNC
#undef PBCG_ROWS
#undef PBCG_FINISH
#undef PBCG_BCAST_BEGIN
#undef PBCG_BCAST_END
#undef PBCG_BCAST_DONE
}

// One cooperative grid solves one system; block b owns rows [b*chunk, (b+1)*chunk).
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 1) pbicgstab_kernel(const SolverParams<T> p) {
  __shared__ double smem[32 * 8 + 3 * kMaxDots];
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
  solve_body(p, team);
}

// Several independent solves that share the grid: team t is blocks
// [t*bpt, (t+1)*bpt) and runs the whole algorithm on params[t] (its own b, x,
// work vectors, barrier counter, partials and result) with team-local barriers.
// Used for many right-hand sides with one matrix (the matrix is read by every
// team; at moderate sizes it stays in L2).
template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 1) pbicgstab_multi_kernel(const SolverParams<T>* params, int bpt) {
  __shared__ double smem[32 * 8 + 3 * kMaxDots];
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
  solve_body(sp, team);
}

}  // namespace pbcg
