// Device building blocks shared by the p-BiCGStab kernels: sparse matrix views and
// row products (SPMV, Section 1), deterministic block / grid reductions of dot
// products (DOTPR + GLRED), a grid-wide barrier whose wait gives up after a time
// limit, and compensated FP32 accumulation for the mixed-precision dots.
#pragma once
#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace pbcg {

constexpr int kMaxDiag = 16;
constexpr int kMaxThreads = 1024;
constexpr int kMaxDots = 16;
constexpr int kWork = 32 * 16;   // shared work area of block reductions (doubles)

enum DevStatus : int {
  kRunning = -1, kOK = 0, kNotConverged = 4, kBreakdown = 5, kStagnated = 6, kTimeout = 7
};

// ---------------------------------------------------------------- matrices
// A CSR matrix (row_ptr/col int32), a DIA matrix (ndiag diagonals, diagonal-major
// values, val[d*n + i] = A[i, i+off[d]]) or a constant-coefficient stencil: one value
// per offset (cval[d]) and a per-row presence mask (bit mbit[d] of mask[i] set when row
// i has its entry at offset off[d]), which is what a structured-grid operator with
// constant coefficients reduces to -- 2 bytes per row instead of its values.  For the
// operator A D^{-1} of the Jacobi fold, DIA drops its main diagonal (whose exact value
// is 1) and sets unit_diag.
template <typename V>
struct MatView {
  int fmt;          // 0 CSR, 1 DIA, 2 stencil
  int n;
  const int* __restrict__ row_ptr;
  const int* __restrict__ col;
  const V* __restrict__ val;
  const unsigned short* __restrict__ mask;   // stencil: presence bits per row
  int ndiag;
  int unit_diag;    // DIA / stencil: add x[i] (exact unit main diagonal) before the others
  int off[kMaxDiag];
  V cval[kMaxDiag];                 // stencil: the value at offset off[d]
  unsigned char mbit[kMaxDiag];     // stencil: mask bit of offset off[d]
  int pattern;                      // stencil: stencil_pattern of the offsets (0: none)
};

// Offset patterns of the 3D and 2D stencils (with or without the main diagonal), as kinds
// per offset in ascending order: 0 a nonzero multiple of 4 (an aligned quad), 1 / 2 / 3 the
// offsets -1 / 0 / +1.  A pattern is named by its offset count: 7 (3D), 6 (3D without the
// diagonal), 5 (2D), 4 (2D without the diagonal).
__host__ __device__ constexpr int stencil_kind(int pat, int d) {
  return pat == 7 ? (d < 2 ? 0 : d < 5 ? d - 1 : 0)
       : pat == 6 ? (d < 2 ? 0 : d == 2 ? 1 : d == 3 ? 3 : 0)
       : pat == 5 ? (d == 0 ? 0 : d < 4 ? d : 0)
       : (d == 0 ? 0 : d == 1 ? 1 : d == 2 ? 3 : 0);
}
__host__ __device__ inline int offset_kind(int off) {
  return off == -1 ? 1 : off == 0 ? 2 : off == 1 ? 3 : (off % 4 == 0) ? 0 : -1;
}
// The pattern the ascending offsets off[0 .. nd-1] follow, or 0.
__host__ __device__ inline int stencil_pattern(const int* off, int nd) {
  for (int q = 7; q >= 4; --q) {
    if (nd != q) continue;
    bool match = true;
    for (int d = 0; d < q; ++d) match = match && offset_kind(off[d]) == stencil_kind(q, d);
    return match ? q : 0;
  }
  return 0;
}
// f(d, kind) for d = 0 .. PAT-1 with the kind a compile-time constant.
template <int PAT, int D = 0, typename F>
__device__ __forceinline__ void for_pattern(F& f) {
  if constexpr (D < PAT) {
    f(D, std::integral_constant<int, stencil_kind(PAT, D)>{});
    for_pattern<PAT, D + 1>(f);
  }
}

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
  } else if (A.fmt == 1) {
    if (A.unit_diag) acc = Acc(x[i]);
    const int n = A.n;
#pragma unroll 4
    for (int d = 0; d < A.ndiag; ++d) {
      const int j = i + A.off[d];
      if (j >= 0 && j < n) acc = fma(Acc(__ldg(A.val + (size_t)d * n + i)), Acc(x[j]), acc);
    }
  } else {
    const unsigned msk = __ldg(A.mask + i);
    if (A.unit_diag) acc = Acc(x[i]);
#pragma unroll 4
    for (int d = 0; d < A.ndiag; ++d)
      if ((msk >> A.mbit[d]) & 1u) acc = fma(Acc(A.cval[d]), Acc(x[i + A.off[d]]), acc);
  }
  return acc;
}

// CSR row product split over the L lanes of a lane group (L a power of two <= 32, the
// group's lanes consecutive in a warp and all active): lane `sub` takes entries sub,
// sub + L, ...; the partial sums are combined by shuffles, and every lane of the group
// returns the total.  Shortens the chain of dependent column -> x loads per thread.
template <typename Acc, typename V, typename X>
__device__ __forceinline__ Acc row_dot_lanes(const MatView<V>& A, const X* __restrict__ x, int i, int sub, int L) {
  Acc acc = Acc(0);
  const int e0 = __ldg(A.row_ptr + i), e1 = __ldg(A.row_ptr + i + 1);
  for (int e = e0 + sub; e < e1; e += L) acc = fma(Acc(__ldg(A.val + e)), Acc(x[__ldg(A.col + e)]), acc);
  // the group's own lanes (they may leave the loop above at different times)
  const unsigned lane = threadIdx.x & 31u;
  const unsigned mask = L >= 32 ? 0xffffffffu : (((1u << L) - 1u) << (lane & ~(unsigned)(L - 1)));
  for (int o = L >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o, L);
  return acc;
}

// The same row product with the operand given by a function of the column, so that a
// vector which is a linear combination of stored ones (q = r - alpha s) need not be
// written out before the product reads it at neighbouring rows.
template <typename Acc, typename V, typename F>
__device__ __forceinline__ Acc row_dot_fn(const MatView<V>& A, int i, F xj) {
  Acc acc = Acc(0);
  if (A.fmt == 0) {
    const int e0 = __ldg(A.row_ptr + i), e1 = __ldg(A.row_ptr + i + 1);
    for (int e = e0; e < e1; ++e) acc = fma(Acc(__ldg(A.val + e)), Acc(xj(__ldg(A.col + e))), acc);
  } else if (A.fmt == 1) {
    if (A.unit_diag) acc = Acc(xj(i));
    const int n = A.n;
#pragma unroll 4
    for (int d = 0; d < A.ndiag; ++d) {
      const int j = i + A.off[d];
      if (j >= 0 && j < n) acc = fma(Acc(__ldg(A.val + (size_t)d * n + i)), Acc(xj(j)), acc);
    }
  } else {
    const unsigned msk = __ldg(A.mask + i);
    if (A.unit_diag) acc = Acc(xj(i));
#pragma unroll 4
    for (int d = 0; d < A.ndiag; ++d)
      if ((msk >> A.mbit[d]) & 1u) acc = fma(Acc(A.cval[d]), Acc(xj(i + A.off[d])), acc);
  }
  return acc;
}

// ---------------------------------------------------------------- four rows per thread
// The structured-stencil operator is applied to four consecutive rows i0 .. i0+3 at a
// time (i0 a multiple of 4, n a multiple of 4, 16-byte aligned vectors): own-row vectors
// move as one 128-bit access (two for FP64), and each stencil offset reads the one or two
// aligned quads that hold its four neighbours.  Those loads depend only on the row index
// (a quad is read whenever it lies inside 0 .. n-1), so they are issued together with the
// mask load instead of after it; the mask then decides which products enter each row.
template <typename T> struct Quad { T v[4]; };

template <typename T> __device__ __forceinline__ Quad<T> ld4(const T* p, int i);
template <> __device__ __forceinline__ Quad<float> ld4<float>(const float* p, int i) {
  const float4 f = *reinterpret_cast<const float4*>(p + i);
  return Quad<float>{{f.x, f.y, f.z, f.w}};
}
template <> __device__ __forceinline__ Quad<double> ld4<double>(const double* p, int i) {
  const double2 a = *reinterpret_cast<const double2*>(p + i);
  const double2 b = *reinterpret_cast<const double2*>(p + i + 2);
  return Quad<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, int i, const Quad<float>& q) {
  *reinterpret_cast<float4*>(p + i) = make_float4(q.v[0], q.v[1], q.v[2], q.v[3]);
}
__device__ __forceinline__ void st4(double* p, int i, const Quad<double>& q) {
  *reinterpret_cast<double2*>(p + i) = make_double2(q.v[0], q.v[1]);
  *reinterpret_cast<double2*>(p + i + 2) = make_double2(q.v[2], q.v[3]);
}

// The presence masks of rows i0 .. i0+3 (one 8-byte load).
__device__ __forceinline__ void ld_mask4(const unsigned short* __restrict__ mask, int i0, unsigned (&m)[4]) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(mask + i0));
  m[0] = u.x & 0xffffu; m[1] = u.x >> 16; m[2] = u.y & 0xffffu; m[3] = u.y >> 16;
}

// y_{i0+j} = sum_d c_d x_{i0+j+off_d} over the offsets present in row i0+j (stencil view),
// products summed in ascending offset order as row_dot does: the same value per row.
template <typename Acc, typename V, typename X>
__device__ __forceinline__ Quad<Acc> quad_dot(const MatView<V>& A, const X* __restrict__ x, int i0,
                                              const unsigned (&m)[4]) {
  Quad<Acc> acc;
  if (A.unit_diag) {
    const Quad<X> c = ld4(x, i0);
#pragma unroll
    for (int j = 0; j < 4; ++j) acc.v[j] = Acc(c.v[j]);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) acc.v[j] = Acc(0);
  }
  const int n = A.n;
  // offset d's products
  auto product = [&](int d) {
    const int off = A.off[d];
    const unsigned bit = A.mbit[d];
    const Acc c = Acc(A.cval[d]);
    const int r = off & 3;             // neighbour quad misalignment (two's complement)
    const int a = i0 + off - r;        // first of the aligned quads holding the neighbours
    Quad<X> lo, hi;
    lo.v[0] = lo.v[1] = lo.v[2] = lo.v[3] = X(0);
    hi = lo;
    if (a >= 0 && a < n) lo = ld4(x, a);
    if (r != 0 && a + 4 >= 0 && a + 4 < n) hi = ld4(x, a + 4);
    X e[4];
    if (r == 0) { e[0] = lo.v[0]; e[1] = lo.v[1]; e[2] = lo.v[2]; e[3] = lo.v[3]; }
    else if (r == 1) { e[0] = lo.v[1]; e[1] = lo.v[2]; e[2] = lo.v[3]; e[3] = hi.v[0]; }
    else if (r == 2) { e[0] = lo.v[2]; e[1] = lo.v[3]; e[2] = hi.v[0]; e[3] = hi.v[1]; }
    else { e[0] = lo.v[3]; e[1] = hi.v[0]; e[2] = hi.v[1]; e[3] = hi.v[2]; }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((m[j] >> bit) & 1u) acc.v[j] = fma(c, Acc(e[j]), acc.v[j]);
  };
  if constexpr (std::is_same<Acc, float>::value) {
    if (A.pattern) {
      // FP32, a stencil pattern: the offset kinds are compile-time constants, and the -1, 0
      // and +1 products share the quads i0-4, i0, i0+4 (loaded once, zero outside 0 .. n-1)
      Quad<X> qm, q0, qp;
      qm.v[0] = qm.v[1] = qm.v[2] = qm.v[3] = X(0);
      qp = qm;
      q0 = ld4(x, i0);
      if (i0 >= 4) qm = ld4(x, i0 - 4);
      if (i0 + 4 < n) qp = ld4(x, i0 + 4);
      auto product_k = [&](int d, auto kc) {
        constexpr int K = decltype(kc)::value;
        const unsigned bit = A.mbit[d];
        const Acc c = Acc(A.cval[d]);
        X e[4];
        if constexpr (K == 1) { e[0] = qm.v[3]; e[1] = q0.v[0]; e[2] = q0.v[1]; e[3] = q0.v[2]; }
        else if constexpr (K == 2) { e[0] = q0.v[0]; e[1] = q0.v[1]; e[2] = q0.v[2]; e[3] = q0.v[3]; }
        else if constexpr (K == 3) { e[0] = q0.v[1]; e[1] = q0.v[2]; e[2] = q0.v[3]; e[3] = qp.v[0]; }
        else {
          const int a = i0 + A.off[d];   // a multiple of 4
          Quad<X> q;
          q.v[0] = q.v[1] = q.v[2] = q.v[3] = X(0);
          if (a >= 0 && a < n) q = ld4(x, a);
          e[0] = q.v[0]; e[1] = q.v[1]; e[2] = q.v[2]; e[3] = q.v[3];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if ((m[j] >> bit) & 1u) acc.v[j] = fma(c, Acc(e[j]), acc.v[j]);
      };
      switch (A.pattern) {
        case 7: for_pattern<7>(product_k); return acc;
        case 6: for_pattern<6>(product_k); return acc;
        case 5: for_pattern<5>(product_k); return acc;
        default: for_pattern<4>(product_k); return acc;
      }
    }
    // FP32: with the offset count known at compile time (4-7: the 2D and 3D stencils, with
    // or without the main diagonal) the loop unrolls and the offsets become constant-bank
    // operands whose tests are loop-invariant (measured 1% faster per iteration on the 2D
    // mixed solve; the FP64 builds, bound by the FP64 pipe, were 1-4% slower so)
    switch (A.ndiag) {
      case 4:
#pragma unroll
        for (int d = 0; d < 4; ++d) product(d);
        return acc;
      case 5:
#pragma unroll
        for (int d = 0; d < 5; ++d) product(d);
        return acc;
      case 6:
#pragma unroll
        for (int d = 0; d < 6; ++d) product(d);
        return acc;
      case 7:
#pragma unroll
        for (int d = 0; d < 7; ++d) product(d);
        return acc;
      default:
        break;
    }
  }
#pragma unroll 2
  for (int d = 0; d < A.ndiag; ++d) product(d);
  return acc;
}

// ---------------------------------------------------------------- time
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------- bulk copies (TMA, untiled)
// One thread moves a contiguous range global -> shared with cp.async.bulk; the copy counts
// its bytes off an mbarrier (complete_tx), which the consumers wait on with a phase parity.
__device__ __forceinline__ unsigned smem_addr(const void* q) { return (unsigned)__cvta_generic_to_shared(q); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for the phase with the given parity: false after timeout_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned long long timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  unsigned spins = 0;
  while (!mbar_try_wait(bar, parity))
    if ((++spins & 15u) == 0 && global_ns() - t0 > timeout_ns) return false;
  return true;
}
// bytes: a multiple of 16; dst and src 16-byte aligned.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Bring a contiguous range into L2 without waiting for it (bytes: a multiple of 16; src
// 16-byte aligned).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// Generic-proxy writes (earlier plain stores, seen through a grid barrier) before async-proxy
// reads of global memory; an initialised mbarrier before the async proxy signals it.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory layout of one stage of the staged stencil sweeps (two quads of four rows
// per thread, R = 8 x threads rows per trip), the same on the host (dynamic shared memory
// size) and the device: a near window of the gathered vector, rows [base - H, base + R + H)
// with H the largest offset of magnitude <= R rounded up to 4 (at least 4); one R-row window
// per farther offset (at base + offset, which must be a multiple of 4); R + 8 row masks from
// the multiple of 8 at or below base (16-byte bulk copies; the mask array is padded to a
// multiple of 8 rows plus 8).  The source vector's own rows are read from global memory (one
// coalesced 16-byte load per quad), which leaves the L1 share of the unified cache to the
// other passes.  Sizes in floats; every part starts on a 16-byte boundary.
struct StageLayout {
  int R, H, nfar;
  int far[kMaxDiag];
  int src_f, mask_f, stage_f;   // offsets of the parts within a stage, and its size
  int ok;                       // 0: an offset this layout cannot stage
};

__host__ __device__ inline void stage_layout(StageLayout& L, const int* off, int ndiag, int R) {
  L.R = R;
  L.H = 0;
  L.nfar = 0;
  L.ok = 1;
  for (int d = 0; d < ndiag; ++d) {
    const int a = off[d] < 0 ? -off[d] : off[d];
    if (a <= R) {
      L.H = a > L.H ? a : L.H;
    } else {
      if (off[d] % 4 != 0) L.ok = 0;
      L.far[L.nfar++] = off[d];
    }
  }
  L.H = (L.H + 3) / 4 * 4;
  if (L.H < 4) L.H = 4;   // the sweep reads up to 3 rows beyond a warp's first and last quad
  if (R % 8 != 0) L.ok = 0;
  L.src_f = (R + 2 * L.H) + L.nfar * R;
  L.mask_f = L.src_f;   // the source rows are read from global memory
  L.stage_f = L.mask_f + (R + 8) / 2;    // R + 8 16-bit masks
}

// Hint: bring the 128-byte line holding *ptr into L2 (no register is written, so a
// thread can request the next row's operands while it computes the current one).
template <typename V>
__device__ __forceinline__ void prefetch_l2(const V* ptr) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

// ---------------------------------------------------------------- timing / sync
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier over `nblk` co-resident blocks (a cooperatively launched grid, or one
// team of blocks inside it).  The counter is monotone within a launch: barrier
// number `epoch` (1, 2, ...) completes when it reaches epoch * nblk.  Thread 0 of each block arrives (release) and polls
// (acquire); the poll gives up after timeout_ns and raises *err = kTimeout.
// Returns false when the grid must stop (timeout here or elsewhere).
__device__ __forceinline__ bool grid_barrier(unsigned* counter, unsigned epoch, unsigned nblk, int* err,
                                             unsigned long long timeout_ns) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    red_release_add(counter, 1u);
    const unsigned target = epoch * nblk;
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

// The same barrier in two halves, so that a block can do work that needs no other block's
// writes between its arrival and its wait (the single-GPU form of hiding a global
// reduction behind computation).  grid_arrive publishes this block's earlier writes
// (block-wide __syncthreads, then one release by thread 0); grid_wait returns once all
// nblk blocks arrived at barrier `epoch` (false: timeout here or elsewhere).
__device__ __forceinline__ void grid_arrive(unsigned* counter) {
  __syncthreads();
  if (threadIdx.x == 0) red_release_add(counter, 1u);
}

__device__ __forceinline__ bool grid_wait(unsigned* counter, unsigned epoch, unsigned nblk, int* err,
                                          unsigned long long timeout_ns) {
  __shared__ int s_ok2;
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = epoch * nblk;
    const unsigned long long t0 = global_ns();
    unsigned spins = 0;
    while (ld_acquire_u32(counter) < target) {
      if ((++spins & 63u) == 0 && (global_ns() - t0 > timeout_ns || *(volatile int*)err)) {
        atomicCAS(err, 0, (int)kTimeout);
        ok = 0;
        break;
      }
    }
    __threadfence();
    if (ok && *(volatile int*)err) ok = 0;
    s_ok2 = ok;
  }
  __syncthreads();
  return s_ok2 != 0;
}

// ---------------------------------------------------------------- reductions
// FP64 arithmetic is scarce on GB300 (about 2 lane-FMAs per SM per cycle), so the
// reductions are written to issue few FP64 instructions:
//  * warp level: a "transpose" butterfly.  With P (power of two) values per lane,
//    the first log2(P) shuffle levels exchange half of the values and halve the
//    count, so P values cost P-1 adds plus the remaining plain levels (8 values: 9
//    adds instead of 40).  Afterwards lane l holds the total of value
//    vidx<P>(l).
//  * block level: one value per (warp, index) in shared memory, reduced by warp 0.
//  * grid level: warp 0 of every block sums all blocks' partials in a fixed order.
// All orders are fixed, so results are bitwise reproducible for a given launch
// shape, and every block obtains bit-identical totals.
constexpr unsigned kFull = 0xffffffffu;

template <int P>
__device__ __forceinline__ int vidx(int lane) {
  int j = 0;
#pragma unroll
  for (int k = 0, off = 16; (1 << k) < P; ++k, off >>= 1) j |= ((lane & off) ? 1 : 0) << k;
  return j;
}

template <int P>
__device__ __forceinline__ double warp_transpose_sum(double (&v)[P]) {
  const int lane = threadIdx.x & 31;
  int off = 16;
#pragma unroll
  for (int cnt = P; cnt > 1; cnt >>= 1) {
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int j = 0; j < cnt / 2; ++j) {
      const double keep = upper ? v[2 * j + 1] : v[2 * j];
      const double send = upper ? v[2 * j] : v[2 * j + 1];
      v[j] = keep + __shfl_xor_sync(kFull, send, off);
    }
    off >>= 1;
  }
  double s = v[0];
#pragma unroll
  for (; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
  return s;
}

template <int ND> struct Pad {
  static constexpr int value = ND <= 1 ? 1 : ND <= 2 ? 2 : ND <= 4 ? 4 : ND <= 8 ? 8 : 16;
};

// Block-wide sums of ND per-thread doubles; block totals land in out_smem[0..ND)
// (valid after the trailing __syncthreads).  work_smem: >= kWork doubles.
template <int ND>
__device__ __forceinline__ void block_reduce(const double (&in)[ND], double* work_smem, double* out_smem) {
  constexpr int P = Pad<ND>::value;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double v[P];
#pragma unroll
  for (int j = 0; j < P; ++j) v[j] = j < ND ? in[j] : 0.0;
  const double s = warp_transpose_sum<P>(v);
  const int j = vidx<P>(lane);
  if ((lane & (32 / P - 1)) == 0) work_smem[j * 32 + wid] = s;
  __syncthreads();
  if (wid == 0) {
    double w[P];
#pragma unroll
    for (int q = 0; q < P; ++q) w[q] = lane < nw ? work_smem[q * 32 + lane] : 0.0;
    const double t = warp_transpose_sum<P>(w);
    if ((lane & (32 / P - 1)) == 0 && j < ND) out_smem[j] = t;
  }
  __syncthreads();
}

// Block totals of ND per-thread values written to part[bid * kMaxDots + d].
template <int ND>
__device__ __forceinline__ void block_publish(double (&v)[ND], double* smem, double* part, int bid) {
  block_reduce<ND>(v, smem, smem + kWork);
  if (threadIdx.x < ND) part[bid * kMaxDots + threadIdx.x] = smem[kWork + threadIdx.x];
}

// Block-wide sum returning the totals to every thread (used outside the solver loop).
template <int ND>
__device__ __forceinline__ void block_sum(double (&v)[ND], double* smem) {
  block_reduce<ND>(v, smem, smem + kWork);
#pragma unroll
  for (int d = 0; d < ND; ++d) v[d] = smem[kWork + d];
  __syncthreads();
}

// After a grid barrier: warp 0 of every block sums all blocks' partials in one fixed
// order, so every block obtains bit-identical totals (the GLRED result).
template <int ND>
__device__ __forceinline__ void grid_combine(const double* part, int nblk, double (&out)[ND], double* smem) {
  constexpr int P = Pad<ND>::value;
  const int lane = threadIdx.x & 31;
  double* res = smem + kWork;
  if (threadIdx.x < 32) {
    double v[P];
#pragma unroll
    for (int j = 0; j < P; ++j) v[j] = 0.0;
    for (int b = lane; b < nblk; b += 32) {
#pragma unroll
      for (int d = 0; d < ND; ++d) v[d] += __ldcg(part + b * kMaxDots + d);
    }
    const double t = warp_transpose_sum<P>(v);
    const int j = vidx<P>(lane);
    if ((lane & (32 / P - 1)) == 0 && j < ND) res[j] = t;
  }
  __syncthreads();
#pragma unroll
  for (int d = 0; d < ND; ++d) out[d] = res[d];
  __syncthreads();
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
