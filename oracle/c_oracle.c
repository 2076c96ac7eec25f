/* C oracle: Algorithm 2 (p-BiCGStab) of arXiv 1809.01948 with the residual replacement
 * step of Eq. (rr) and its policies, in FP64 and in the mixed FP32/FP64 emulation, on all
 * host cores (OpenMP).  TEST INFRASTRUCTURE ONLY: only tests/ and the CPU legs of
 * bench.py (the cpu_baseline and the reference arm) load it; it shares no code with the
 * CUDA library.  It restates the numpy oracle (oracle/krylov.py) step for step -- the same
 * readings, evaluation order and brackets -- so that the CPU baseline can run the
 * benchmark workloads to completion; tests/test_oracle_c.py pins it to the numpy oracle.
 * Compiled with -ffp-contract=off (no fused multiply-adds). */
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int n;
  const int* row_ptr;
  const int* col;
  const double* val;
} csr_t;

typedef struct {
  double tol;
  int max_it;
  int rr_period;
  double rr_theta;
  int restart_period;
  int stag_window;
  int max_restarts;
} oracle_opts;

typedef struct {
  int status, iterations, n_replacements, n_restarts;
  double rel_res_recursive, rel_res_true;
} oracle_result;

#define T double
#define FN(name) name##_f64
#include "c_oracle_body.h"
#undef T
#undef FN
#define T float
#define FN(name) name##_f32
#include "c_oracle_body.h"
#undef T
#undef FN

/* kind: 0 none, 1 Jacobi, 2 Neumann of the given degree; mixed: FP32 vectors and values.
 * Returns 0, or -1 (allocation failure). */
int oracle_pbicgstab(int n, const int* row_ptr, const int* col, const double* val, int kind, int degree,
                     int mixed, const double* b, double* x, const oracle_opts* o, oracle_result* res,
                     int nthreads) {
  if (nthreads > 0) omp_set_num_threads(nthreads);
  csr_t A = {n, row_ptr, col, val};
  const int nnz = row_ptr[n];
  double* dinv = (double*)malloc(sizeof(double) * (size_t)n);
  if (!dinv) return -1;
  for (int i = 0; i < n; ++i) {
    double d = 0.0;
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
      if (col[e] == i) d = val[e];
    dinv[i] = kind ? 1.0 / d : 1.0;
  }
  int rc;
  if (!mixed) {
    rc = pbicgstab_f64(&A, val, dinv, kind, degree, b, x, o, res);
  } else {
    float* v32 = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    float* d32 = (float*)malloc(sizeof(float) * (size_t)n);
    if (!v32 || !d32) { free(v32); free(d32); free(dinv); return -1; }
    for (int e = 0; e < nnz; ++e) v32[e] = (float)val[e];
    for (int i = 0; i < n; ++i) d32[i] = (float)dinv[i];
    rc = pbicgstab_f32(&A, v32, d32, kind, degree, b, x, o, res);
    free(v32);
    free(d32);
  }
  free(dinv);
  return rc;
}

/* Host memory bandwidth: a parallel copy of n doubles, best of reps, bytes read + written
 * per second (the roofline of the CPU oracle). */
double oracle_stream_copy_gbs(long n, int reps, int nthreads) {
  if (nthreads > 0) omp_set_num_threads(nthreads);
  double* a = (double*)malloc(sizeof(double) * (size_t)n);
  double* c = (double*)malloc(sizeof(double) * (size_t)n);
  if (!a || !c) { free(a); free(c); return -1.0; }
#pragma omp parallel for schedule(static)
  for (long i = 0; i < n; ++i) { a[i] = (double)i; c[i] = 0.0; }
  double best = 1e30;
  for (int r = 0; r < reps; ++r) {
    const double t0 = omp_get_wtime();
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) c[i] = a[i];
    const double dt = omp_get_wtime() - t0;
    if (dt < best) best = dt;
  }
  const double gbs = 16.0 * (double)n / best / 1e9 + 0.0 * c[n / 2];
  free(a);
  free(c);
  return gbs;
}

int oracle_threads(void) { return omp_get_max_threads(); }
