/* Body of the C oracle for one vector precision (included by c_oracle.c with T = double
 * and T = float).  TEST INFRASTRUCTURE ONLY; see c_oracle.c.
 *
 * Every loop over rows is an OpenMP static partition; every dot product sums each
 * thread's block in index order and then the thread partials in thread order, so a
 * result depends only on the thread count.  Element-wise operations are evaluated in T
 * with the brackets and left-to-right order of Eq. (auxrec) (compiled without
 * floating-point contraction), exactly as the numpy oracle evaluates them. */

/* y = A v in T (stored values in T, each row summed in ascending column order) */
static void FN(spmv)(const csr_t* A, const T* vals, const T* v, T* y) {
  const int n = A->n;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    T s = (T)0;
    for (int e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e) s += vals[e] * v[A->col[e]];
    y[i] = s;
  }
}

/* M^{-1} v: identity, Jacobi D^{-1} v, or the Neumann sweeps y_0 = D^{-1} v,
 * y_j = y_{j-1} + D^{-1} (v - A y_{j-1}) (the polynomial sum_{j<=d} (I - D^{-1}A)^j D^{-1}) */
static void FN(prec)(const csr_t* A, const T* vals, const T* dinv, int kind, int degree, const T* v, T* y, T* tmp) {
  const int n = A->n;
  if (kind == 0) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) y[i] = v[i];
    return;
  }
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) y[i] = dinv[i] * v[i];
  if (kind == 1) return;
  for (int j = 0; j < degree; ++j) {
    FN(spmv)(A, vals, y, tmp);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) y[i] = y[i] + dinv[i] * (v[i] - tmp[i]);
  }
}

/* (a, b) in FP64 from T inputs: fixed-order partials per thread, then thread order */
static double FN(dot)(int n, const T* a, const T* b, double* part) {
  int nt = 1;
#pragma omp parallel
  {
    const int t = omp_get_thread_num();
#pragma omp single
    nt = omp_get_num_threads();
    double s = 0.0;
#pragma omp for schedule(static)
    for (int i = 0; i < n; ++i) s += (double)a[i] * (double)b[i];
    part[t] = s;
  }
  double tot = 0.0;
  for (int t = 0; t < nt; ++t) tot += part[t];
  return tot;
}

/* r = fl_T(b - A64 x): the residual in FP64 with the FP64 values, rounded to T */
static void FN(residual)(const csr_t* A, const double* b, const double* x, T* r) {
  const int n = A->n;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e) s += A->val[e] * x[A->col[e]];
    r[i] = (T)(b[i] - s);
  }
}

/* Algorithm 2 with Eq. (rr) and the restart policy; the readings match the numpy oracle:
 * R2 shadow = r_0, R3 zero vectors at i = -1, R5 stop / verify / force, R6 placement,
 * R7 period with the sqrt(eps) cutoff, R8 relative trigger, R15 breakdowns, R20 periodic
 * restart, R21 progress window (best (re)start iterate). */
static int FN(pbicgstab)(const csr_t* A, const T* vals, const T* dinv, int kind, int degree, const double* b,
                         double* x, const oracle_opts* o, oracle_result* res) {
  const int n = A->n;
  const size_t nb = sizeof(T) * (size_t)n;
  T* buf = (T*)malloc(nb * 20);
  double* part = (double*)malloc(sizeof(double) * 1024);
  double* xbest = (double*)malloc(sizeof(double) * (size_t)n);
  double* r64 = (double*)malloc(sizeof(double) * (size_t)n);
  if (!buf || !part || !xbest || !r64) { free(buf); free(part); free(xbest); free(r64); return -1; }
  T *r = buf, *rh = buf + n, *k = buf + 2 * n, *w = buf + 3 * n, *m = buf + 4 * n, *t = buf + 5 * n;
  T *g = buf + 6 * n, *s = buf + 7 * n, *l = buf + 8 * n, *z = buf + 9 * n, *nv = buf + 10 * n, *v = buf + 11 * n;
  T *q = buf + 12 * n, *u = buf + 13 * n, *y = buf + 14 * n, *rn = buf + 15 * n, *kn = buf + 16 * n;
  T *wn = buf + 17 * n, *tmp = buf + 18 * n, *tmp2 = buf + 19 * n;
  const double eps = 2.220446049250313e-16;
  const int any_rr = o->rr_period > 0 || o->rr_theta > 0.0;
  double bnorm = 0.0;
  for (int i = 0; i < n; ++i) bnorm += b[i] * b[i];
  bnorm = sqrt(bnorm);
  memset(res, 0, sizeof *res);
  res->status = 4;
  if (bnorm == 0.0) {
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    res->status = 0;
    free(buf); free(part); free(xbest); free(r64);
    return 0;
  }
  int it = 0, nbd = 0, nper = 0, first = 1, have_best = 0;
  double rn0 = 0.0, ref_true = INFINITY, best_true = INFINITY, rnv = 0.0;
  int ref_it = 0;
  for (;;) {
    /* initialisation of Algorithm 2 */
    FN(residual)(A, b, x, r);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
      double sacc = 0.0;
      for (int e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e) sacc += A->val[e] * x[A->col[e]];
      r64[i] = b[i] - sacc;
    }
    memcpy(rh, r, nb);
    FN(prec)(A, vals, dinv, kind, degree, r, k, tmp);
    FN(spmv)(A, vals, k, w);
    FN(prec)(A, vals, dinv, kind, degree, w, m, tmp);
    FN(spmv)(A, vals, m, t);
    double rho = FN(dot)(n, rh, r, part), rw = FN(dot)(n, rh, w, part);
    double rn_ = sqrt(FN(dot)(n, r, r, part));
    double rt = 0.0;
    for (int i = 0; i < n; ++i) rt += r64[i] * r64[i];
    rt = sqrt(rt);
    rnv = rn_;
    if (first) rn0 = rn_;
    const int it_start = it;
    if (rt <= o->tol * bnorm) { res->status = 0; break; }
    if (o->stag_window > 0) {
      if (rt <= 0.5 * ref_true) { ref_true = rt; ref_it = it; }
      else if (it - ref_it >= o->stag_window) {
        if (have_best && best_true < rt) memcpy(x, xbest, sizeof(double) * (size_t)n);
        res->status = 6;
        break;
      }
      if (rt < best_true) { best_true = rt; memcpy(xbest, x, sizeof(double) * (size_t)n); have_best = 1; }
    }
    double alpha = rw != 0.0 ? rho / rw : INFINITY;
    if (rw == 0.0 || !isfinite(alpha)) { res->status = 5; break; }
    double beta = 0.0, omega_prev = 0.0, rn_last_rr = rn_;
    memset(g, 0, nb); memset(s, 0, nb); memset(l, 0, nb); memset(z, 0, nb); memset(nv, 0, nb); memset(v, 0, nb);
    first = 0;
    int restart = 0;
    while (it < o->max_it) {
      const int i_ = it;
      const T a_ = (T)alpha, b_ = (T)beta, wp_ = (T)omega_prev;
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) {
        g[i] = k[i] + b_ * (g[i] - wp_ * l[i]);
        s[i] = w[i] + b_ * (s[i] - wp_ * z[i]);
        l[i] = m[i] + b_ * (l[i] - wp_ * nv[i]);
        z[i] = t[i] + b_ * (z[i] - wp_ * v[i]);
        q[i] = r[i] - a_ * s[i];
        u[i] = k[i] - a_ * l[i];
        y[i] = w[i] - a_ * z[i];
      }
      const double qy = FN(dot)(n, q, y, part), yy = FN(dot)(n, y, y, part);
      FN(prec)(A, vals, dinv, kind, degree, z, nv, tmp);
      FN(spmv)(A, vals, nv, v);
      const double omega = yy == 0.0 ? 0.0 : qy / yy;
      if (!isfinite(omega)) {
        if (nbd < o->max_restarts) { ++nbd; ++it; restart = 1; break; }
        res->status = 5;
        break;
      }
      const T o_ = (T)omega;
      int do_rr = 0;
      if (o->rr_period > 0 && i_ > 0 && i_ % o->rr_period == 0 && rnv >= sqrt(eps) * rn0) do_rr = 1;
      if (o->rr_theta > 0.0 && rnv <= o->rr_theta * rn_last_rr) do_rr = 1;
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) {
        x[i] = (x[i] + alpha * (double)g[i]) + omega * (double)u[i];
        rn[i] = q[i] - o_ * y[i];
        kn[i] = u[i] - o_ * (m[i] - a_ * nv[i]);
        wn[i] = y[i] - o_ * (t[i] - a_ * v[i]);
      }
      memcpy(r, rn, nb); memcpy(k, kn, nb); memcpy(w, wn, nb);
      if (do_rr) {   /* Eq. (rr): r = b - A x, k = M^{-1} r, w = A k, s = A g, l = M^{-1} s, z = A l */
        FN(residual)(A, b, x, r);
        FN(prec)(A, vals, dinv, kind, degree, r, k, tmp);
        FN(spmv)(A, vals, k, w);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) {
          double sacc = 0.0;
          for (int e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e) sacc += A->val[e] * (double)g[A->col[e]];
          s[i] = (T)sacc;
        }
        FN(prec)(A, vals, dinv, kind, degree, s, l, tmp2);
        FN(spmv)(A, vals, l, z);
        res->n_replacements++;
      }
      double rho_new = FN(dot)(n, rh, r, part), rwv = FN(dot)(n, rh, w, part);
      double rs = FN(dot)(n, rh, s, part), rz = FN(dot)(n, rh, z, part);
      double rr2 = FN(dot)(n, r, r, part);
      FN(prec)(A, vals, dinv, kind, degree, w, m, tmp);
      FN(spmv)(A, vals, m, t);
      res->iterations = i_ + 1;
      rnv = sqrt(rr2);
      if (rnv <= o->tol * bnorm) {   /* R5: verify with the FP64 true residual */
        double tr = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : tr)
        for (int i = 0; i < n; ++i) {
          double sacc = 0.0;
          for (int e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e) sacc += A->val[e] * x[A->col[e]];
          tr += (b[i] - sacc) * (b[i] - sacc);
        }
        tr = sqrt(tr);
        if (tr <= o->tol * bnorm) { res->status = 0; break; }
        if (!any_rr) {
          if (o->restart_period > 0) { ++nper; ++it; restart = 1; break; }
          res->status = 6;
          break;
        }
        FN(residual)(A, b, x, r);   /* forced replacement */
        FN(prec)(A, vals, dinv, kind, degree, r, k, tmp);
        FN(spmv)(A, vals, k, w);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) {
          double sacc = 0.0;
          for (int e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e) sacc += A->val[e] * (double)g[A->col[e]];
          s[i] = (T)sacc;
        }
        FN(prec)(A, vals, dinv, kind, degree, s, l, tmp2);
        FN(spmv)(A, vals, l, z);
        res->n_replacements++;
        do_rr = 1;
        rho_new = FN(dot)(n, rh, r, part); rwv = FN(dot)(n, rh, w, part);
        rs = FN(dot)(n, rh, s, part); rz = FN(dot)(n, rh, z, part);
        rnv = sqrt(FN(dot)(n, r, r, part));
        FN(prec)(A, vals, dinv, kind, degree, w, m, tmp);
        FN(spmv)(A, vals, m, t);
      }
      if (do_rr) rn_last_rr = rnv;
      if (omega == 0.0 || rho == 0.0) {
        if (nbd < o->max_restarts) { ++nbd; ++it; restart = 1; break; }
        res->status = 5;
        break;
      }
      const double beta_new = (alpha / omega) * (rho_new / rho);
      const double den = (rwv + beta_new * rs) - (beta_new * omega) * rz;
      const double alpha_new = den != 0.0 ? rho_new / den : INFINITY;
      if (!(isfinite(beta_new) && den != 0.0 && isfinite(alpha_new))) {
        if (nbd < o->max_restarts) { ++nbd; ++it; restart = 1; break; }
        res->status = 5;
        break;
      }
      alpha = alpha_new; beta = beta_new; omega_prev = omega; rho = rho_new;
      ++it;
      if (o->restart_period > 0 && it - it_start >= o->restart_period) { ++nper; restart = 1; break; }
    }
    if (!restart) break;
  }
  if (res->status == 4 && have_best) {   /* R21 at max_it: the better of last and best */
    double tr = 0.0;
    for (int i = 0; i < n; ++i) {
      double sacc = 0.0;
      for (int e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e) sacc += A->val[e] * x[A->col[e]];
      tr += (b[i] - sacc) * (b[i] - sacc);
    }
    if (best_true < sqrt(tr)) memcpy(x, xbest, sizeof(double) * (size_t)n);
  }
  res->n_restarts = nbd + nper;
  res->rel_res_recursive = rnv / bnorm;
  double tr = 0.0;
  for (int i = 0; i < n; ++i) {
    double sacc = 0.0;
    for (int e = A->row_ptr[i]; e < A->row_ptr[i + 1]; ++e) sacc += A->val[e] * x[A->col[e]];
    tr += (b[i] - sacc) * (b[i] - sacc);
  }
  res->rel_res_true = sqrt(tr) / bnorm;
  free(buf); free(part); free(xbest); free(r64);
  return 0;
}
