/*
 * Plain FP64 CPU oracle for restarted PDHG on the LP of Eq. (LP)
 * (arXiv 2312.14832, Section 2 "Overview of the Method").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product solver never
 * calls it and shares no code with it.
 *
 * It is written for a reader checking it against the paper by eye: plain loops,
 * one step after another in the paper's order, no blocking or fusion, IEEE double
 * everywhere (build with -ffp-contract=off so no FMA contraction happens).
 *
 * Problem (Eq. LP):  min c'x  s.t.  Ax = b, Gx >= h, l <= x <= u,
 *                    K = [A; G] (rows 0..m1-1 are A), q = [b; h].
 * Saddle point (Eq. saddle-point): min_{x in X} max_{y in Y} c'x - y'Kx + q'y,
 *                    X = [l, u], Y = R^{m1} x R_+^{m2}.
 *
 * Readings of points the paper leaves open (each is a choice of this code):
 *  - Lambda_i (Section 2): both bounds infinite -> {0}; only u finite -> R^-;
 *    only l finite -> R^+ (the printed "l_i = +inf" is read as u_i = +inf);
 *    both finite -> R.
 *  - lambda^+ = max(lambda, 0), lambda^- = max(-lambda, 0); a product of a zero
 *    multiplier and an infinite bound is 0 (Lambda makes these the only cases).
 *  - Step size eta is constant: step_scale / ||K||_2, ||K||_2 from power_iters
 *    power iterations on K'K from v0 = 1/sqrt(n); eta = 1 when ||K||_2 = 0.
 *  - step_rule = 1 replaces it by the adaptive rule of the cited PDLP paper
 *    (Applegate et al., "Practical large-scale linear programming using
 *    primal-dual hybrid gradient"): a step with eta is accepted when
 *      eta <= eta_max = (omega ||dx||^2 + ||dy||^2 / omega) / (2 |dy' K dx|)
 *    (eta_max = +inf when dy' K dx = 0), and either way the next eta is
 *      min((1 - (s+1)^-0.3) eta_max, (1 + (s+1)^-0.6) eta),
 *    s = 1 + the number of steps accepted so far.  A rejected attempt leaves the
 *    point unchanged; after reject_cap rejections in a row (64 by default; a
 *    safeguard of this implementation, the cited rule has none) the attempt is
 *    accepted.  The
 *    first eta is 1 / max_ij |K_ij| (of the scaled K; 1 when K = 0).  The average
 *    of an inner loop is weighted by the accepted steps' eta.  Iteration counts
 *    (k, t, max_iter, check_every) count attempts.
 *  - Initial primal weight omega0 = ||c||/||q|| when both exceed 1e-10, else 1.
 *  - At a restart the primal weight becomes
 *      omega <- exp(theta log(dy/dx) + (1-theta) log omega),
 *    dx = ||x^{n+1,0} - x^{n,0}||, dy likewise, when both exceed 1e-10.
 *  - The average is uniform over the iterates 1..t of the current inner loop.
 *  - The restart goes to the candidate z_c (current or average).
 *  - Restart conditions and termination are evaluated every check_every
 *    iterations and at k = max_iter; condition 2 compares with the candidate of
 *    the previous check of the same inner loop (+inf at its first check).
 *  - k counts all PDHG steps taken so far, including the current one.
 *  - KKT_omega (restarts) is measured on the scaled problem; the termination
 *    tests on the original, unscaled problem.
 *  - At a check both the current iterate and the average are tested; the one
 *    passing is returned (the smaller largest relative error if both pass; a tie
 *    goes to the average).  At the iteration limit the same rule picks the output.
 *  - Scaling (when enabled): ruiz_iters passes of Ruiz equilibration (rows and
 *    columns divided by the square root of their infinity norms, both computed
 *    from the matrix at the start of the pass), then one Pock-Chambolle pass with
 *    alpha = 1 (square roots of the 1-norms).  Empty rows/columns keep factor 1.
 *    With Kt = Dr K Dc:  ct = Dc c, qt = Dr q, lt = l / Dc, ut = u / Dc,
 *    x = Dc xt, y = Dr yt.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double tol;          /* relative tolerance epsilon of the three termination tests */
  int64_t max_iter;
  int32_t check_every;
  int32_t scaling;     /* 0 off, 1 Ruiz + Pock-Chambolle */
  double beta_suff, beta_nec, beta_art;   /* 0.2, 0.8, 0.36 (restart conditions) */
  double step_scale;   /* eta = step_scale / ||K||_2 */
  double omega_theta;  /* smoothing of the primal-weight update */
  int32_t ruiz_iters;
  int32_t power_iters;
  double eta;          /* > 0: use this step size instead of the power-iteration rule */
  double omega0;       /* > 0: use this initial primal weight */
  int32_t step_rule;   /* 0 constant eta, 1 adaptive (PDLP) */
  int32_t reject_cap;  /* adaptive rule: an attempt is kept after this many rejections in a
                          row (a safeguard of this implementation, 64 by default; 0 keeps
                          every attempt) */
} orc_params;

typedef struct {
  int32_t status;      /* 0 optimal, 1 iteration limit */
  int32_t which;       /* returned point: 0 current iterate, 1 average */
  int64_t iters, restarts;
  double primal_obj, dual_obj, rel_primal, rel_dual, rel_gap, kkt_omega, omega, eta;
  int64_t accepted;    /* steps accepted (= iters with the constant rule) */
  int64_t checks;      /* checks made (restart / termination tests) */
} orc_result;

typedef struct {
  double pres2, dres2, pobj, dobj, gap;
} orc_kkt;

/* One record per check of orc_solve (optional output). */
typedef struct {
  int64_t k, t;        /* iteration count and inner-loop length at the check */
  int32_t restart;     /* 0 none (or the solve ended here), 1/2/3 the restart condition that held */
  int32_t candidate;   /* restart candidate: 0 current iterate, 1 average */
  double omega;        /* primal weight in force at the check (before any update) */
  double kkt_cur, kkt_avg, kkt_anchor;   /* KKT_omega (scaled problem) of z, z-bar, z^{n,0} */
  double rel_primal, rel_dual, rel_gap;  /* relative tests of the point with the smaller largest ratio */
} orc_check;

/* ---------- linear algebra on CSR ---------- */

/* y = K x, row by row. */
void orc_spmv(int64_t m, const int64_t* rp, const int32_t* ci, const double* v,
              const double* x, double* y) {
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * x[ci[k]];
    y[i] = s;
  }
}

/* g = K' y, scattering each row of K. */
void orc_spmv_t(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci,
                const double* v, const double* y, double* g) {
  for (int64_t j = 0; j < n; ++j) g[j] = 0.0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) g[ci[k]] += v[k] * y[i];
}

static double norm2(int64_t n, const double* a) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * a[i];
  return sqrt(s);
}

static double dist2(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += (a[i] - b[i]) * (a[i] - b[i]);
  return sqrt(s);
}

/* ---------- projections (Section 2) ---------- */

/* proj_Lambda for one coordinate: the cone of bound multipliers. */
double orc_proj_lambda(double d, double l, double u) {
  int lf = isfinite(l), uf = isfinite(u);
  if (!lf && !uf) return 0.0;            /* {0}  */
  if (!lf && uf) return d < 0.0 ? d : 0.0; /* R^-  */
  if (lf && !uf) return d > 0.0 ? d : 0.0; /* R^+  */
  return d;                               /* R    */
}

static double proj_box(double x, double l, double u) {
  if (x < l) return l;
  if (x > u) return u;
  return x;
}

/* ---------- KKT quantities (Section 2, termination criteria and KKT_omega) ---------- */

/* Residual parts of (x, y) for the LP (K, c, q, l, u, m1):
 *   pres2 = ||(Ax - b, [h - Gx]^+)||^2
 *   dres2 = ||c - K'y - lambda||^2,  lambda = proj_Lambda(c - K'y)
 *   pobj  = c'x,  dobj = q'y + l'lambda^+ - u'lambda^-,  gap = dobj - pobj */
orc_kkt orc_kkt_parts(int64_t m, int64_t n, int64_t m1, const int64_t* rp, const int32_t* ci,
                      const double* v, const double* c, const double* q, const double* l,
                      const double* u, const double* x, const double* y) {
  orc_kkt r = {0, 0, 0, 0, 0};
  double* Kx = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  double* g = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  orc_spmv(m, rp, ci, v, x, Kx);
  orc_spmv_t(m, n, rp, ci, v, y, g);
  for (int64_t i = 0; i < m; ++i) {
    double ri;
    if (i < m1) ri = Kx[i] - q[i];
    else ri = (q[i] - Kx[i] > 0.0) ? (q[i] - Kx[i]) : 0.0;
    r.pres2 += ri * ri;
  }
  double qy = 0.0, lterm = 0.0, cx = 0.0;
  for (int64_t i = 0; i < m; ++i) qy += q[i] * y[i];
  for (int64_t j = 0; j < n; ++j) {
    double d = c[j] - g[j];
    double lam = orc_proj_lambda(d, l[j], u[j]);
    r.dres2 += (d - lam) * (d - lam);
    if (lam > 0.0) lterm += l[j] * lam;        /* l' lambda^+   */
    else if (lam < 0.0) lterm -= u[j] * (-lam); /* - u' lambda^- */
    cx += c[j] * x[j];
  }
  r.pobj = cx;
  r.dobj = qy + lterm;
  r.gap = r.dobj - r.pobj;
  free(Kx);
  free(g);
  return r;
}

double orc_kkt_omega(orc_kkt p, double omega) {
  return sqrt(omega * omega * p.pres2 + p.dres2 / (omega * omega) + p.gap * p.gap);
}

/* The three relative tests of Section 2; returns the largest ratio to epsilon's
 * coefficient (so the point passes at tolerance eps iff the result <= eps). */
static double rel_errors(orc_kkt p, double qnorm, double cnorm, double* rp_, double* rd_, double* rg_) {
  double rp = sqrt(p.pres2) / (1.0 + qnorm);
  double rd = sqrt(p.dres2) / (1.0 + cnorm);
  double rg = fabs(p.gap) / (1.0 + fabs(p.dobj) + fabs(p.pobj));
  *rp_ = rp; *rd_ = rd; *rg_ = rg;
  double mx = rp;
  if (rd > mx) mx = rd;
  if (rg > mx) mx = rg;
  return mx;
}

/* ---------- restart conditions (Section 2, restart criteria) ---------- */

/* The restart candidate: the current iterate when its KKT_omega is strictly smaller
 * than the average's, otherwise the average.  Returns 1 for the average. */
int orc_restart_candidate(double kkt_cur, double kkt_avg) {
  if (kkt_cur < kkt_avg) return 0;
  return 1;
}

/* 0: no restart; 1: sufficient decay; 2: necessary decay without local progress;
 * 3: long inner loop.  kkt_prev_c is +inf at the first check of an inner loop. */
int orc_restart_decision(double kkt_c, double kkt_anchor, double kkt_prev_c, int64_t t, int64_t k,
                         double beta_suff, double beta_nec, double beta_art) {
  if (kkt_c <= beta_suff * kkt_anchor) return 1;
  if (kkt_c <= beta_nec * kkt_anchor && kkt_c > kkt_prev_c) return 2;
  if ((double)t >= beta_art * (double)k) return 3;
  return 0;
}

/* ---------- scaling ---------- */

/* Ruiz (ruiz_iters passes, infinity norms) then, if pc, Pock-Chambolle (alpha = 1).
 * Scales v in place (v <- Dr v Dc) and returns Dr (m), Dc (n). */
void orc_scale(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, double* v,
               int32_t ruiz_iters, int32_t pc_pass, double* Dr, double* Dc) {
  double* rs = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  double* cs = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  for (int64_t i = 0; i < m; ++i) Dr[i] = 1.0;
  for (int64_t j = 0; j < n; ++j) Dc[j] = 1.0;
  int32_t passes = ruiz_iters + (pc_pass ? 1 : 0);
  for (int32_t pass = 0; pass < passes; ++pass) {
    int pc = (pass == ruiz_iters);  /* the pass after the Ruiz passes: Pock-Chambolle */
    for (int64_t i = 0; i < m; ++i) rs[i] = 0.0;
    for (int64_t j = 0; j < n; ++j) cs[j] = 0.0;
    for (int64_t i = 0; i < m; ++i)
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        double a = fabs(v[k]);
        if (pc) { rs[i] += a; cs[ci[k]] += a; }
        else {
          if (a > rs[i]) rs[i] = a;
          if (a > cs[ci[k]]) cs[ci[k]] = a;
        }
      }
    for (int64_t i = 0; i < m; ++i) rs[i] = rs[i] > 0.0 ? 1.0 / sqrt(rs[i]) : 1.0;
    for (int64_t j = 0; j < n; ++j) cs[j] = cs[j] > 0.0 ? 1.0 / sqrt(cs[j]) : 1.0;
    for (int64_t i = 0; i < m; ++i)
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) v[k] = (v[k] * rs[i]) * cs[ci[k]];
    for (int64_t i = 0; i < m; ++i) Dr[i] *= rs[i];
    for (int64_t j = 0; j < n; ++j) Dc[j] *= cs[j];
  }
  free(rs);
  free(cs);
}

/* ||K||_2 estimate: v <- K'K v / ||K'K v|| from v0 = 1/sqrt(n); returns ||K v||. */
double orc_power_norm(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                      int32_t iters) {
  if (n == 0 || m == 0) return 0.0;
  double* a = (double*)malloc(sizeof(double) * n);
  double* w = (double*)malloc(sizeof(double) * n);
  double* Ka = (double*)malloc(sizeof(double) * m);
  for (int64_t j = 0; j < n; ++j) a[j] = 1.0 / sqrt((double)n);
  for (int32_t it = 0; it < iters; ++it) {
    orc_spmv(m, rp, ci, v, a, Ka);
    orc_spmv_t(m, n, rp, ci, v, Ka, w);
    double nw = norm2(n, w);
    if (nw == 0.0) break;
    for (int64_t j = 0; j < n; ++j) a[j] = w[j] / nw;
  }
  orc_spmv(m, rp, ci, v, a, Ka);
  double s = norm2(m, Ka);
  free(a); free(w); free(Ka);
  return s;
}

/* ---------- one PDHG step (Section 2, primal and dual updates) ---------- */

/* x <- proj_X(x - (eta/omega)(c - K'y));  y <- proj_Y(y + eta omega (q - K(2x_new - x_old))). */
void orc_pdhg_step(int64_t m, int64_t n, int64_t m1, const int64_t* rp, const int32_t* ci,
                   const double* v, const double* c, const double* q, const double* l,
                   const double* u, double eta, double omega, double* x, double* y) {
  double* g = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* w = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* Kw = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  orc_spmv_t(m, n, rp, ci, v, y, g);
  for (int64_t j = 0; j < n; ++j) {
    double xn = proj_box(x[j] - (eta / omega) * (c[j] - g[j]), l[j], u[j]);
    w[j] = 2.0 * xn - x[j];
    x[j] = xn;
  }
  orc_spmv(m, rp, ci, v, w, Kw);
  for (int64_t i = 0; i < m; ++i) {
    double yn = y[i] + (eta * omega) * (q[i] - Kw[i]);
    if (i >= m1 && yn < 0.0) yn = 0.0;
    y[i] = yn;
  }
  free(g); free(w); free(Kw);
}

/* ---------- the same step on several host threads (CPU baseline timing only) ---------- */

/* K' in CSR by a counting sort of K's entries on their column (stable: each row of K'
 * lists its entries in increasing row of K).  tp[n + 1], tc[nnz] (row of K), tv[nnz]. */
void orc_transpose(int64_t m, int64_t n, const int64_t* rp, const int32_t* ci, const double* v,
                   int64_t* tp, int32_t* tc, double* tv) {
  for (int64_t j = 0; j <= n; ++j) tp[j] = 0;
  for (int64_t k = 0; k < rp[m]; ++k) tp[ci[k] + 1] += 1;
  for (int64_t j = 0; j < n; ++j) tp[j + 1] += tp[j];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t j = 0; j < n; ++j) fill[j] = tp[j];
  for (int64_t i = 0; i < m; ++i)
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      int64_t d = fill[ci[k]]++;
      tc[d] = (int32_t)i;
      tv[d] = v[k];
    }
  free(fill);
}

/* orc_pdhg_step split over `threads` host threads: the primal update by columns (rows
 * of K', each column's terms added in increasing row order, as orc_spmv_t adds them),
 * the dual update by rows.  The arithmetic and its order are orc_pdhg_step's, so the
 * result is bit-identical; only the CPU baseline's timing uses it. */
void orc_pdhg_step_par(int64_t m, int64_t n, int64_t m1, const int64_t* rp, const int32_t* ci,
                       const double* v, const int64_t* tp, const int32_t* tc, const double* tv,
                       const double* c, const double* q, const double* l, const double* u, double eta,
                       double omega, double* x, double* y, int32_t threads) {
  double* w = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  if (threads < 1) threads = 1;
#pragma omp parallel for num_threads(threads) schedule(static)
  for (int64_t j = 0; j < n; ++j) {
    double g = 0.0;
    for (int64_t k = tp[j]; k < tp[j + 1]; ++k) g += tv[k] * y[tc[k]];
    double xn = proj_box(x[j] - (eta / omega) * (c[j] - g), l[j], u[j]);
    w[j] = 2.0 * xn - x[j];
    x[j] = xn;
  }
#pragma omp parallel for num_threads(threads) schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += v[k] * w[ci[k]];
    double yn = y[i] + (eta * omega) * (q[i] - s);
    if (i >= m1 && yn < 0.0) yn = 0.0;
    y[i] = yn;
  }
  free(w);
}

/* ---------- the adaptive step (step_rule = 1) ---------- */

/* One attempt of the adaptive rule from (x, y) with step eta: the candidate goes to
 * (xn, yn); returns eta_max of the candidate (+inf when dy' K dx = 0). */
static double adaptive_attempt(int64_t m, int64_t n, int64_t m1, const int64_t* rp, const int32_t* ci,
                               const double* v, const double* c, const double* q, const double* l,
                               const double* u, double eta, double omega, const double* x, const double* y,
                               double* xn, double* yn) {
  memcpy(xn, x, sizeof(double) * (size_t)n);
  memcpy(yn, y, sizeof(double) * (size_t)m);
  orc_pdhg_step(m, n, m1, rp, ci, v, c, q, l, u, eta, omega, xn, yn);
  double* dx = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  double* Kdx = (double*)malloc(sizeof(double) * (m > 0 ? m : 1));
  double dx2 = 0.0, dy2 = 0.0, inter = 0.0;
  for (int64_t j = 0; j < n; ++j) { dx[j] = xn[j] - x[j]; dx2 += dx[j] * dx[j]; }
  orc_spmv(m, rp, ci, v, dx, Kdx);
  for (int64_t i = 0; i < m; ++i) {
    double dy = yn[i] - y[i];
    dy2 += dy * dy;
    inter += dy * Kdx[i];
  }
  free(dx); free(Kdx);
  if (inter == 0.0) return INFINITY;
  return (omega * dx2 + dy2 / omega) / (2.0 * fabs(inter));
}

/* ---------- the restarted PDHG solve ---------- */

static void unscale(int64_t len, const double* d, const double* a, double* out) {
  for (int64_t i = 0; i < len; ++i) out[i] = d[i] * a[i];
}

/* Returns 0 on success, -1 on bad input.  Outputs (all optional, unscaled, length n or m):
 * x_out/y_out = returned point; x_cur/y_cur = current iterate; x_avg/y_avg = average of
 * the current inner loop (equals the current iterate when t = 0); restart_iters receives
 * up to restart_cap iteration counts at which restarts happened; check_log receives up to
 * log_cap per-check records (the last one is the check that ended the solve). */
int orc_solve(int64_t m, int64_t n, int64_t m1, const int64_t* rp, const int32_t* ci,
              const double* val, const double* c, const double* q, const double* l,
              const double* u, const orc_params* P, const double* x0, const double* y0,
              orc_result* R, double* x_out, double* y_out, double* x_cur, double* y_cur,
              double* x_avg, double* y_avg, int64_t* restart_iters, int64_t restart_cap,
              orc_check* check_log, int64_t log_cap) {
  if (m < 0 || n < 0 || m1 < 0 || m1 > m || P->check_every <= 0) return -1;
  int64_t nnz = rp[m];
  size_t nb = sizeof(double) * (size_t)(n > 0 ? n : 1), mb = sizeof(double) * (size_t)(m > 0 ? m : 1);
  double *vt = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  double *Dr = (double*)malloc(mb), *Dc = (double*)malloc(nb);
  double *ct = (double*)malloc(nb), *lt = (double*)malloc(nb), *ut = (double*)malloc(nb);
  double *qt = (double*)malloc(mb);
  double *x = (double*)malloc(nb), *y = (double*)malloc(mb);
  double *sx = (double*)malloc(nb), *sy = (double*)malloc(mb);
  double *xa = (double*)malloc(nb), *ya = (double*)malloc(mb);   /* averages */
  double *x0a = (double*)malloc(nb), *y0a = (double*)malloc(mb); /* restart anchor z^{n,0} */
  double *xu = (double*)malloc(nb), *yu = (double*)malloc(mb);   /* unscaled copies */
  memcpy(vt, val, sizeof(double) * (size_t)nnz);

  /* scaled problem */
  if (P->scaling) orc_scale(m, n, rp, ci, vt, P->ruiz_iters, 1, Dr, Dc);
  else {
    for (int64_t i = 0; i < m; ++i) Dr[i] = 1.0;
    for (int64_t j = 0; j < n; ++j) Dc[j] = 1.0;
  }
  for (int64_t j = 0; j < n; ++j) { ct[j] = Dc[j] * c[j]; lt[j] = l[j] / Dc[j]; ut[j] = u[j] / Dc[j]; }
  for (int64_t i = 0; i < m; ++i) qt[i] = Dr[i] * q[i];

  double qnorm = norm2(m, q), cnorm = norm2(n, c);  /* unscaled, for termination */
  double eta;
  if (P->eta > 0.0) eta = P->eta;
  else if (P->step_rule == 1) {
    double mx = 0.0;
    for (int64_t e = 0; e < nnz; ++e) if (fabs(vt[e]) > mx) mx = fabs(vt[e]);
    eta = mx > 0.0 ? 1.0 / mx : 1.0;
  } else {
    double s = orc_power_norm(m, n, rp, ci, vt, P->power_iters);
    eta = s > 0.0 ? P->step_scale / s : 1.0;
  }
  double omega;
  if (P->omega0 > 0.0) omega = P->omega0;
  else {
    double cn = norm2(n, ct), qn = norm2(m, qt);
    omega = (cn > 1e-10 && qn > 1e-10) ? cn / qn : 1.0;
  }

  /* initial point: x0 = proj_X(given or 0), y0 = proj_Y(given or 0) */
  for (int64_t j = 0; j < n; ++j) x[j] = proj_box(x0 ? x0[j] / Dc[j] : 0.0, lt[j], ut[j]);
  for (int64_t i = 0; i < m; ++i) {
    double yi = y0 ? y0[i] / Dr[i] : 0.0;
    y[i] = (i >= m1 && yi < 0.0) ? 0.0 : yi;
  }
  memcpy(x0a, x, nb);
  memcpy(y0a, y, mb);
  memset(sx, 0, nb);
  memset(sy, 0, mb);
  orc_kkt pa = orc_kkt_parts(m, n, m1, rp, ci, vt, ct, qt, lt, ut, x, y);
  double kkt_anchor = orc_kkt_omega(pa, omega);
  double kkt_prev_c = INFINITY;
  int64_t k = 0, t = 0, nrestart = 0, accepted = 0, ncheck = 0;
  int rejects = 0;
  double wsum = 0.0;   /* sum of the weights of the iterates in sx, sy */
  double *xn = (double*)malloc(nb), *yn = (double*)malloc(mb);
  int status = 1, which = 0;
  orc_kkt fin = pa;
  double frp = 0, frd = 0, frg = 0;

  for (;;) {
    int final_check = (k >= P->max_iter);
    if (!final_check) {
      if (P->step_rule == 1) {
        double emax = adaptive_attempt(m, n, m1, rp, ci, vt, ct, qt, lt, ut, eta, omega, x, y, xn, yn);
        double sidx = (double)(accepted + 2);   /* s + 1, s = accepted + 1 */
        double e1 = (1.0 - pow(sidx, -0.3)) * emax, e2 = (1.0 + pow(sidx, -0.6)) * eta;
        double enext = e1 < e2 ? e1 : e2;
        if (eta <= emax || rejects >= P->reject_cap) {
          memcpy(x, xn, nb);
          memcpy(y, yn, mb);
          for (int64_t j = 0; j < n; ++j) sx[j] += eta * x[j];
          for (int64_t i = 0; i < m; ++i) sy[i] += eta * y[i];
          wsum += eta;
          ++accepted;
          rejects = 0;
        } else {
          ++rejects;
        }
        eta = enext;
      } else {
        orc_pdhg_step(m, n, m1, rp, ci, vt, ct, qt, lt, ut, eta, omega, x, y);
        for (int64_t j = 0; j < n; ++j) sx[j] += x[j];
        for (int64_t i = 0; i < m; ++i) sy[i] += y[i];
        wsum += 1.0;
        ++accepted;
      }
      ++t;
      ++k;
      final_check = (k >= P->max_iter);
      if (!(k % P->check_every == 0 || final_check)) continue;
    }
    /* ---- check ---- */
    if (wsum > 0.0) {
      for (int64_t j = 0; j < n; ++j) xa[j] = sx[j] / wsum;
      for (int64_t i = 0; i < m; ++i) ya[i] = sy[i] / wsum;
    } else {
      memcpy(xa, x, nb);
      memcpy(ya, y, mb);
    }
    /* termination on the unscaled problem, current and average */
    unscale(n, Dc, x, xu); unscale(m, Dr, y, yu);
    orc_kkt uc = orc_kkt_parts(m, n, m1, rp, ci, val, c, q, l, u, xu, yu);
    unscale(n, Dc, xa, xu); unscale(m, Dr, ya, yu);
    orc_kkt ua = orc_kkt_parts(m, n, m1, rp, ci, val, c, q, l, u, xu, yu);
    double rpc, rdc, rgc, rpa, rda, rga;
    double ec = rel_errors(uc, qnorm, cnorm, &rpc, &rdc, &rgc);
    double ea = rel_errors(ua, qnorm, cnorm, &rpa, &rda, &rga);
    int pass_c = ec <= P->tol, pass_a = ea <= P->tol;
    /* KKT_omega of both points on the scaled problem (restart test and log) */
    orc_kkt sc = orc_kkt_parts(m, n, m1, rp, ci, vt, ct, qt, lt, ut, x, y);
    orc_kkt sa = orc_kkt_parts(m, n, m1, rp, ci, vt, ct, qt, lt, ut, xa, ya);
    double kc = orc_kkt_omega(sc, omega), ka = orc_kkt_omega(sa, omega);
    int cand_avg = orc_restart_candidate(kc, ka);
    orc_check* rec = (check_log && ncheck < log_cap) ? &check_log[ncheck] : NULL;
    ++ncheck;
    if (rec) {
      int cur_better = ec < ea;
      rec->k = k;
      rec->t = t;
      rec->restart = 0;
      rec->candidate = cand_avg;
      rec->omega = omega;
      rec->kkt_cur = kc;
      rec->kkt_avg = ka;
      rec->kkt_anchor = kkt_anchor;
      rec->rel_primal = cur_better ? rpc : rpa;
      rec->rel_dual = cur_better ? rdc : rda;
      rec->rel_gap = cur_better ? rgc : rga;
    }
    if (pass_c || pass_a || final_check) {
      if (pass_c || pass_a) status = 0;
      if (pass_c && !pass_a) which = 0;
      else if (pass_a && !pass_c) which = 1;
      else which = (ec < ea) ? 0 : 1;
      fin = which ? ua : uc;
      frp = which ? rpa : rpc; frd = which ? rda : rdc; frg = which ? rga : rgc;
      break;
    }
    /* restart conditions for the candidate */
    double kkt_c = cand_avg ? ka : kc;
    orc_kkt pc = cand_avg ? sa : sc;
    int why = orc_restart_decision(kkt_c, kkt_anchor, kkt_prev_c, t, k, P->beta_suff, P->beta_nec,
                                   P->beta_art);
    if (rec) rec->restart = why;
    if (why) {
      const double* xc = cand_avg ? xa : x;
      const double* yc = cand_avg ? ya : y;
      double dx = dist2(n, xc, x0a), dy = dist2(m, yc, y0a);
      if (dx > 1e-10 && dy > 1e-10)
        omega = exp(P->omega_theta * log(dy / dx) + (1.0 - P->omega_theta) * log(omega));
      if (cand_avg) { memcpy(x, xa, nb); memcpy(y, ya, mb); }
      memcpy(x0a, x, nb);
      memcpy(y0a, y, mb);
      memset(sx, 0, nb);
      memset(sy, 0, mb);
      t = 0;
      wsum = 0.0;
      kkt_anchor = orc_kkt_omega(pc, omega);
      kkt_prev_c = INFINITY;
      if (nrestart < restart_cap && restart_iters) restart_iters[nrestart] = k;
      ++nrestart;
    } else {
      kkt_prev_c = kkt_c;
    }
  }

  if (wsum > 0.0) {
    for (int64_t j = 0; j < n; ++j) xa[j] = sx[j] / wsum;
    for (int64_t i = 0; i < m; ++i) ya[i] = sy[i] / wsum;
  } else {
    memcpy(xa, x, nb);
    memcpy(ya, y, mb);
  }
  if (x_cur) unscale(n, Dc, x, x_cur);
  if (y_cur) unscale(m, Dr, y, y_cur);
  if (x_avg) unscale(n, Dc, xa, x_avg);
  if (y_avg) unscale(m, Dr, ya, y_avg);
  if (x_out) unscale(n, Dc, which ? xa : x, x_out);
  if (y_out) unscale(m, Dr, which ? ya : y, y_out);
  if (R) {
    orc_kkt sfin = orc_kkt_parts(m, n, m1, rp, ci, vt, ct, qt, lt, ut, which ? xa : x, which ? ya : y);
    R->status = status;
    R->which = which;
    R->iters = k;
    R->restarts = nrestart;
    R->primal_obj = fin.pobj;
    R->dual_obj = fin.dobj;
    R->rel_primal = frp;
    R->rel_dual = frd;
    R->rel_gap = frg;
    R->kkt_omega = orc_kkt_omega(sfin, omega);
    R->omega = omega;
    R->eta = eta;
    R->accepted = accepted;
    R->checks = ncheck;
  }
  free(vt); free(Dr); free(Dc); free(ct); free(lt); free(ut); free(qt);
  free(x); free(y); free(sx); free(sy); free(xa); free(ya); free(x0a); free(y0a);
  free(xu); free(yu); free(xn); free(yn);
  return 0;
}
