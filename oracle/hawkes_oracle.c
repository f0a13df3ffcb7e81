/*
 * Plain FP64 CPU oracle for the spatiotemporal Hawkes log-likelihood and its
 * gradient.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only tests/, __graft_entry__.smoke()
 * and bench.py (its cpu_baseline leg and its `--impl reference` arm) may load
 * or call this library. The CUDA library shares no code, header, constant or
 * helper with this file, and neither side includes or links the other.
 *
 * Source: Holbrook, Loeffler, Flaxman, Suchard, "Scalable Bayesian inference
 * for self-excitatory stochastic processes applied to big American gunfire
 * data", Section 2.1 (model, compensator, Eq. 1 log-likelihood, Eq. 2
 * self-excitation probabilities). Spatial dimension d = 2.
 *
 *   lambda(x,t) = mu(x,t) + sum_{t_n' < t} g(x - x_n', t - t_n')
 *   mu(x,t)     = mu0 / (tau_x^2 tau_t) * sum_{n'=1..N} phi2((x - x_n')/tau_x) phi1((t - t_n')/tau_t)
 *   g(dx, dt)   = theta * omega / h^2 * exp(-omega dt) * phi2(dx / h)
 *   Lambda_n    = mu0 (Phi((t_N - t_n)/tau_t) - Phi(-t_n/tau_t)) - theta (exp(-omega (t_N - t_n)) - 1)
 *   ell         = sum_n [ log lambda(x_n, t_n) - Lambda_n ]                  (Eq. 1)
 *   pi_n        = xi_n / lambda_n, xi_n = lambda_n - mu(x_n, t_n)           (Eq. 2)
 *
 * phi1 / phi2 are the standard normal densities on R and R^2 (the 2-D one is
 * the product of two 1-D ones), Phi the standard normal CDF.
 *
 * Readings where the paper is ambiguous (each is a choice, stated once):
 *  - Trigger prefactor. Section 2.1 prints theta / (omega h^d) in front of the
 *    trigger sum, but its closed-form compensator term theta (1 - e^{-omega s})
 *    is the time integral of theta * omega * e^{-omega u}, not of
 *    (theta / omega) e^{-omega u}. The oracle uses theta * omega / h^2 so that
 *    Lambda is the integral of lambda. ORACLE_LITERAL_PREFACTOR switches to
 *    the printed theta / (omega h^2); it exists so that a test can show that
 *    the printed form breaks that integral identity, and nothing else uses it.
 *  - Self term. The background sum in Eq. 1 runs over all n' = 1..N, so n' = n
 *    contributes phi2(0) phi1(0). That is the default. ORACLE_EXCLUDE_SELF
 *    drops it (the "all other events" reading).
 *  - Ties. The trigger indicator is strict, t_n' < t_n, comparing the stored
 *    time values. Events with equal times never trigger each other.
 *  - Integration window. Lambda integrates t over [0, t_N] with t_N the last
 *    (largest) event time, and x over all of R^2.
 *
 * Arithmetic: every sum (over n' inside a row, over rows, over threads) is a
 * Neumaier-compensated FP64 sum; the per-thread partials are combined in thread
 * order, so results do not depend on scheduling. Threads own contiguous row
 * blocks (the multi-core row partition of the paper's CPU likelihood
 * algorithm, Section 2.3.1), written with plain pthreads.
 *
 * Gradient: the paper has no gradient. d ell / d p = sum_n (d lambda_n / d p) /
 * lambda_n - d Lambda / d p, with every pair term differentiated directly.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_EXCLUDE_SELF 1
#define ORACLE_LITERAL_PREFACTOR 2

typedef struct {
  double mu0, tau_x, tau_t, theta, omega, h; /* Theta, in the order of Section 2.1 */
} oracle_params;

static const double PI = 3.14159265358979323846;

/* ---- Neumaier-compensated accumulator ---------------------------------- */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum *a, double v) {
  double t = a->s + v;
  if (!isfinite(t)) {  /* an infinite term (log 0 = -inf): the sum is that infinity, uncompensated */
    a->s = t;
    return;
  }
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static double nsum_get(const nsum *a) { return a->s + a->c; }

/* ---- the normal densities and CDF --------------------------------------- */
static double phi1(double u) { return exp(-0.5 * u * u) / sqrt(2.0 * PI); }
static double phi2(double u, double v) { return exp(-0.5 * (u * u + v * v)) / (2.0 * PI); }
static double Phi(double u) { return 0.5 * erfc(-u / sqrt(2.0)); }

static double trigger_prefactor(const oracle_params *p, int flags) {
  if (flags & ORACLE_LITERAL_PREFACTOR) return p->theta / (p->omega * p->h * p->h);
  return p->theta * p->omega / (p->h * p->h);
}

/* One term of the background sum, mu0/(tau_x^2 tau_t) phi2(dx/tau_x) phi1(dt/tau_t). */
static double background_term(const oracle_params *p, double dx, double dy, double dt) {
  return p->mu0 / (p->tau_x * p->tau_x * p->tau_t) * phi2(dx / p->tau_x, dy / p->tau_x) * phi1(dt / p->tau_t);
}
/* One term of the trigger sum without the indicator: prefactor * e^{-omega dt} phi2(dx/h). */
static double trigger_term(const oracle_params *p, int flags, double dx, double dy, double dt) {
  return trigger_prefactor(p, flags) * exp(-p->omega * dt) * phi2(dx / p->h, dy / p->h);
}

/*
 * Per-row quantities for event n (Section 2.1, Eq. 1 inner sum; Eq. 2):
 *   out[0] = mu_n      (background rate at event n, sum over all n')
 *   out[1] = xi_n      (self-excitation part, sum over t_n' < t_n)
 *   out[2..7] = d lambda_n / d (mu0, tau_x, tau_t, theta, omega, h)
 */
static void row_terms(int64_t n, const double *x, const double *y, const double *t,
                      const oracle_params *p, int flags, int64_t row, int want_grad,
                      double out[8]) {
  nsum mu = {0, 0}, xi = {0, 0}, g[6];
  memset(g, 0, sizeof g);
  const double xr = x[row], yr = y[row], tr = t[row];
  for (int64_t j = 0; j < n; ++j) {
    const double dx = xr - x[j], dy = yr - y[j], dt = tr - t[j];
    const double r2 = dx * dx + dy * dy;
    if (!((flags & ORACLE_EXCLUDE_SELF) && j == row)) {
      const double b = background_term(p, dx, dy, dt);
      nsum_add(&mu, b);
      if (want_grad) {
        /* d/d mu0, d/d tau_x, d/d tau_t of the background term */
        nsum_add(&g[0], b / p->mu0);
        nsum_add(&g[1], b * (-2.0 / p->tau_x + r2 / (p->tau_x * p->tau_x * p->tau_x)));
        nsum_add(&g[2], b * (-1.0 / p->tau_t + dt * dt / (p->tau_t * p->tau_t * p->tau_t)));
      }
    }
    if (t[j] < tr) { /* strict indicator on stored times */
      const double s = trigger_term(p, flags, dx, dy, dt);
      nsum_add(&xi, s);
      if (want_grad) {
        double ds_dtheta, ds_domega;
        if (flags & ORACLE_LITERAL_PREFACTOR) {
          ds_dtheta = exp(-p->omega * dt) * phi2(dx / p->h, dy / p->h) / (p->omega * p->h * p->h);
          ds_domega = s * (-1.0 / p->omega - dt);
        } else {
          ds_dtheta = p->omega / (p->h * p->h) * exp(-p->omega * dt) * phi2(dx / p->h, dy / p->h);
          ds_domega = s * (1.0 / p->omega - dt);
        }
        nsum_add(&g[3], ds_dtheta);
        nsum_add(&g[4], ds_domega);
        nsum_add(&g[5], s * (-2.0 / p->h + r2 / (p->h * p->h * p->h)));
      }
    }
  }
  out[0] = nsum_get(&mu);
  out[1] = nsum_get(&xi);
  for (int k = 0; k < 6; ++k) out[2 + k] = want_grad ? nsum_get(&g[k]) : 0.0;
}

/* Lambda_n and its derivatives (Section 2.1 closed form); t_N = last event time. */
static void compensator_terms(double tn, double tN, const oracle_params *p, double out[7]) {
  const double a = (tN - tn) / p->tau_t, b = -tn / p->tau_t;
  const double D = tN - tn, e = exp(-p->omega * D);
  out[0] = p->mu0 * (Phi(a) - Phi(b)) - p->theta * (e - 1.0);
  out[1] = Phi(a) - Phi(b);                                         /* d/d mu0   */
  out[2] = 0.0;                                                     /* d/d tau_x */
  out[3] = p->mu0 / p->tau_t * (-a * phi1(a) + b * phi1(b));        /* d/d tau_t */
  out[4] = 1.0 - e;                                                 /* d/d theta */
  out[5] = p->theta * D * e;                                        /* d/d omega */
  out[6] = 0.0;                                                     /* d/d h     */
}

/* ---- threading ------------------------------------------------------------ */
typedef struct {
  int64_t n;
  const double *x, *y, *t;
  const oracle_params *p;
  int flags, want_grad;
  /* rows [lo, hi) of either the identity list or rows[] */
  const int64_t *rows;
  int64_t lo, hi;
  /* per-row outputs (optional) */
  double *row_out;   /* 8 + 7 doubles per listed row */
  /* block totals */
  nsum ell, grad[6];
} job;

static void *run_job(void *arg) {
  job *J = (job *)arg;
  const double tN = J->t[J->n - 1];
  memset(&J->ell, 0, sizeof J->ell);
  memset(J->grad, 0, sizeof J->grad);
  for (int64_t i = J->lo; i < J->hi; ++i) {
    const int64_t row = J->rows ? J->rows[i] : i;
    double rt[8], ct[7];
    row_terms(J->n, J->x, J->y, J->t, J->p, J->flags, row, J->want_grad, rt);
    compensator_terms(J->t[row], tN, J->p, ct);
    const double lam = rt[0] + rt[1];
    nsum_add(&J->ell, log(lam) - ct[0]);
    if (J->want_grad)
      for (int k = 0; k < 6; ++k) nsum_add(&J->grad[k], rt[2 + k] / lam - ct[1 + k]);
    if (J->row_out) {
      double *o = J->row_out + 15 * i;
      memcpy(o, rt, 8 * sizeof(double));
      memcpy(o + 8, ct, 7 * sizeof(double));
    }
  }
  return NULL;
}

static int check_inputs(int64_t n, const double *t, const oracle_params *p) {
  if (n < 1 || !t || !p) return -1;
  for (int64_t i = 1; i < n; ++i)
    if (!(t[i] >= t[i - 1])) return -2;
  return 0;
}

static int run_threads(job *proto, int64_t count, int nthreads, double *ell_out, double *grad_out) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > count) nthreads = (int)(count > 0 ? count : 1);
  job *jobs = (job *)calloc((size_t)nthreads, sizeof(job));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return -3; }
  for (int k = 0; k < nthreads; ++k) {
    jobs[k] = *proto;
    jobs[k].lo = count * k / nthreads;
    jobs[k].hi = count * (k + 1) / nthreads;
  }
  for (int k = 1; k < nthreads; ++k) pthread_create(&th[k], NULL, run_job, &jobs[k]);
  run_job(&jobs[0]);
  for (int k = 1; k < nthreads; ++k) pthread_join(th[k], NULL);
  nsum ell = {0, 0}, g[6];
  memset(g, 0, sizeof g);
  for (int k = 0; k < nthreads; ++k) {
    nsum_add(&ell, nsum_get(&jobs[k].ell));
    for (int q = 0; q < 6; ++q) nsum_add(&g[q], nsum_get(&jobs[k].grad[q]));
  }
  if (ell_out) *ell_out = nsum_get(&ell);
  if (grad_out) for (int q = 0; q < 6; ++q) grad_out[q] = nsum_get(&g[q]);
  free(jobs);
  free(th);
  return 0;
}

/*
 * Full log-likelihood (Eq. 1) and, if grad_out is not NULL, its gradient with
 * respect to (mu0, tau_x, tau_t, theta, omega, h). Events must be sorted by
 * time. Returns 0, or -1 (bad arguments), -2 (times not sorted), -3 (no memory).
 */
int oracle_loglik(int64_t n, const double *x, const double *y, const double *t,
                  const oracle_params *p, int flags, int nthreads,
                  double *ell_out, double *grad_out) {
  int rc = check_inputs(n, t, p);
  if (rc) return rc;
  job proto;
  memset(&proto, 0, sizeof proto);
  proto.n = n; proto.x = x; proto.y = y; proto.t = t; proto.p = p;
  proto.flags = flags; proto.want_grad = grad_out != NULL;
  return run_threads(&proto, n, nthreads, ell_out, grad_out);
}

/*
 * Per-row quantities for the listed rows (any order, repeats allowed). For
 * listed row i, out[15 i + k] holds
 *   k = 0: mu_n, 1: xi_n, 2..7: d lambda_n / d Theta,
 *   k = 8: Lambda_n, 9..14: d Lambda_n / d Theta.
 * The sums over the listed rows of (log lambda_n - Lambda_n) and of the
 * gradient terms go to ell_out / grad_out when those are not NULL.
 */
int oracle_rows(int64_t n, const double *x, const double *y, const double *t,
                const oracle_params *p, int flags, int want_grad,
                int64_t m, const int64_t *rows, int nthreads, double *out,
                double *ell_out, double *grad_out) {
  int rc = check_inputs(n, t, p);
  if (rc) return rc;
  if (m < 0 || (m > 0 && (!rows || !out))) return -1;
  for (int64_t i = 0; i < m; ++i)
    if (rows[i] < 0 || rows[i] >= n) return -1;
  job proto;
  memset(&proto, 0, sizeof proto);
  proto.n = n; proto.x = x; proto.y = y; proto.t = t; proto.p = p;
  proto.flags = flags; proto.want_grad = want_grad;
  proto.rows = rows; proto.row_out = out;
  if (m == 0) {
    if (ell_out) *ell_out = 0.0;
    if (grad_out) memset(grad_out, 0, 6 * sizeof(double));
    return 0;
  }
  return run_threads(&proto, m, nthreads, ell_out, want_grad ? grad_out : NULL);
}

/*
 * The intensity lambda(q) at arbitrary query points q = (qx, qy, qt), given
 * the events (Section 2.1): the background sum over all events plus the
 * trigger sum over events strictly earlier than qt. Used by the tests to
 * integrate lambda numerically and to evaluate it between events.
 */
int oracle_intensity(int64_t n, const double *x, const double *y, const double *t,
                     const oracle_params *p, int flags, int64_t m,
                     const double *qx, const double *qy, const double *qt, double *out) {
  if (n < 1 || m < 0 || !p) return -1;
  for (int64_t q = 0; q < m; ++q) {
    nsum mu = {0, 0}, xi = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
      const double dx = qx[q] - x[j], dy = qy[q] - y[j], dt = qt[q] - t[j];
      nsum_add(&mu, background_term(p, dx, dy, dt));
      if (t[j] < qt[q]) nsum_add(&xi, trigger_term(p, flags, dx, dy, dt));
    }
    out[q] = nsum_get(&mu) + nsum_get(&xi);
  }
  return 0;
}

/* Lambda(t_N) = sum_n Lambda_n and its gradient (Section 2.1 closed form). */
int oracle_compensator(int64_t n, const double *t, const oracle_params *p,
                       double *Lambda_out, double *grad_out) {
  int rc = check_inputs(n, t, p);
  if (rc) return rc;
  nsum L = {0, 0}, g[6];
  memset(g, 0, sizeof g);
  for (int64_t i = 0; i < n; ++i) {
    double ct[7];
    compensator_terms(t[i], t[n - 1], p, ct);
    nsum_add(&L, ct[0]);
    for (int k = 0; k < 6; ++k) nsum_add(&g[k], ct[1 + k]);
  }
  if (Lambda_out) *Lambda_out = nsum_get(&L);
  if (grad_out) for (int k = 0; k < 6; ++k) grad_out[k] = nsum_get(&g[k]);
  return 0;
}

/* ==========================================================================
 * Mixture of triggering functions (the extension the paper's Discussion
 * proposes: several triggering functions that combine a very short time frame,
 * multi-shot events, with a longer one, retaliation over days to months).
 * Reading: each component is the paper's triggering function with its own
 * (theta_m, omega_m, h_m), taken with the same prefactor reading as above,
 *
 *   g(dx, dt) = sum_{m=1..M} theta_m * omega_m / h_m^2 * exp(-omega_m dt) * phi2(dx / h_m),
 *
 * so the branching ratio is sum_m theta_m, M = 1 is the model of Section 2.1,
 * and the compensator's trigger part is sum_m theta_m (1 - e^{-omega_m (t_N - t_n)}).
 * The background, the self term, ties and the window are as above. Gradient
 * order: (mu0, tau_x, tau_t, theta_1, omega_1, h_1, ..., theta_M, omega_M, h_M).
 * ========================================================================== */
#define ORACLE_MIX_MAX 2

typedef struct {
  double mu0, tau_x, tau_t;
  double theta[ORACLE_MIX_MAX], omega[ORACLE_MIX_MAX], h[ORACLE_MIX_MAX];
} oracle_mix_params;

/* The background-only parameter view (theta unused) of a mixture. */
static oracle_params mix_background(const oracle_mix_params *p) {
  oracle_params b;
  memset(&b, 0, sizeof b);
  b.mu0 = p->mu0; b.tau_x = p->tau_x; b.tau_t = p->tau_t;
  return b;
}

/* Per-row quantities of the mixture for event `row`: out[0] = mu_n, out[1] = xi_n (all
 * components), out[2 .. 2 + 3 + 3M) = d lambda_n / d Theta in the gradient order above. */
static void mix_row_terms(int64_t n, const double *x, const double *y, const double *t,
                          const oracle_mix_params *p, int M, int flags, int64_t row, int want_grad,
                          double *out) {
  const oracle_params bp = mix_background(p);
  const int np = 3 + 3 * M;
  nsum mu = {0, 0}, xi = {0, 0}, g[3 + 3 * ORACLE_MIX_MAX];
  memset(g, 0, sizeof g);
  const double xr = x[row], yr = y[row], tr = t[row];
  for (int64_t j = 0; j < n; ++j) {
    const double dx = xr - x[j], dy = yr - y[j], dt = tr - t[j];
    const double r2 = dx * dx + dy * dy;
    if (!((flags & ORACLE_EXCLUDE_SELF) && j == row)) {
      const double b = background_term(&bp, dx, dy, dt);
      nsum_add(&mu, b);
      if (want_grad) {
        nsum_add(&g[0], b / p->mu0);
        nsum_add(&g[1], b * (-2.0 / p->tau_x + r2 / (p->tau_x * p->tau_x * p->tau_x)));
        nsum_add(&g[2], b * (-1.0 / p->tau_t + dt * dt / (p->tau_t * p->tau_t * p->tau_t)));
      }
    }
    if (t[j] < tr) { /* strict indicator on stored times */
      for (int m = 0; m < M; ++m) {
        const double hm = p->h[m], om = p->omega[m];
        const double kern = om / (hm * hm) * exp(-om * dt) * phi2(dx / hm, dy / hm); /* s_m / theta_m */
        const double s = p->theta[m] * kern;
        nsum_add(&xi, s);
        if (want_grad) {
          nsum_add(&g[3 + 3 * m], kern);
          nsum_add(&g[4 + 3 * m], s * (1.0 / om - dt));
          nsum_add(&g[5 + 3 * m], s * (-2.0 / hm + r2 / (hm * hm * hm)));
        }
      }
    }
  }
  out[0] = nsum_get(&mu);
  out[1] = nsum_get(&xi);
  for (int k = 0; k < np; ++k) out[2 + k] = want_grad ? nsum_get(&g[k]) : 0.0;
}

/* Lambda_n of the mixture and its derivatives in the gradient order (out[0] = Lambda_n). */
static void mix_compensator_terms(double tn, double tN, const oracle_mix_params *p, int M, double *out) {
  const double a = (tN - tn) / p->tau_t, b = -tn / p->tau_t, D = tN - tn;
  out[0] = p->mu0 * (Phi(a) - Phi(b));
  out[1] = Phi(a) - Phi(b);
  out[2] = 0.0;
  out[3] = p->mu0 / p->tau_t * (-a * phi1(a) + b * phi1(b));
  for (int m = 0; m < M; ++m) {
    const double e = exp(-p->omega[m] * D);
    out[0] += p->theta[m] * (1.0 - e);
    out[4 + 3 * m] = 1.0 - e;
    out[5 + 3 * m] = p->theta[m] * D * e;
    out[6 + 3 * m] = 0.0;
  }
}

typedef struct {
  int64_t n;
  const double *x, *y, *t;
  const oracle_mix_params *p;
  int M, flags, want_grad;
  int64_t lo, hi;
  nsum ell, grad[3 + 3 * ORACLE_MIX_MAX];
} mix_job;

static void *run_mix_job(void *arg) {
  mix_job *J = (mix_job *)arg;
  const double tN = J->t[J->n - 1];
  const int np = 3 + 3 * J->M;
  memset(&J->ell, 0, sizeof J->ell);
  memset(J->grad, 0, sizeof J->grad);
  for (int64_t row = J->lo; row < J->hi; ++row) {
    double rt[2 + 3 + 3 * ORACLE_MIX_MAX], ct[1 + 3 + 3 * ORACLE_MIX_MAX];
    mix_row_terms(J->n, J->x, J->y, J->t, J->p, J->M, J->flags, row, J->want_grad, rt);
    mix_compensator_terms(J->t[row], tN, J->p, J->M, ct);
    const double lam = rt[0] + rt[1];
    nsum_add(&J->ell, log(lam) - ct[0]);
    if (J->want_grad)
      for (int k = 0; k < np; ++k) nsum_add(&J->grad[k], rt[2 + k] / lam - ct[1 + k]);
  }
  return NULL;
}

/*
 * Log-likelihood (Eq. 1 with the mixture trigger) and, if grad_out is not NULL, its gradient
 * (3 + 3M entries in the order above). 1 <= M <= ORACLE_MIX_MAX. Returns 0, -1 (bad
 * arguments), -2 (times not sorted), -3 (no memory).
 */
int oracle_loglik_mix(int64_t n, const double *x, const double *y, const double *t,
                      const oracle_mix_params *p, int M, int flags, int nthreads,
                      double *ell_out, double *grad_out) {
  if (M < 1 || M > ORACLE_MIX_MAX || !p || !t || n < 1) return -1;
  for (int64_t i = 1; i < n; ++i)
    if (!(t[i] >= t[i - 1])) return -2;
  const int np = 3 + 3 * M;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > n) nthreads = (int)n;
  mix_job *jobs = (mix_job *)calloc((size_t)nthreads, sizeof(mix_job));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  if (!jobs || !th) { free(jobs); free(th); return -3; }
  for (int k = 0; k < nthreads; ++k) {
    jobs[k].n = n; jobs[k].x = x; jobs[k].y = y; jobs[k].t = t; jobs[k].p = p;
    jobs[k].M = M; jobs[k].flags = flags; jobs[k].want_grad = grad_out != NULL;
    jobs[k].lo = n * k / nthreads;
    jobs[k].hi = n * (k + 1) / nthreads;
  }
  for (int k = 1; k < nthreads; ++k) pthread_create(&th[k], NULL, run_mix_job, &jobs[k]);
  run_mix_job(&jobs[0]);
  for (int k = 1; k < nthreads; ++k) pthread_join(th[k], NULL);
  nsum ell = {0, 0}, g[3 + 3 * ORACLE_MIX_MAX];
  memset(g, 0, sizeof g);
  for (int k = 0; k < nthreads; ++k) {
    nsum_add(&ell, nsum_get(&jobs[k].ell));
    for (int q = 0; q < np; ++q) nsum_add(&g[q], nsum_get(&jobs[k].grad[q]));
  }
  if (ell_out) *ell_out = nsum_get(&ell);
  if (grad_out) for (int q = 0; q < np; ++q) grad_out[q] = nsum_get(&g[q]);
  free(jobs);
  free(th);
  return 0;
}

/* The mixture intensity lambda(q) at query points (background over all events, every
 * component's trigger over events strictly earlier than qt), for the integral pins. */
int oracle_intensity_mix(int64_t n, const double *x, const double *y, const double *t,
                         const oracle_mix_params *p, int M, int64_t m,
                         const double *qx, const double *qy, const double *qt, double *out) {
  if (n < 1 || m < 0 || !p || M < 1 || M > ORACLE_MIX_MAX) return -1;
  const oracle_params bp = mix_background(p);
  for (int64_t q = 0; q < m; ++q) {
    nsum s = {0, 0};
    for (int64_t j = 0; j < n; ++j) {
      const double dx = qx[q] - x[j], dy = qy[q] - y[j], dt = qt[q] - t[j];
      nsum_add(&s, background_term(&bp, dx, dy, dt));
      if (t[j] < qt[q])
        for (int c = 0; c < M; ++c)
          nsum_add(&s, p->theta[c] * p->omega[c] / (p->h[c] * p->h[c]) * exp(-p->omega[c] * dt) *
                           phi2(dx / p->h[c], dy / p->h[c]));
    }
    out[q] = nsum_get(&s);
  }
  return 0;
}
