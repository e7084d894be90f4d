/*
 * oracle.c -- plain single-threaded FP64 reference of the multi-cell stiff
 * chemistry solve.  TEST INFRASTRUCTURE ONLY (see oracle.h): the product path
 * never calls this code.
 *
 * Everything here is written for a reader checking it against the paper and
 * the integrator specification by eye: straight loops in species and reaction
 * order, a dense Jacobian, a dense LU with partial pivoting.  Build with
 * -O2 -ffp-contract=off (no fused multiply-add contraction, no fast-math).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- constants */

/* Boltzmann constant (J/K); number density of air in molecules/cm^3 is
 * n_air = P / (k_B T) * 1e-6. */
static const double K_BOLTZMANN = 1.380649e-23;

/* Integrator constants of the project's BDF specification (CVODE-style). */
#define NEWTON_MAXITER 3      /* corrector iterations per attempt */
#define CRDOWN 0.3            /* convergence-rate memory decay */
#define RDIV 2.0              /* divergence: del_m > RDIV * del_{m-1} */
#define NLSCOEF 0.1           /* corrector tolerance = NLSCOEF * (q+1) */
#define DGMAX 0.3             /* re-form M when |c/c_M - 1| > DGMAX */
#define MSBP 20               /* re-form M at least every MSBP steps */
#define THRESH 1.5            /* change h only for a factor >= THRESH */
#define BIAS_DOWN 2.0          /* error-estimate biases for orders q-1, q, q+1 */
#define BIAS_SAME 2.0
#define BIAS_UP 3.0
#define MXNEF 7               /* error-test failures per step before giving up */
#define MXNCF 10              /* corrector failures per step before giving up */
#define ETA_CF 0.25           /* step factor after a corrector failure */
#define ETA_MXF 0.2           /* cap on the step factor after 2+ error failures */
#define ETA_CST_SAFETY 0.9    /* constraint failure: h shrinks to 0.9 of the zero crossing */
#define ETA_CST_MIN 0.1       /* ... but by no more than a factor 10 */
#define STRETCH 1e-3          /* final step may stretch h by this fraction */
#define GRID_IMIN (-26)       /* step-factor grid g_i = 2^(i/8), i in [IMIN, IMAX] */
#define GRID_IMAX 26

/* gamma_m = sum_{i=1..m} 1/i, and 1/gamma_m, m = 0..QMAX+1 (gamma_0 unused) */
static double gamma_of(int m) {
  double g = 0.0;
  for (int i = 1; i <= m; ++i) g += 1.0 / (double)i;
  return g;
}

/* ------------------------------------------------------------ a1: k~_j(T,P) */

static double arrhenius(double A, double Ea_over_R, double B, double T) {
  return A * exp(-Ea_over_R / T) * pow(T / 300.0, B);
}

/*
 * The rate constant of a pressure-dependent reaction (the rate is a function of
 * the state, T and P: Background section), from the first Arrhenius term ka
 * and the air number density nm = [M]:
 *   Troe fall-off: the Lindemann-Hinshelwood interpolation between the
 *     low-pressure rate k0 [M] (k0 = ka) and the high-pressure limit kinf
 *     (second term), times the broadening factor F with
 *     log10 F = log10 Fc / (1 + (log10(k0 [M] / kinf) / N)^2);
 *   pressure sum: ka + kb [M];
 *   fall-off sum: ka plus a Lindemann term between kc [M] and kb.
 */
static double pressure_dependent(const orc_mech *m, int j, double ka, double T, double nm) {
  const double *e = m->ext + (size_t)j * 8;
  const double kb = arrhenius(e[0], e[1], e[2], T);
  switch (m->kind[j]) {
    case ORC_TROE: {
      const double low = ka * nm;                 /* k0 [M] */
      const double lindemann = low * kb / (low + kb);
      const double c = log10(low / kb) / e[7];
      const double logF = log10(e[6]) / (1.0 + c * c);
      return lindemann * pow(10.0, logF);
    }
    case ORC_PRESSURE_SUM:
      return ka + kb * nm;
    case ORC_FALLOFF_SUM: {
      const double low = arrhenius(e[3], e[4], e[5], T) * nm;   /* kc [M] */
      return ka + low * kb / (low + kb);
    }
    default:
      return ka;
  }
}

void orc_rate_constants(const orc_mech *m, double T, double P, const double *jphot,
                        const double *theta, double *kt) {
  const double n_air = P / (K_BOLTZMANN * T) * 1e-6;
  int iphot = 0;
  for (int j = 0; j < m->n_reactions; ++j) {
    double k;
    if (m->kind[j] == ORC_PHOTOLYSIS) {
      k = jphot ? jphot[iphot] : m->J[j];
      iphot++;
    } else {
      /* Arrhenius k = A exp(-Ea/T) (T/300)^B; n-th order rates act on mixing
       * ratios, so multiply by n_air once per reactant beyond the first. */
      k = arrhenius(m->A[j], m->Ea[j], m->B[j], T);
      if (m->kind[j] != ORC_THERMAL) k = pressure_dependent(m, j, k, T, n_air);
      for (int r = 1; r < m->n_reac[j]; ++r) k *= n_air;
    }
    if (theta) k *= exp(theta[j]);
    kt[j] = k;
  }
}

/* --------------------------------------------------------------- a2: f(y) */

/* rate of reaction j: r_j = k~_j * prod over reactant slots of y */
static double rate(const orc_mech *m, const double *kt, const double *y, int j) {
  double r = kt[j];
  for (int s = 0; s < m->n_reac[j]; ++s) r *= y[m->reac[j * ORC_MAX_REAC + s]];
  return r;
}

void orc_deriv(const orc_mech *m, const double *kt, const double *y, double *f) {
  const int S = m->n_species;
  for (int i = 0; i < S; ++i) f[i] = 0.0;
  /* each reaction adds its contribution: -r_j per reactant slot, +yield*r_j per product */
  for (int j = 0; j < m->n_reactions; ++j) {
    const double r = rate(m, kt, y, j);
    for (int s = 0; s < m->n_reac[j]; ++s) f[m->reac[j * ORC_MAX_REAC + s]] -= r;
    for (int p = 0; p < m->n_prod[j]; ++p)
      f[m->prod[j * ORC_MAX_PROD + p]] += m->yld[j * ORC_MAX_PROD + p] * r;
  }
}

/* --------------------------------------------------------- a3: Jacobian */

void orc_jacobian(const orc_mech *m, const double *kt, const double *y, double *J) {
  const int S = m->n_species;
  for (int i = 0; i < S * S; ++i) J[i] = 0.0;
  for (int j = 0; j < m->n_reactions; ++j) {
    const int nr = m->n_reac[j];
    const int32_t *rc = m->reac + j * ORC_MAX_REAC;
    for (int s = 0; s < nr; ++s) {
      /* partial of r_j through reactant slot s: k~ times the other slots' y */
      double p = kt[j];
      for (int s2 = 0; s2 < nr; ++s2)
        if (s2 != s) p *= y[rc[s2]];
      const int l = rc[s];
      for (int s2 = 0; s2 < nr; ++s2) J[rc[s2] * S + l] -= p;
      for (int q = 0; q < m->n_prod[j]; ++q)
        J[m->prod[j * ORC_MAX_PROD + q] * S + l] += m->yld[j * ORC_MAX_PROD + q] * p;
    }
  }
}

/* ------------------------------------------- dense LU, partial pivoting */

int orc_lu_factor(int n, double *A, int32_t *piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); p = i; }
    piv[k] = p;
    if (best == 0.0) return k + 1;
    if (p != k)
      for (int c = 0; c < n; ++c) { double t = A[k * n + c]; A[k * n + c] = A[p * n + c]; A[p * n + c] = t; }
    for (int i = k + 1; i < n; ++i) {
      const double l = A[i * n + k] / A[k * n + k];
      A[i * n + k] = l;
      for (int c = k + 1; c < n; ++c) A[i * n + c] -= l * A[k * n + c];
    }
  }
  return 0;
}

void orc_lu_solve(int n, const double *LU, const int32_t *piv, double *b) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < i; ++c) b[i] -= LU[i * n + c] * b[c];
  for (int i = n - 1; i >= 0; --i) {
    for (int c = i + 1; c < n; ++c) b[i] -= LU[i * n + c] * b[c];
    b[i] /= LU[i * n + i];
  }
}

/* ------------------------------------------------------ history rescale */

/*
 * The differences D_1..D_q represent the interpolating polynomial through the
 * last q+1 solution values at spacing h.  For a new spacing eta*h the new
 * differences are D'_i = sum_m (U R(eta))_{im} D_m, with
 *   R(eta)_{jm} = prod_{l=0}^{m-1} (l - j*eta) / m!,   j, m = 1..q,
 *   U = R(1)  (so U R(1) = I and eta = 1 changes nothing),
 * Shampine & Reichelt, "The MATLAB ODE Suite" (1997), quasi-constant step BDF.
 */
static void rescale_matrix(int q, double eta, double T[ORC_QMAX][ORC_QMAX]) {
  double R[ORC_QMAX][ORC_QMAX], U[ORC_QMAX][ORC_QMAX];
  for (int j = 1; j <= q; ++j)
    for (int mm = 1; mm <= q; ++mm) {
      double r = 1.0, u = 1.0;
      for (int l = 0; l < mm; ++l) {
        r *= ((double)l - (double)j * eta) / (double)(l + 1);
        u *= ((double)l - (double)j) / (double)(l + 1);
      }
      R[j - 1][mm - 1] = r;
      U[j - 1][mm - 1] = u;
    }
  for (int i = 0; i < q; ++i)
    for (int mm = 0; mm < q; ++mm) {
      double s = 0.0;
      for (int j = 0; j < q; ++j) s += U[i][j] * R[j][mm];
      T[i][mm] = s;
    }
}

void orc_rescale(int S, int q, double eta, double *D) {
  double T[ORC_QMAX][ORC_QMAX];
  rescale_matrix(q, eta, T);
  double *tmp = (double *)malloc(sizeof(double) * (size_t)q * S);
  for (int i = 0; i < q; ++i)
    for (int s = 0; s < S; ++s) {
      double v = 0.0;
      for (int mm = 0; mm < q; ++mm) v += T[i][mm] * D[(size_t)(mm + 1) * S + s];
      tmp[(size_t)i * S + s] = v;
    }
  memcpy(D + S, tmp, sizeof(double) * (size_t)q * S);
  free(tmp);
}

/* ----------------------------------------------------- step-factor grid */

/* Step factors are drawn from the grid g_i = 2^(i/8).  For an error estimate
 * err of a method of order p the chosen factor is the largest g_i with
 * err <= 1 / (bias * g_i^(p+1)); if none qualifies, the smallest g_i.  The
 * integrator works with squared norms, so the test is made on err2 = err^2
 * against the squared threshold 1 / (bias^2 * 2^(i(p+1)/4)). */
double orc_grid_eta(double err2, int p, double bias) {
  for (int i = GRID_IMAX; i >= GRID_IMIN; --i) {
    const double thr2 = 1.0 / (bias * bias * exp2((double)i * (double)(p + 1) / 4.0));
    if (err2 <= thr2) return exp2((double)i / 8.0);
  }
  return exp2((double)GRID_IMIN / 8.0);
}

/* The same grid in the plain form: err against 1 / (bias * 2^(i(p+1)/8)). */
static double grid_eta_plain(double err, int p, double bias) {
  for (int i = GRID_IMAX; i >= GRID_IMIN; --i) {
    const double thr = 1.0 / (bias * exp2((double)i * (double)(p + 1) / 8.0));
    if (err <= thr) return exp2((double)i / 8.0);
  }
  return exp2((double)GRID_IMIN / 8.0);
}

/* ---------------------------------------------------------- helpers */

static double wrms(int S, const double *v, const double *w) {
  double s = 0.0;
  for (int i = 0; i < S; ++i) { const double t = v[i] * w[i]; s += t * t; }
  return sqrt(s / (double)S);
}

/* The squared norm (1/S) sum (v_i w_i)^2, formed as the sum times 1/S.  The
 * corrector, constraint and error tests compare squared norms with squared
 * bounds (the same tests as on the norms, without a square root). */
static double wrms2(int S, const double *v, const double *w) {
  double s = 0.0;
  for (int i = 0; i < S; ++i) { const double t = v[i] * w[i]; s += t * t; }
  return s * (1.0 / (double)S);
}

/* 1/n^2 */
static double isq(int n) { return 1.0 / (double)(n * n); }

static void set_weights(int S, const double *y, double rtol, double atol, double *w) {
  for (int i = 0; i < S; ++i) w[i] = 1.0 / (rtol * fabs(y[i]) + atol);
}

static void tape_push(orc_tape *tp, int S, int kind, int q, double val, const double *y) {
  if (!tp) return;
  if (tp->n >= tp->cap) { tp->overflow = 1; return; }
  tp->kind[tp->n] = kind;
  tp->q[tp->n] = q;
  tp->val[tp->n] = val;
  if (y) memcpy(tp->y + (size_t)tp->n * S, y, sizeof(double) * S);
  tp->n++;
}

/* ------------------------------------------------- a4-a7: the integrator */

int orc_integrate(const orc_mech *m, const double *kt, double *y0, double dt, const orc_opts *o,
                  orc_stats *st, orc_tape *tape) {
  const int S = m->n_species;
  const int fixed = o->fixed_h > 0.0;
  int qmax = fixed ? o->fixed_order : o->max_order;
  if (qmax < 1) qmax = 1;
  if (qmax > ORC_QMAX) qmax = ORC_QMAX;
  memset(st, 0, sizeof(*st));
  if (tape) { tape->n = 0; tape->overflow = 0; }

  for (int i = 0; i < S; ++i)
    if (!isfinite(y0[i])) { st->status = ORC_BAD_INPUT; return st->status; }
  for (int j = 0; j < m->n_reactions; ++j)
    if (!isfinite(kt[j])) { st->status = ORC_BAD_INPUT; return st->status; }

  const int NROW = ORC_QMAX + 3;
  double *D = (double *)calloc((size_t)NROW * S, sizeof(double));
  double *ypred = (double *)malloc(sizeof(double) * S);
  double *y = (double *)malloc(sizeof(double) * S);
  double *d = (double *)malloc(sizeof(double) * S);
  double *psi = (double *)malloc(sizeof(double) * S);
  double *w = (double *)malloc(sizeof(double) * S);
  double *f = (double *)malloc(sizeof(double) * S);
  double *dy = (double *)malloc(sizeof(double) * S);
  double *M = (double *)malloc(sizeof(double) * S * S);
  int32_t *piv = (int32_t *)malloc(sizeof(int32_t) * S);

  double gam[ORC_QMAX + 2], igam[ORC_QMAX + 2];
  for (int k = 1; k <= ORC_QMAX + 1; ++k) { gam[k] = gamma_of(k); igam[k] = 1.0 / gam[k]; }

  double t = 0.0, h;
  int q;
  set_weights(S, y0, o->rtol, o->atol, w);
  if (fixed) {
    h = o->fixed_h;
    q = qmax;
    if (o->init_D) {
      memcpy(D, o->init_D, sizeof(double) * (size_t)(q + 1) * S);
    } else {
      memcpy(D, y0, sizeof(double) * S);
      orc_deriv(m, kt, y0, f);
      st->f_evals++;
      for (int i = 0; i < S; ++i) D[S + i] = h * f[i];
    }
  } else {
    /* initial step for order 1 (Hairer, Norsett & Wanner, Solving ODEs I, II.4),
     * in the weighted RMS norm, capped at dt */
    q = 1;
    double *f0 = (double *)malloc(sizeof(double) * S);
    orc_deriv(m, kt, y0, f0);
    st->f_evals++;
    const double d0 = wrms(S, y0, w), d1 = wrms(S, f0, w);
    double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 * dt : 0.01 * d0 / d1;
    if (h0 > dt) h0 = dt;
    for (int i = 0; i < S; ++i) ypred[i] = y0[i] + h0 * f0[i];
    orc_deriv(m, kt, ypred, f);
    st->f_evals++;
    for (int i = 0; i < S; ++i) dy[i] = f[i] - f0[i];
    const double d2 = wrms(S, dy, w) / h0;
    const double dm = d1 > d2 ? d1 : d2;
    double h1 = (dm <= 1e-15) ? fmax(1e-6 * dt, h0 * 1e-3) : sqrt(0.01 / dm);
    h = fmin(fmin(100.0 * h0, h1), dt);
    memcpy(D, y0, sizeof(double) * S);
    for (int i = 0; i < S; ++i) D[S + i] = h * f0[i];
    free(f0);
  }
  tape_push(tape, S, 0 /*INIT*/, q, h, y0);

  const long n_fixed = fixed ? lround(dt / h) : 0;
  int *projected = (int *)malloc(sizeof(int) * S);   /* species projected onto y = 0 in this attempt */
  int n_projected = 0;
  double *iters = (double *)malloc(sizeof(double) * (size_t)(NEWTON_MAXITER + 64) * S);  /* iterates of the attempt */
  int n_iters = 0;
  int n_eq = 0, have_M = 0, force_M = 0, n_since_M = 0, nef = 0, ncf = 0, last = 0;
  double cM = 0.0, icM = 0.0, rho2 = 1.0;    /* rho2: squared convergence-rate estimate */
  double rho = 1.0;                          /* the estimate itself (plain form) */
  const int plain = o->plain_form;
  int status = ORC_OK;

  for (;;) {
    /* -- step length: stop at dt exactly (a7) */
    if (fixed) {
      if (st->steps >= n_fixed) break;
      last = (st->steps + 1 == n_fixed);
    } else {
      if (st->steps >= o->max_steps) { status = ORC_MAX_STEPS; break; }
      if (dt - t <= h * (1.0 + STRETCH)) {
        const double hn = dt - t;
        if (hn != h) {
          orc_rescale(S, q, hn / h, D);
          tape_push(tape, S, 1 /*RESCALE*/, q, hn / h, NULL);
          h = hn;
          n_eq = 0;
        }
        last = 1;
      } else {
        last = 0;
      }
      if (!last && t + h == t) { status = ORC_H_TOO_SMALL; break; }   /* no progress in t */
    }

    /* -- predictor y_pred = sum_{m<=q} D_m, history term psi (a6) */
    const double c = h * igam[q];
    for (int i = 0; i < S; ++i) {
      double s = D[i];
      for (int k = 1; k <= q; ++k) s += D[(size_t)k * S + i];
      ypred[i] = s;
    }
    for (int i = 0; i < S; ++i) {
      double s = 0.0;
      for (int k = 1; k <= q; ++k) s += gam[k] * D[(size_t)k * S + i];
      psi[i] = s * igam[q];
    }

    /* -- iteration matrix M = I - c J(y_pred), re-formed only when stale (a4, a5) */
    int fresh = 0;
    const double c_ratio = plain ? (have_M ? c / cM : 0.0) : c * icM;
    if (!have_M || force_M || fabs(c_ratio - 1.0) > DGMAX || n_since_M >= MSBP) {
      orc_jacobian(m, kt, ypred, M);
      for (int i = 0; i < S * S; ++i) M[i] = -c * M[i];
      for (int i = 0; i < S; ++i) M[i * S + i] += 1.0;
      if (orc_lu_factor(S, M, piv) != 0) { status = ORC_CONV_FAIL; break; }
      have_M = 1;
      cM = c;
      icM = 1.0 / c;
      n_since_M = 0;
      rho2 = 1.0;
      rho = 1.0;
      fresh = 1;
      st->jac_evals++;
      tape_push(tape, S, 4 /*REFACTOR*/, 0, c, ypred);
    }
    force_M = 0;
    const double scale = (c == cM) ? 1.0 : (plain ? 2.0 / (1.0 + c / cM) : 2.0 / (1.0 + c * icM));

    /* -- modified Newton corrector: M dy = c f(y) - psi - d (a6) */
    const double tol = o->newton_tol > 0.0 ? o->newton_tol : NLSCOEF * (double)(q + 1);
    const double tol2 = tol * tol;
    const int maxit = o->newton_maxiter > 0 ? o->newton_maxiter : NEWTON_MAXITER;
    for (int i = 0; i < S; ++i) { d[i] = 0.0; y[i] = ypred[i]; }
    double del2 = 0.0, del2_prev = 0.0, del = 0.0, del_prev = 0.0;
    int conv = 0;
    n_iters = 0;
    for (int it = 0; it < maxit; ++it) {
      if (it < NEWTON_MAXITER + 64) memcpy(iters + (size_t)it * S, y, sizeof(double) * S);
      n_iters = it + 1;
      orc_deriv(m, kt, y, f);
      st->f_evals++;
      for (int i = 0; i < S; ++i) dy[i] = c * f[i] - psi[i] - d[i];
      orc_lu_solve(S, M, piv, dy);
      st->solves++;
      if (scale != 1.0)
        for (int i = 0; i < S; ++i) dy[i] *= scale;
      if (plain) del = wrms(S, dy, w);
      else del2 = wrms2(S, dy, w);
      for (int i = 0; i < S; ++i) { d[i] += dy[i]; y[i] = ypred[i] + d[i]; }
      st->newton_iters++;
      if (plain) {
        if (it > 0) rho = fmax(CRDOWN * rho, del / del_prev);
        if (del * fmin(1.0, rho) <= tol) { conv = 1; break; }
        if (it > 0 && del > RDIV * del_prev) break;
        del_prev = del;
        continue;
      }
      if (it > 0) rho2 = fmax(CRDOWN * CRDOWN * rho2, del2 / del2_prev);
      if (del2 * fmin(1.0, rho2) <= tol2) { conv = 1; break; }
      if (it > 0 && del2 > RDIV * RDIV * del2_prev) break;
      del2_prev = del2;
    }
    if (!conv) {
      st->conv_fails++;
      ncf++;
      if (ncf >= MXNCF || fixed) { status = ORC_CONV_FAIL; break; }
      if (!fresh) {
        force_M = 1;                 /* retry the same step with a fresh Jacobian */
      } else {
        orc_rescale(S, q, ETA_CF, D);
        tape_push(tape, S, 1, q, ETA_CF, NULL);
        h *= ETA_CF;
        n_eq = 0;
      }
      continue;
    }

    /* -- inequality constraint y >= 0 (CVODE-style): a violation no larger
     *    than the corrector tolerance is projected onto y_i = 0; a larger one
     *    rejects the step and shrinks h towards the first zero crossing of the
     *    linear path from y_n to y. */
    if (!fixed) {
      double vs = 0.0, eta_c = 1.0;
      int nv = 0;
      for (int i = 0; i < S; ++i)
        if (y[i] < 0.0) {
          const double v = y[i] * w[i];
          vs += v * v;
          nv++;
          const double r = (D[i] > 0.0) ? D[i] / (D[i] - y[i]) : 0.0;
          if (r < eta_c) eta_c = r;
        }
      n_projected = 0;
      if (nv > 0) {
        if (plain ? sqrt(vs / (double)S) <= tol : vs * (1.0 / (double)S) <= tol2) {
          for (int i = 0; i < S; ++i)
            if (y[i] < 0.0) { d[i] -= y[i]; y[i] = 0.0; projected[n_projected++] = i; }
        } else {
          st->rejects++;
          nef++;
          if (nef >= MXNEF) { status = ORC_ERR_FAIL; break; }
          double eta = ETA_CST_SAFETY * eta_c;
          if (eta < ETA_CST_MIN) eta = ETA_CST_MIN;
          orc_rescale(S, q, eta, D);
          tape_push(tape, S, 1, q, eta, NULL);
          h *= eta;
          n_eq = 0;
          continue;
        }
      }
    }

    /* -- local error test (a7): err = ||d|| / (q+1), tested squared */
    const double err2 = plain ? 0.0 : wrms2(S, d, w) * isq(q + 1);
    const double err = plain ? wrms(S, d, w) / (double)(q + 1) : 0.0;
    if (!fixed && !(plain ? err <= 1.0 : err2 <= 1.0)) {
      st->rejects++;
      nef++;
      if (nef >= MXNEF) { status = ORC_ERR_FAIL; break; }
      double eta = plain ? grid_eta_plain(err, q, BIAS_SAME) : orc_grid_eta(err2, q, BIAS_SAME);
      if (nef >= 2 && eta > ETA_MXF) eta = ETA_MXF;
      if (nef >= 3 && q > 1) q -= 1;
      orc_rescale(S, q, eta, D);
      tape_push(tape, S, 1, q, eta, NULL);
      h *= eta;
      n_eq = 0;
      continue;
    }

    /* -- accept: update the backward differences */
    t = last ? dt : t + h;
    st->steps++;
    st->order_sum += q;
    n_since_M++;
    nef = 0;
    ncf = 0;
    for (int i = 0; i < S; ++i) {
      D[(size_t)(q + 2) * S + i] = d[i] - D[(size_t)(q + 1) * S + i];
      D[(size_t)(q + 1) * S + i] = d[i];
    }
    for (int k = q; k >= 0; --k)
      for (int i = 0; i < S; ++i) D[(size_t)k * S + i] += D[(size_t)(k + 1) * S + i];
    for (int k = 0; k < n_iters && k < NEWTON_MAXITER + 64; ++k) tape_push(tape, S, 5 /*ITER*/, k, 0.0, iters + (size_t)k * S);
    for (int k = 0; k < n_projected; ++k) tape_push(tape, S, 3 /*PROJECT*/, projected[k], 0.0, NULL);
    n_projected = 0;
    tape_push(tape, S, 2 /*STEP*/, q, c, D);
    if (fixed && o->y_hist) memcpy(o->y_hist + (size_t)(st->steps - 1) * S, D, sizeof(double) * S);
    if (last) break;
    n_eq++;

    /* -- step size and order for the next step */
    if (!fixed) {
      double eta = plain ? grid_eta_plain(err, q, BIAS_SAME) : orc_grid_eta(err2, q, BIAS_SAME);
      int qn = q;
      if (n_eq >= q + 1) {
        if (q > 1) {
          const double em = plain ? grid_eta_plain(wrms(S, D + (size_t)q * S, w) / (double)q, q - 1, BIAS_DOWN)
                                  : orc_grid_eta(wrms2(S, D + (size_t)q * S, w) * isq(q), q - 1, BIAS_DOWN);
          if (em > eta) { eta = em; qn = q - 1; }
        }
        if (q < qmax) {
          const double ep = plain ? grid_eta_plain(wrms(S, D + (size_t)(q + 2) * S, w) / (double)(q + 2), q + 1, BIAS_UP)
                                  : orc_grid_eta(wrms2(S, D + (size_t)(q + 2) * S, w) * isq(q + 2), q + 1, BIAS_UP);
          if (ep > eta) { eta = ep; qn = q + 1; }
        }
      }
      if (eta >= THRESH) {
        q = qn;
        orc_rescale(S, q, eta, D);
        tape_push(tape, S, 1, q, eta, NULL);
        h *= eta;
        n_eq = 0;
      }
    }
    set_weights(S, D, o->rtol, o->atol, w);
  }

  if (status == ORC_OK)
    for (int i = 0; i < S; ++i)
      if (!isfinite(D[i])) status = ORC_NONFINITE;
  if (status == ORC_OK) memcpy(y0, D, sizeof(double) * S);
  st->status = status;
  st->final_order = q;
  st->final_h = h;

  free(D); free(ypred); free(y); free(d); free(psi); free(w); free(f); free(dy); free(M); free(piv);
  free(projected);
  free(iters);
  return status;
}

/* ------------------------------------------------- multi-cell driver */

int orc_solve_cells(const orc_mech *m, int64_t n_cells, const double *T, const double *P,
                    const double *jphot, const double *theta, double *y, double dt,
                    const orc_opts *o, orc_stats *st) {
  const int S = m->n_species, R = m->n_reactions;
  int n_phot = 0;
  for (int j = 0; j < R; ++j) n_phot += (m->kind[j] == ORC_PHOTOLYSIS);
  double *kt = (double *)malloc(sizeof(double) * R);
  double *yc = (double *)malloc(sizeof(double) * S);
  double *jc = (double *)malloc(sizeof(double) * (n_phot > 0 ? n_phot : 1));
  int n_failed = 0;
  for (int64_t c = 0; c < n_cells; ++c) {
    orc_stats *sc = st + c;
    if (!(T[c] > 0.0) || !(P[c] > 0.0) || !isfinite(T[c]) || !isfinite(P[c])) {
      memset(sc, 0, sizeof(*sc));
      sc->status = ORC_BAD_INPUT;
      n_failed++;
      continue;
    }
    if (jphot)
      for (int k = 0; k < n_phot; ++k) jc[k] = jphot[(size_t)k * n_cells + c];
    orc_rate_constants(m, T[c], P[c], jphot ? jc : NULL, theta, kt);
    for (int i = 0; i < S; ++i) yc[i] = y[(size_t)i * n_cells + c];
    if (orc_integrate(m, kt, yc, dt, o, sc, NULL) != ORC_OK) n_failed++;
    for (int i = 0; i < S; ++i) y[(size_t)i * n_cells + c] = yc[i];
  }
  free(kt); free(yc); free(jc);
  return n_failed;
}
