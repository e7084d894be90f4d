/*
 * adjoint.c -- tangent and discrete adjoint of the frozen-step BDF map, for
 * the oracle.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The map.  An integration leaves a tape of the operations that changed the
 * backward-difference history D (orc_tape): INIT (D_0 = y, D_1 = h0 f(y), the
 * rest 0), RESCALE (order q, factor eta: D_{1..q} <- T(eta) D_{1..q}) and
 * accepted STEP (order q, c = h / gamma_q).  The replay map y0 -> y_final
 * re-applies these operations with the step sizes and orders frozen, solving
 * each step equation
 *     d = c f(y_pred + d) - psi,   y_pred = sum_{m<=q} D_m,
 *     psi = (1/gamma_q) sum_{m=1..q} gamma_m D_m
 * exactly (Newton with a fresh Jacobian to rounding level) and without the
 * y >= 0 projection, then updating D_{q+2} = d - D_{q+1}, D_{q+1} = d,
 * D_m += D_{m+1} (m = q..0).  A tape may hold several consecutive solves:
 * every INIT restarts the history from the current D_0.
 *
 * Sensitivities are taken with respect to y0 and to theta, the per-reaction
 * log multipliers of the rate constants (k~_j -> k~_j e^{theta_j}), at the
 * theta already folded into kt; d r_j / d theta_j = r_j.
 *
 * The adjoint of one STEP (lambda' the adjoint of D after it): the step
 * writes D'_m = sum_{i=m..q} D_i + d (m <= q), D'_{q+1} = d,
 * D'_{q+2} = d - D_{q+1}; so
 *     lambda_d = lambda'_{q+2} + lambda'_{q+1} + sum_{m<=q} lambda'_m,
 *     lambda_i = sum_{m<=i} lambda'_m (i <= q), lambda_{q+1} = -lambda'_{q+2},
 *     lambda_{q+2} = 0, higher rows unchanged;
 * and through the implicit step equation (I - cJ) dd = c J dy_pred
 * + c F_theta dtheta - dpsi, with mu = (I - cJ)^{-T} lambda_d:
 *     lambda_i += c J^T mu (i <= q),  lambda_i -= (gamma_i/gamma_q) mu (1 <= i <= q),
 *     dL/dtheta_j += c r_j(y) (nu_j . mu).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define NROW (ORC_QMAX + 3)

static double gamma_m(int m) {
  double g = 0.0;
  for (int i = 1; i <= m; ++i) g += 1.0 / (double)i;
  return g;
}

/* r_j(y) for all reactions */
static void rates(const orc_mech *m, const double *kt, const double *y, double *r) {
  for (int j = 0; j < m->n_reactions; ++j) {
    double v = kt[j];
    for (int s = 0; s < m->n_reac[j]; ++s) v *= y[m->reac[j * ORC_MAX_REAC + s]];
    r[j] = v;
  }
}

/* (nu_j . v) for all reactions: net stoichiometry times a species vector */
static void nu_dot(const orc_mech *m, const double *v, double *out) {
  for (int j = 0; j < m->n_reactions; ++j) {
    double s = 0.0;
    for (int k = 0; k < m->n_reac[j]; ++k) s -= v[m->reac[j * ORC_MAX_REAC + k]];
    for (int p = 0; p < m->n_prod[j]; ++p) s += m->yld[j * ORC_MAX_PROD + p] * v[m->prod[j * ORC_MAX_PROD + p]];
    out[j] = s;
  }
}

/* F_theta dtheta = sum_j nu_j r_j dtheta_j */
static void ftheta_times(const orc_mech *m, const double *r, const double *dth, double *out) {
  const int S = m->n_species;
  for (int i = 0; i < S; ++i) out[i] = 0.0;
  for (int j = 0; j < m->n_reactions; ++j) {
    const double v = r[j] * dth[j];
    for (int k = 0; k < m->n_reac[j]; ++k) out[m->reac[j * ORC_MAX_REAC + k]] -= v;
    for (int p = 0; p < m->n_prod[j]; ++p) out[m->prod[j * ORC_MAX_PROD + p]] += m->yld[j * ORC_MAX_PROD + p] * v;
  }
}

static void matvec(int S, const double *A, const double *x, double *y, int transpose) {
  for (int i = 0; i < S; ++i) {
    double s = 0.0;
    for (int k = 0; k < S; ++k) s += (transpose ? A[k * S + i] : A[i * S + k]) * x[k];
    y[i] = s;
  }
}

/* x = (I - c J)^{-1} b, or its transpose; J dense [S*S] */
static int solve_shifted(int S, double c, const double *J, const double *b, double *x, int transpose) {
  double *M = (double *)malloc(sizeof(double) * S * S);
  int32_t *piv = (int32_t *)malloc(sizeof(int32_t) * S);
  for (int i = 0; i < S; ++i)
    for (int k = 0; k < S; ++k) {
      const double jv = transpose ? J[k * S + i] : J[i * S + k];
      M[i * S + k] = (i == k ? 1.0 : 0.0) - c * jv;
    }
  int rc = orc_lu_factor(S, M, piv);
  if (rc == 0) {
    memcpy(x, b, sizeof(double) * S);
    orc_lu_solve(S, M, piv, x);
  }
  free(M);
  free(piv);
  return rc;
}

static double maxabs(int S, const double *v) {
  double m = 0.0;
  for (int i = 0; i < S; ++i)
    if (fabs(v[i]) > m) m = fabs(v[i]);
  return m;
}

/* exact solution of one step equation; d in/out (start value), y out */
static int step_solve(const orc_mech *m, const double *kt, int S, double c, const double *ypred, const double *psi,
                      double *d, double *y, double newton_tol, int maxit) {
  double *f = (double *)malloc(sizeof(double) * S);
  double *F = (double *)malloc(sizeof(double) * S);
  double *dx = (double *)malloc(sizeof(double) * S);
  double *J = (double *)malloc(sizeof(double) * S * S);
  int rc = 1;
  for (int it = 0; it < maxit; ++it) {
    for (int i = 0; i < S; ++i) y[i] = ypred[i] + d[i];
    orc_deriv(m, kt, y, f);
    for (int i = 0; i < S; ++i) F[i] = c * f[i] - psi[i] - d[i];
    orc_jacobian(m, kt, y, J);
    if (solve_shifted(S, c, J, F, dx, 0)) break;
    for (int i = 0; i < S; ++i) d[i] += dx[i];
    if (maxabs(S, dx) <= newton_tol * (maxabs(S, y) + 1e-300)) { rc = 0; break; }
  }
  for (int i = 0; i < S; ++i) y[i] = ypred[i] + d[i];
  free(f); free(F); free(dx); free(J);
  return rc;
}

static void predict(int S, int q, const double *D, double *ypred, double *psi) {
  const double igq = 1.0 / gamma_m(q);
  for (int i = 0; i < S; ++i) {
    double s = D[i], p = 0.0;
    for (int k = 1; k <= q; ++k) {
      s += D[(size_t)k * S + i];
      p += gamma_m(k) * D[(size_t)k * S + i];
    }
    ypred[i] = s;
    psi[i] = p * igq;
  }
}

static void history_update(int S, int q, double *D, const double *d) {
  for (int i = 0; i < S; ++i) {
    D[(size_t)(q + 2) * S + i] = d[i] - D[(size_t)(q + 1) * S + i];
    D[(size_t)(q + 1) * S + i] = d[i];
  }
  for (int k = q; k >= 0; --k)
    for (int i = 0; i < S; ++i) D[(size_t)k * S + i] += D[(size_t)(k + 1) * S + i];
}

/* the rescale matrix T(eta) (q x q, rows/cols 1..q) as orc_rescale applies it */
static void rescale_T(int S, int q, double eta, double T[ORC_QMAX][ORC_QMAX]) {
  /* apply orc_rescale to unit vectors: column mm of T = rescale(e_mm) */
  double *D = (double *)calloc((size_t)(q + 1), sizeof(double));
  (void)S;
  for (int mm = 0; mm < q; ++mm) {
    memset(D, 0, sizeof(double) * (q + 1));
    D[mm + 1] = 1.0;
    orc_rescale(1, q, eta, D);
    for (int i = 0; i < q; ++i) T[i][mm] = D[i + 1];
  }
  free(D);
}

int orc_replay(const orc_mech *m, const double *kt, const double *y0, const orc_tape *tp, double newton_tol,
               int maxit, double *y_out, double *y_steps) {
  const int S = m->n_species;
  double *D = (double *)calloc((size_t)NROW * S, sizeof(double));
  double *ypred = (double *)malloc(sizeof(double) * S), *psi = (double *)malloc(sizeof(double) * S);
  double *d = (double *)malloc(sizeof(double) * S), *y = (double *)malloc(sizeof(double) * S);
  double *f = (double *)malloc(sizeof(double) * S);
  int rc = 0;
  memcpy(D, y0, sizeof(double) * S);
  for (int e = 0; e < tp->n; ++e) {
    const int kind = tp->kind[e], q = tp->q[e];
    const double val = tp->val[e];
    if (kind == 0) {               /* INIT: restart the history from the current y */
      for (int r = 1; r < NROW; ++r)
        for (int i = 0; i < S; ++i) D[(size_t)r * S + i] = 0.0;
      orc_deriv(m, kt, D, f);
      for (int i = 0; i < S; ++i) D[S + i] = val * f[i];
    } else if (kind == 1) {
      orc_rescale(S, q, val, D);
    } else {
      predict(S, q, D, ypred, psi);
      for (int i = 0; i < S; ++i) d[i] = 0.0;
      if (step_solve(m, kt, S, val, ypred, psi, d, y, newton_tol, maxit)) rc = 1;
      history_update(S, q, D, d);
      if (y_steps) memcpy(y_steps + (size_t)e * S, D, sizeof(double) * S);
    }
  }
  memcpy(y_out, D, sizeof(double) * S);
  free(D); free(ypred); free(psi); free(d); free(y); free(f);
  return rc;
}

int orc_tangent(const orc_mech *m, const double *kt, const double *y0, const orc_tape *tp, const double *dy0,
                const double *dtheta, double *dy_out) {
  const int S = m->n_species, R = m->n_reactions;
  double *D = (double *)calloc((size_t)NROW * S, sizeof(double));
  double *dD = (double *)calloc((size_t)NROW * S, sizeof(double));
  double *ypred = (double *)malloc(sizeof(double) * S), *psi = (double *)malloc(sizeof(double) * S);
  double *dyp = (double *)malloc(sizeof(double) * S), *dpsi = (double *)malloc(sizeof(double) * S);
  double *d = (double *)malloc(sizeof(double) * S), *y = (double *)malloc(sizeof(double) * S);
  double *dd = (double *)malloc(sizeof(double) * S), *b = (double *)malloc(sizeof(double) * S);
  double *f = (double *)malloc(sizeof(double) * S), *tmp = (double *)malloc(sizeof(double) * S);
  double *J = (double *)malloc(sizeof(double) * S * S), *r = (double *)malloc(sizeof(double) * (R > 0 ? R : 1));
  int rc = 0;
  memcpy(D, y0, sizeof(double) * S);
  memcpy(dD, dy0, sizeof(double) * S);
  for (int e = 0; e < tp->n; ++e) {
    const int kind = tp->kind[e], q = tp->q[e];
    const double val = tp->val[e];
    if (kind == 0) {
      for (int row = 1; row < NROW; ++row)
        for (int i = 0; i < S; ++i) D[(size_t)row * S + i] = dD[(size_t)row * S + i] = 0.0;
      orc_deriv(m, kt, D, f);
      orc_jacobian(m, kt, D, J);
      rates(m, kt, D, r);
      matvec(S, J, dD, tmp, 0);
      ftheta_times(m, r, dtheta, b);
      for (int i = 0; i < S; ++i) {
        D[S + i] = val * f[i];
        dD[S + i] = val * (tmp[i] + b[i]);
      }
    } else if (kind == 1) {
      orc_rescale(S, q, val, D);
      orc_rescale(S, q, val, dD);
    } else {
      const double c = val;
      predict(S, q, D, ypred, psi);
      predict(S, q, dD, dyp, dpsi);
      for (int i = 0; i < S; ++i) d[i] = 0.0;
      if (step_solve(m, kt, S, c, ypred, psi, d, y, 1e-15, 30)) rc = 1;
      orc_jacobian(m, kt, y, J);
      rates(m, kt, y, r);
      /* (I - cJ) dd = c J dy_pred + c F_theta dtheta - dpsi */
      matvec(S, J, dyp, tmp, 0);
      ftheta_times(m, r, dtheta, b);
      for (int i = 0; i < S; ++i) b[i] = c * tmp[i] + c * b[i] - dpsi[i];
      if (solve_shifted(S, c, J, b, dd, 0)) rc = 1;
      history_update(S, q, D, d);
      history_update(S, q, dD, dd);
    }
  }
  memcpy(dy_out, dD, sizeof(double) * S);
  free(D); free(dD); free(ypred); free(psi); free(dyp); free(dpsi); free(d); free(y); free(dd); free(b);
  free(f); free(tmp); free(J); free(r);
  return rc;
}

int orc_adjoint(const orc_mech *m, const double *kt, const double *y0, const orc_tape *tp, const double *lam_final,
                double *lam_y0, double *g_theta) {
  const int S = m->n_species, R = m->n_reactions, n = tp->n;
  double *ys = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * S);
  double *yinit = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * S);   /* y at each INIT */
  double *yend = (double *)malloc(sizeof(double) * S);
  double *L = (double *)calloc((size_t)NROW * S, sizeof(double));
  double *nl = (double *)calloc((size_t)NROW * S, sizeof(double));
  double *lamd = (double *)malloc(sizeof(double) * S), *mu = (double *)malloc(sizeof(double) * S);
  double *tmp = (double *)malloc(sizeof(double) * S), *J = (double *)malloc(sizeof(double) * S * S);
  double *r = (double *)malloc(sizeof(double) * (R > 0 ? R : 1)), *nm = (double *)malloc(sizeof(double) * (R > 0 ? R : 1));
  int rc = 0;

  /* forward replay, keeping y after every STEP and at every INIT */
  {
    double *D = (double *)calloc((size_t)NROW * S, sizeof(double));
    double *ypred = (double *)malloc(sizeof(double) * S), *psi = (double *)malloc(sizeof(double) * S);
    double *d = (double *)malloc(sizeof(double) * S), *y = (double *)malloc(sizeof(double) * S);
    memcpy(D, y0, sizeof(double) * S);
    for (int e = 0; e < n; ++e) {
      const int kind = tp->kind[e], q = tp->q[e];
      const double val = tp->val[e];
      if (kind == 0) {
        memcpy(yinit + (size_t)e * S, D, sizeof(double) * S);
        for (int row = 1; row < NROW; ++row)
          for (int i = 0; i < S; ++i) D[(size_t)row * S + i] = 0.0;
        orc_deriv(m, kt, D, tmp);
        for (int i = 0; i < S; ++i) D[S + i] = val * tmp[i];
      } else if (kind == 1) {
        orc_rescale(S, q, val, D);
      } else {
        predict(S, q, D, ypred, psi);
        for (int i = 0; i < S; ++i) d[i] = 0.0;
        if (step_solve(m, kt, S, val, ypred, psi, d, y, 1e-15, 30)) rc = 1;
        history_update(S, q, D, d);
        memcpy(ys + (size_t)e * S, D, sizeof(double) * S);
      }
    }
    memcpy(yend, D, sizeof(double) * S);
    free(D); free(ypred); free(psi); free(d); free(y);
  }
  (void)yend;

  for (int j = 0; j < R; ++j) g_theta[j] = 0.0;
  memcpy(L, lam_final, sizeof(double) * S);
  for (int e = n - 1; e >= 0; --e) {
    const int kind = tp->kind[e], q = tp->q[e];
    const double val = tp->val[e];
    if (kind == 2) {
      const double c = val, igq = 1.0 / gamma_m(q);
      const double *y = ys + (size_t)e * S;
      for (int i = 0; i < S; ++i) {
        double s = L[(size_t)(q + 2) * S + i] + L[(size_t)(q + 1) * S + i];
        for (int k = 0; k <= q; ++k) s += L[(size_t)k * S + i];
        lamd[i] = s;
      }
      memcpy(nl, L, sizeof(double) * NROW * S);
      for (int i = 0; i < S; ++i) {
        nl[(size_t)(q + 1) * S + i] = -L[(size_t)(q + 2) * S + i];
        nl[(size_t)(q + 2) * S + i] = 0.0;
        double acc = 0.0;
        for (int k = 0; k <= q; ++k) {
          acc += L[(size_t)k * S + i];
          nl[(size_t)k * S + i] = acc;
        }
      }
      orc_jacobian(m, kt, y, J);
      if (solve_shifted(S, c, J, lamd, mu, 1)) rc = 1;
      matvec(S, J, mu, tmp, 1);                 /* J^T mu */
      for (int i = 0; i < S; ++i) {
        for (int k = 0; k <= q; ++k) nl[(size_t)k * S + i] += c * tmp[i];
        for (int k = 1; k <= q; ++k) nl[(size_t)k * S + i] -= gamma_m(k) * igq * mu[i];
      }
      rates(m, kt, y, r);
      nu_dot(m, mu, nm);
      for (int j = 0; j < R; ++j) g_theta[j] += c * r[j] * nm[j];
      memcpy(L, nl, sizeof(double) * NROW * S);
    } else if (kind == 1) {
      double T[ORC_QMAX][ORC_QMAX];
      rescale_T(S, q, val, T);
      for (int i = 0; i < S; ++i) {
        double in[ORC_QMAX];
        for (int k = 0; k < q; ++k) in[k] = L[(size_t)(k + 1) * S + i];
        for (int mm = 0; mm < q; ++mm) {
          double s = 0.0;
          for (int k = 0; k < q; ++k) s += T[k][mm] * in[k];
          L[(size_t)(mm + 1) * S + i] = s;
        }
      }
    } else {
      /* INIT: D_0 = y, D_1 = h0 f(y), higher rows reset */
      const double *y = yinit + (size_t)e * S;
      orc_jacobian(m, kt, y, J);
      matvec(S, J, L + S, tmp, 1);              /* J^T lambda_1 */
      rates(m, kt, y, r);
      nu_dot(m, L + S, nm);
      for (int j = 0; j < R; ++j) g_theta[j] += val * r[j] * nm[j];
      for (int i = 0; i < S; ++i) L[i] += val * tmp[i];
      for (size_t i = S; i < (size_t)NROW * S; ++i) L[i] = 0.0;
    }
  }
  memcpy(lam_y0, L, sizeof(double) * S);
  free(ys); free(yinit); free(yend); free(L); free(nl); free(lamd); free(mu); free(tmp); free(J); free(r); free(nm);
  return rc;
}
