/*
 * adjoint.c -- the frozen-control map of a tape, its tangent and its discrete
 * adjoint, for the oracle.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The map.  An integration leaves a tape (orc_tape) of everything that
 * determined its result.  The frozen-control map (y0, theta) -> y_final
 * recomputes that result with every control decision of the integrator held
 * fixed (step sizes, orders, the number of corrector iterations, the
 * iteration matrices, the projections):
 *   INIT      D_0 = y (the current state), D_1 = h0 f(y), higher rows 0;
 *   RESCALE   D_{1..q} <- T(eta) D_{1..q}  (history rescale at order q);
 *   REFACTOR  M = I - c_M J(y_J) with y_J the RECORDED state and the rate
 *             constants of the recorded run: the iteration matrix is a
 *             preconditioner, a constant of the map (it depends neither on y0
 *             nor on theta);
 *   ITER      counts the corrector iterations K of the next STEP;
 *   PROJECT   marks a species that the next STEP projects onto y = 0;
 *   STEP      (q, c): y_pred = sum_{m<=q} D_m, psi = (1/gamma_q) sum_{m=1..q}
 *             gamma_m D_m, d_0 = 0 and K modified-Newton iterations
 *                 d_{k+1} = d_k + s M^{-1} (c f(y_pred + d_k) - psi - d_k),
 *             s = 1 if c == c_M else 2/(1 + c (1/c_M)); projected species then
 *             get d_i = -y_pred_i (y_i = 0); the history is updated with
 *             D_{q+2} = d - D_{q+1}, D_{q+1} = d, D_m += D_{m+1} (m = q..0).
 * With the recorded inputs this is the integrator's own arithmetic, so the map
 * reproduces its result exactly; the adjoint below is the exact adjoint of the
 * map.  A tape may hold several consecutive solves: every INIT restarts the
 * history from the current D_0.
 *
 * Sensitivities are taken with respect to y0 and to theta, the per-reaction
 * log multipliers of the rate constants (k~_j -> k~_j e^{theta_j}), at the
 * theta already folded into kt; d r_j / d theta_j = r_j.
 *
 * Adjoint of a STEP (lambda' the adjoint of D after it):
 *   lambda_d = lambda'_{q+2} + lambda'_{q+1} + sum_{m<=q} lambda'_m;
 *   lambda_i = sum_{m<=i} lambda'_m (i <= q), lambda_{q+1} = -lambda'_{q+2},
 *   lambda_{q+2} = 0;
 *   projected i: lambda_ypred,i = -lambda_d,i and lambda_d,i = 0;
 *   for k = K-1..0, with g = s M^{-T} lambda_d and y_k = y_pred + d_k:
 *     lambda_ypred += c J(y_k)^T g,  lambda_psi -= g,
 *     lambda_d += c J(y_k)^T g - g,  dL/dtheta_j += c r_j(y_k) (nu_j . g);
 *   lambda_i += lambda_ypred (i <= q),
 *   lambda_i += (gamma_i/gamma_q) lambda_psi (1 <= i <= q).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define NROW (ORC_QMAX + 3)

enum { EV_INIT = 0, EV_RESCALE = 1, EV_STEP = 2, EV_PROJECT = 3, EV_REFACTOR = 4, EV_ITER = 5 };

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

/* the iteration matrix of a REFACTOR event, M = I - c_M J(y_J), as dense LUs
 * of M and of M^T */
typedef struct {
  double *LU, *LUT;
  int32_t *piv, *pivT;
  double cM;
} iter_matrix;

static void im_alloc(iter_matrix *im, int S) {
  im->LU = (double *)malloc(sizeof(double) * S * S);
  im->LUT = (double *)malloc(sizeof(double) * S * S);
  im->piv = (int32_t *)malloc(sizeof(int32_t) * S);
  im->pivT = (int32_t *)malloc(sizeof(int32_t) * S);
  im->cM = 0.0;
}
static void im_free(iter_matrix *im) { free(im->LU); free(im->LUT); free(im->piv); free(im->pivT); }

/* forms M the way the integrator does; returns nonzero for an exactly singular M */
static int im_form(iter_matrix *im, const orc_mech *m, const double *kt, const double *yJ, double cM) {
  const int S = m->n_species;
  orc_jacobian(m, kt, yJ, im->LU);
  for (int i = 0; i < S * S; ++i) im->LU[i] = -cM * im->LU[i];
  for (int i = 0; i < S; ++i) im->LU[i * S + i] += 1.0;
  for (int i = 0; i < S; ++i)
    for (int k = 0; k < S; ++k) im->LUT[i * S + k] = im->LU[k * S + i];
  im->cM = cM;
  const int a = orc_lu_factor(S, im->LU, im->piv);
  const int b = orc_lu_factor(S, im->LUT, im->pivT);
  return a != 0 || b != 0;
}

/* y_pred and psi of a step at order q, summed in the integrator's order */
static void predict(int S, int q, const double *D, double *ypred, double *psi) {
  const double igq = 1.0 / gamma_m(q);
  for (int i = 0; i < S; ++i) {
    double s = D[i];
    for (int k = 1; k <= q; ++k) s += D[(size_t)k * S + i];
    ypred[i] = s;
  }
  for (int i = 0; i < S; ++i) {
    double p = 0.0;
    for (int k = 1; k <= q; ++k) p += gamma_m(k) * D[(size_t)k * S + i];
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

/* the rescale matrix T(eta) on rows 1..q, read off orc_rescale column by column */
static void rescale_T(int q, double eta, double T[ORC_QMAX][ORC_QMAX]) {
  double D[ORC_QMAX + 1];
  for (int mm = 0; mm < q; ++mm) {
    memset(D, 0, sizeof(D));
    D[mm + 1] = 1.0;
    orc_rescale(1, q, eta, D);
    for (int i = 0; i < q; ++i) T[i][mm] = D[i + 1];
  }
}

static double step_scale(double c, double cM) { return (c == cM) ? 1.0 : 2.0 / (1.0 + c * (1.0 / cM)); }

/*
 * One walk of the map; iteration matrices are formed with the rate constants
 * ktM, the map's arithmetic uses kt.  With dy0 non-NULL it also carries the tangent dD
 * (dtheta then non-NULL too).  iters (optional) receives every corrector
 * iterate y_k in tape order ([number of ITER events][S]); yinit the state at
 * every INIT ([tape n][S]); y_steps y after every STEP ([tape n][S]).
 */
static int walk(const orc_mech *m, const double *kt, const double *ktM, const double *y0, const orc_tape *tp,
                const double *dy0,
                const double *dtheta, double *y_out, double *dy_out, double *iters, double *yinit,
                double *y_steps) {
  const int S = m->n_species, R = m->n_reactions;
  const int tan = dy0 != NULL;
  double *D = (double *)calloc((size_t)NROW * S, sizeof(double));
  double *dD = (double *)calloc((size_t)NROW * S, sizeof(double));
  double *ypred = (double *)malloc(sizeof(double) * S), *psi = (double *)malloc(sizeof(double) * S);
  double *dyp = (double *)malloc(sizeof(double) * S), *dpsi = (double *)malloc(sizeof(double) * S);
  double *d = (double *)malloc(sizeof(double) * S), *dd = (double *)malloc(sizeof(double) * S);
  double *y = (double *)malloc(sizeof(double) * S), *dyv = (double *)malloc(sizeof(double) * S);
  double *f = (double *)malloc(sizeof(double) * S), *rr = (double *)malloc(sizeof(double) * S);
  double *tmp = (double *)malloc(sizeof(double) * S), *b = (double *)malloc(sizeof(double) * S);
  double *J = (double *)malloc(sizeof(double) * S * S);
  double *r = (double *)malloc(sizeof(double) * (R > 0 ? R : 1));
  int *mask = (int *)calloc((size_t)S, sizeof(int));
  iter_matrix im;
  im_alloc(&im, S);
  int K = 0, rc = 0, have_M = 0;
  long row = 0;
  memcpy(D, y0, sizeof(double) * S);
  if (tan) memcpy(dD, dy0, sizeof(double) * S);
  for (int e = 0; e < tp->n; ++e) {
    const int kind = tp->kind[e], q = tp->q[e];
    const double val = tp->val[e];
    if (kind == EV_INIT) {
      if (yinit) memcpy(yinit + (size_t)e * S, D, sizeof(double) * S);
      for (size_t i = S; i < (size_t)NROW * S; ++i) D[i] = dD[i] = 0.0;
      orc_deriv(m, kt, D, f);
      if (tan) {
        orc_jacobian(m, kt, D, J);
        rates(m, kt, D, r);
        matvec(S, J, dD, tmp, 0);
        ftheta_times(m, r, dtheta, b);
      }
      for (int i = 0; i < S; ++i) {
        D[S + i] = val * f[i];
        if (tan) dD[S + i] = val * (tmp[i] + b[i]);
      }
    } else if (kind == EV_RESCALE) {
      orc_rescale(S, q, val, D);
      if (tan) orc_rescale(S, q, val, dD);
    } else if (kind == EV_REFACTOR) {
      if (im_form(&im, m, ktM, tp->y + (size_t)e * S, val)) rc = 1;
      have_M = 1;
    } else if (kind == EV_ITER) {
      K++;
    } else if (kind == EV_PROJECT) {
      mask[q] = 1;
    } else if (kind == EV_STEP) {
      if (!have_M) { rc = 1; break; }
      const double c = val, s = step_scale(c, im.cM);
      predict(S, q, D, ypred, psi);
      if (tan) predict(S, q, dD, dyp, dpsi);
      for (int i = 0; i < S; ++i) d[i] = dd[i] = 0.0;
      for (int k = 0; k < K; ++k) {
        for (int i = 0; i < S; ++i) y[i] = ypred[i] + d[i];
        if (iters) memcpy(iters + (size_t)(row + k) * S, y, sizeof(double) * S);
        orc_deriv(m, kt, y, f);
        for (int i = 0; i < S; ++i) rr[i] = c * f[i] - psi[i] - d[i];
        orc_lu_solve(S, im.LU, im.piv, rr);
        if (tan) {
          for (int i = 0; i < S; ++i) dyv[i] = dyp[i] + dd[i];
          orc_jacobian(m, kt, y, J);
          rates(m, kt, y, r);
          matvec(S, J, dyv, tmp, 0);
          ftheta_times(m, r, dtheta, b);
          for (int i = 0; i < S; ++i) b[i] = c * (tmp[i] + b[i]) - dpsi[i] - dd[i];
          orc_lu_solve(S, im.LU, im.piv, b);
        }
        for (int i = 0; i < S; ++i) {
          if (s != 1.0) rr[i] *= s;
          d[i] += rr[i];
          if (tan) dd[i] += s * b[i];
        }
      }
      row += K;
      for (int i = 0; i < S; ++i)
        if (mask[i]) {
          d[i] -= ypred[i] + d[i];
          if (tan) dd[i] = -dyp[i];
        }
      history_update(S, q, D, d);
      if (tan) history_update(S, q, dD, dd);
      if (y_steps) memcpy(y_steps + (size_t)e * S, D, sizeof(double) * S);
      memset(mask, 0, sizeof(int) * S);
      K = 0;
    }
  }
  if (y_out) memcpy(y_out, D, sizeof(double) * S);
  if (dy_out) memcpy(dy_out, dD, sizeof(double) * S);
  im_free(&im);
  free(D); free(dD); free(ypred); free(psi); free(dyp); free(dpsi); free(d); free(dd); free(y); free(dyv);
  free(f); free(rr); free(tmp); free(b); free(J); free(r); free(mask);
  return rc;
}

int orc_replay(const orc_mech *m, const double *kt, const double *kt_M, const double *y0, const orc_tape *tp,
               double *y_out, double *y_steps) {
  return walk(m, kt, kt_M ? kt_M : kt, y0, tp, NULL, NULL, y_out, NULL, NULL, NULL, y_steps);
}

int orc_tangent(const orc_mech *m, const double *kt, const double *y0, const orc_tape *tp, const double *dy0,
                const double *dtheta, double *dy_out) {
  return walk(m, kt, kt, y0, tp, dy0, dtheta, NULL, dy_out, NULL, NULL, NULL);
}

int orc_adjoint(const orc_mech *m, const double *kt, const double *y0, const orc_tape *tp, const double *lam_final,
                double *lam_y0, double *g_theta) {
  const int S = m->n_species, R = m->n_reactions, n = tp->n;
  long n_rows = 0;
  for (int e = 0; e < n; ++e) n_rows += tp->kind[e] == EV_ITER;
  double *iters = (double *)malloc(sizeof(double) * (size_t)(n_rows > 0 ? n_rows : 1) * S);
  double *yinit = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * S);
  double *L = (double *)calloc((size_t)NROW * S, sizeof(double));
  double *lamd = (double *)malloc(sizeof(double) * S), *g = (double *)malloc(sizeof(double) * S);
  double *lyp = (double *)malloc(sizeof(double) * S), *lpsi = (double *)malloc(sizeof(double) * S);
  double *tmp = (double *)malloc(sizeof(double) * S), *J = (double *)malloc(sizeof(double) * S * S);
  double *r = (double *)malloc(sizeof(double) * (R > 0 ? R : 1));
  double *nm = (double *)malloc(sizeof(double) * (R > 0 ? R : 1));
  int *mask = (int *)calloc((size_t)S, sizeof(int));
  iter_matrix im;
  im_alloc(&im, S);
  int im_event = -1;
  int rc = walk(m, kt, kt, y0, tp, NULL, NULL, NULL, NULL, iters, yinit, NULL);

  for (int j = 0; j < R; ++j) g_theta[j] = 0.0;
  memcpy(L, lam_final, sizeof(double) * S);
  long row = n_rows;               /* iterates of the STEPs not yet visited: rows [0, row) */
  for (int e = n - 1; e >= 0 && rc == 0; --e) {
    const int kind = tp->kind[e], q = tp->q[e];
    const double val = tp->val[e];
    if (kind == EV_STEP) {
      /* the step's projections and iteration count precede it */
      memset(mask, 0, sizeof(int) * S);
      int K = 0, e2 = e - 1;
      for (; e2 >= 0 && (tp->kind[e2] == EV_PROJECT || tp->kind[e2] == EV_ITER); --e2) {
        if (tp->kind[e2] == EV_PROJECT) mask[tp->q[e2]] = 1;
        else K++;
      }
      /* the iteration matrix in force: the last REFACTOR before the step */
      int er = e2;
      while (er >= 0 && tp->kind[er] != EV_REFACTOR) --er;
      if (er < 0) { rc = 1; break; }
      if (er != im_event) {
        if (im_form(&im, m, kt, tp->y + (size_t)er * S, tp->val[er])) rc = 1;
        im_event = er;
      }
      const double c = val, s = step_scale(c, im.cM), igq = 1.0 / gamma_m(q);
      row -= K;
      /* history update, then projection */
      for (int i = 0; i < S; ++i) {
        double acc = 0.0;
        for (int k = 0; k <= q; ++k) {
          acc += L[(size_t)k * S + i];
          L[(size_t)k * S + i] = acc;
        }
        lamd[i] = L[(size_t)(q + 2) * S + i] + L[(size_t)(q + 1) * S + i] + acc;
        L[(size_t)(q + 1) * S + i] = -L[(size_t)(q + 2) * S + i];
        L[(size_t)(q + 2) * S + i] = 0.0;
        lyp[i] = 0.0;
        lpsi[i] = 0.0;
        if (mask[i]) {
          lyp[i] = -lamd[i];
          lamd[i] = 0.0;
        }
      }
      /* the K corrector iterations, last first */
      for (int k = K - 1; k >= 0; --k) {
        const double *yk = iters + (size_t)(row + k) * S;
        memcpy(g, lamd, sizeof(double) * S);
        orc_lu_solve(S, im.LUT, im.pivT, g);
        for (int i = 0; i < S; ++i) g[i] *= s;
        orc_jacobian(m, kt, yk, J);
        matvec(S, J, g, tmp, 1);
        rates(m, kt, yk, r);
        nu_dot(m, g, nm);
        for (int j = 0; j < R; ++j) g_theta[j] += c * r[j] * nm[j];
        for (int i = 0; i < S; ++i) {
          lamd[i] += c * tmp[i] - g[i];
          lyp[i] += c * tmp[i];
          lpsi[i] -= g[i];
        }
      }
      for (int i = 0; i < S; ++i) {
        for (int k = 0; k <= q; ++k) L[(size_t)k * S + i] += lyp[i];
        for (int k = 1; k <= q; ++k) L[(size_t)k * S + i] += gamma_m(k) * igq * lpsi[i];
      }
    } else if (kind == EV_RESCALE) {
      double T[ORC_QMAX][ORC_QMAX];
      rescale_T(q, val, T);
      for (int i = 0; i < S; ++i) {
        double in[ORC_QMAX];
        for (int k = 0; k < q; ++k) in[k] = L[(size_t)(k + 1) * S + i];
        for (int mm = 0; mm < q; ++mm) {
          double s2 = 0.0;
          for (int k = 0; k < q; ++k) s2 += T[k][mm] * in[k];
          L[(size_t)(mm + 1) * S + i] = s2;
        }
      }
    } else if (kind == EV_INIT) {
      /* D_0 = y, D_1 = h0 f(y), higher rows reset */
      const double *y = yinit + (size_t)e * S;
      orc_jacobian(m, kt, y, J);
      matvec(S, J, L + S, tmp, 1);
      rates(m, kt, y, r);
      nu_dot(m, L + S, nm);
      for (int j = 0; j < R; ++j) g_theta[j] += val * r[j] * nm[j];
      for (int i = 0; i < S; ++i) L[i] += val * tmp[i];
      for (size_t i = S; i < (size_t)NROW * S; ++i) L[i] = 0.0;
    }
    /* ITER, PROJECT and REFACTOR are consumed by their STEP */
  }
  memcpy(lam_y0, L, sizeof(double) * S);
  im_free(&im);
  free(iters); free(yinit); free(L); free(lamd); free(g); free(lyp); free(lpsi); free(tmp); free(J); free(r);
  free(nm); free(mask);
  return rc;
}
