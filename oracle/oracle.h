/*
 * oracle.h -- plain single-threaded FP64 CPU reference of the multi-cell stiff
 * chemistry solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
 * this code; it exists so that tests, the smoke check and the CPU-baseline leg
 * of the benchmark can compare the CUDA library against an independent,
 * obviously-correct implementation.  It shares no code, header or table with
 * the CUDA library.
 *
 * What it computes (paper: "Adapting atmospheric chemistry components for
 * efficient GPU accelerators", Background and Implementations sections):
 *   - reactions of the general form c1 y1 + ... -> c_{m+1} y_{m+1} + ...
 *     (Background, displayed reaction form);
 *   - per-reaction rate r_j and per-species contributions -c_i r_j for
 *     reactants and +c_i r_j for products (Background, per-reaction rate of
 *     change);
 *   - the derivative f_i = sum_j (dy_i/dt)_j (Background, derivative sum),
 *     evaluated independently per grid cell (Implementations, multi-cell
 *     derivative);
 *   - the analytic Jacobian of f (Background: CVODE is given a sparse
 *     Jacobian by the chemistry module);
 *   - an implicit BDF / Newton integration of y' = f(y) per cell (Background:
 *     CVODE, BDF with Newton iteration).  The paper only names CVODE; the
 *     integrator steps are the project's written specification (variable-order
 *     BDF in backward-difference form, Shampine & Reichelt 1997, with
 *     CVODE-style modified Newton, error test and step/order control).
 *
 * The oracle solves the Newton systems with a dense LU with partial pivoting,
 * deliberately unlike the GPU's static-order sparse LU.
 */
#ifndef CHEM_ORACLE_H
#define CHEM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_REAC 3
#define ORC_MAX_PROD 8
#define ORC_QMAX 5

enum { ORC_THERMAL = 0, ORC_PHOTOLYSIS = 1, ORC_TROE = 2, ORC_PRESSURE_SUM = 3, ORC_FALLOFF_SUM = 4 };

enum {
  ORC_OK = 0,
  ORC_MAX_STEPS = 1,
  ORC_H_TOO_SMALL = 2,
  ORC_ERR_FAIL = 3,
  ORC_CONV_FAIL = 4,
  ORC_NONFINITE = 5,
  ORC_BAD_INPUT = 6
};

/* Reaction tables; arrays owned by the caller. reac is [R][3], prod/yld [R][8].
 * ext [R][8] (may be NULL when every reaction is thermal or photolysis): the
 * second Arrhenius term (A2, Ea2/R, B2), the third (A3, Ea3/R, B3), and the
 * Troe broadening Fc, N. */
typedef struct {
  int32_t n_species, n_reactions;
  const int32_t *kind, *n_reac, *reac, *n_prod, *prod;
  const double *yld, *A, *Ea, *B, *J;
  const double *ext;
} orc_mech;

typedef struct {
  double rtol, atol;
  int32_t max_order, max_steps;
  /* test hooks, all off when zero / NULL */
  double fixed_h;            /* >0: constant step, no error test, no step/order selection */
  int32_t fixed_order;       /* order used with fixed_h */
  int32_t newton_maxiter;    /* >0: overrides the corrector iteration cap */
  double newton_tol;         /* >0: overrides the corrector tolerance */
  const double *init_D;      /* fixed_h: initial differences D_0..D_q, [q+1][S] */
  double *y_hist;            /* fixed_h: receives y after each step, [n][S] */
  int32_t plain_form;        /* 1: every test in its plain form -- norms with the square root,
                                the convergence-rate estimate on norms, divisions by q + 1, q,
                                q + 2 and c_M, the step-factor grid on unsquared thresholds -- for
                                the pin that the default form (squared norms against squared
                                bounds, reciprocal multiplications) makes the same decisions */
} orc_opts;

typedef struct {
  int32_t status, steps, rejects, conv_fails, newton_iters, f_evals, jac_evals, solves, final_order, order_sum;
  double final_h;
} orc_stats;

/* Tape of one cell's integration: the operations that determined its result,
 * in order.  kind 0 = INIT (val = h0, y = y0); 1 = RESCALE of the history
 * (q, val = eta); 2 = accepted STEP (q, val = c = h/gamma_q, y = accepted y);
 * 3 = PROJECT (q = a species the following STEP projected onto y = 0);
 * 4 = REFACTOR (val = c_M, y = the state J was evaluated at: M = I - c_M J(y));
 * 5 = ITER (y = a Newton iterate of the following STEP, in order).
 * Arrays are sized by the caller (cap events; y is [cap][S]). */
typedef struct {
  int32_t cap, n, overflow, pad;
  int32_t *kind, *q;
  double *val;
  double *y;
} orc_tape;

/* a1: per-reaction rate constants k~_j of one cell.  jphot: photolysis rates in
 * photolysis-reaction order (NULL: the mechanism's J).  theta: per-reaction log
 * multipliers (NULL: none). */
void orc_rate_constants(const orc_mech *m, double T, double P, const double *jphot,
                        const double *theta, double *kt);
/* a2: f(y). */
void orc_deriv(const orc_mech *m, const double *kt, const double *y, double *f);
/* a3: dense Jacobian J[i*S+l] = df_i/dy_l. */
void orc_jacobian(const orc_mech *m, const double *kt, const double *y, double *J);
/* dense LU with partial pivoting (in place); returns 0, or k+1 for an exactly zero pivot k */
int orc_lu_factor(int n, double *A, int32_t *piv);
void orc_lu_solve(int n, const double *LU, const int32_t *piv, double *b);
/* history rescale of differences D_1..D_q (rows of length S) for a step ratio eta */
void orc_rescale(int S, int q, double eta, double *D);
/* step-factor grid: largest grid factor g with bias*err*g^(p+1) <= 1, tested on
 * err2 = err^2 against 1/(bias^2 g^(2(p+1))) */
double orc_grid_eta(double err2, int p, double bias);
/* integrate one cell over [0, dt]; y is in/out (kept on failure); tape may be NULL */
int orc_integrate(const orc_mech *m, const double *kt, double *y, double dt, const orc_opts *o,
                  orc_stats *st, orc_tape *tape);
/* all cells: y [S][C] (cell unit stride) in/out, jphot [n_phot][C] or NULL, theta [R] or NULL */
int orc_solve_cells(const orc_mech *m, int64_t n_cells, const double *T, const double *P,
                    const double *jphot, const double *theta, double *y, double dt,
                    const orc_opts *o, orc_stats *st);

/* adjoint.c: the frozen-control map of a tape (every control decision of the
 * integrator held fixed: step sizes, orders, corrector iteration counts,
 * iteration matrices formed from the recorded states, projections), its
 * tangent and its discrete adjoint.  kt includes theta.  orc_replay forms the
 * iteration matrices with kt_M (NULL: kt), so that a perturbed kt can be
 * replayed against the matrices of the recorded run.  y_steps (optional)
 * receives y after every STEP event ([tape n][S], other rows untouched).
 * Return 0, or 1 if an iteration matrix was exactly singular or a STEP had no
 * iteration matrix before it. */
int orc_replay(const orc_mech *m, const double *kt, const double *kt_M, const double *y0, const orc_tape *tape,
               double *y_out, double *y_steps);
int orc_tangent(const orc_mech *m, const double *kt, const double *y0, const orc_tape *tape, const double *dy0,
                const double *dtheta, double *dy_out);
int orc_adjoint(const orc_mech *m, const double *kt, const double *y0, const orc_tape *tape,
                const double *lam_final, double *lam_y0, double *g_theta);

#ifdef __cplusplus
}
#endif
#endif
