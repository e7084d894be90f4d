/*
 * chemgpu.h -- C ABI of the GB300 multi-cell stiff chemistry solver.
 *
 * The library integrates a gas-phase mass-action mechanism independently in
 * every grid cell of a batch with an implicit BDF / modified-Newton method,
 * entirely on the GPU: per-cell rate constants and derivative f(y), the
 * analytic sparse Jacobian, and a static-order sparse LU factor/solve of the
 * Newton iteration matrix I - c*J.
 *
 * Paper: "Adapting atmospheric chemistry components for efficient GPU
 * accelerators" (arXiv 2501.00011).  The chemistry follows its Background
 * section (reaction form c1 y1 + ... -> c_{m+1} y_{m+1} + ..., per-reaction
 * rate of change -c_i r_j / +c_i r_j, derivative f_i = sum_j (dy_i/dt)_j);
 * the batching of all cells into one structure with the cell loop inside the
 * solver follows its Implementations section (Multi-cells); its Conclusions
 * name the whole ODE solve on the GPU, which is what this library does.  The
 * integrator (BDF orders 1-5, modified Newton, error and step/order control)
 * stands for the CVODE solver the Background section names.
 *
 * Conventions for every entry point:
 *   - return value 0 = success, negative = error (CHEM_E*); on error nothing
 *     was launched and chem_last_error() (thread-local) describes it;
 *   - "mem" arguments say where a pointer lives: CHEM_MEM_HOST (pageable or
 *     pinned host memory) or CHEM_MEM_DEVICE (memory of the current CUDA
 *     device, or managed memory); a CHEM_MEM_DEVICE pointer that is neither
 *     (host memory, another device's memory) is refused with CHEM_EINVAL
 *     before anything is launched or copied;
 *   - "stream" is a cudaStream_t (NULL = the legacy default stream); device
 *     work is enqueued on it and the call returns without waiting, except
 *     where a host buffer is read back;
 *   - pointers passed in are borrowed for the duration of the call only;
 *   - state arrays are [n_species][n_cells] with the cell index at unit
 *     stride, FP64, in mol/mol; T in K; P in Pa.
 * No entry point aborts the process or traps the GPU.  A cell that cannot be
 * integrated keeps its input state and reports a non-zero status.
 */
#ifndef CHEMGPU_H
#define CHEMGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHEM_MAX_REAC 3
#define CHEM_MAX_PROD 8
#define CHEM_MAX_SPECIES 128
#define CHEM_MAX_TAPE_ROWS (1 << 20)   /* largest chem_opts.tape_steps */
#define CHEM_MAX_GRAPH_STEPS 4096      /* largest n_steps of chem_solve_steps */
#define CHEM_AUTOTUNE_SAMPLE 16384     /* default sample of chem_autotune */

/* error codes (negative returns) */
#define CHEM_EINVAL (-1)   /* bad argument or mechanism table */
#define CHEM_ENOMEM (-2)   /* device or host allocation failed */
#define CHEM_ECUDA (-3)    /* a CUDA runtime call failed */
#define CHEM_ESTATE (-4)   /* call out of order (e.g. solve before set_state) */
#define CHEM_EABORTED (-5) /* a chem_pipeline_run callback asked to stop */

/* where a pointer lives */
#define CHEM_MEM_HOST 0
#define CHEM_MEM_DEVICE 1

/* reaction kinds.  The rate r_j is a function of the state, T and P
 * (Background section); every kind keeps mass action r = k~(T, P) prod y, with
 * k~ the rate constant below times n_air^(n_reac-1) so that rates act on
 * mixing ratios.  Arrhenius terms: k_a = A exp(-Ea/T) (T/300)^B (parameters
 * A, Ea_over_R, B), k_b likewise from A2, Ea2_over_R, B2 and k_c from A3,
 * Ea3_over_R, B3; [M] = n_air, the number density of air (molecules cm^-3). */
#define CHEM_THERMAL 0     /* k = k_a */
#define CHEM_PHOTOLYSIS 1  /* first-order rate J (s^-1), optionally per cell */
#define CHEM_TROE 2        /* pressure fall-off between k0 = k_a (low-pressure limit, per [M]) and
                              kinf = k_b (high-pressure limit): with x = k0 [M] / kinf,
                              k = k0 [M] / (1 + x) * Fc^(1 / (1 + (log10(x) / N)^2)); Fc in (0, 1],
                              N > 0 (Fc = 1: Lindemann-Hinshelwood) */
#define CHEM_PRESSURE_SUM 3   /* k = k_a + k_b [M] (a pressure-dependent term added to a
                                 bimolecular one, as for HO2 + HO2) */
#define CHEM_FALLOFF_SUM 4    /* k = k_a + k_c [M] / (1 + k_c [M] / k_b) (as for OH + HNO3) */

/* per-cell status */
#define CHEM_CELL_OK 0
#define CHEM_CELL_MAX_STEPS 1
#define CHEM_CELL_H_TOO_SMALL 2
#define CHEM_CELL_ERR_FAIL 3
#define CHEM_CELL_CONV_FAIL 4
#define CHEM_CELL_NONFINITE 5
#define CHEM_CELL_BAD_INPUT 6

/* drivers */
#define CHEM_DRIVER_PLAIN 0       /* one warp per cell, cells assigned by block */
#define CHEM_DRIVER_PERSISTENT 1  /* resident warps pop cells from a device queue, most expensive
                                     first: by each cell's cost in the previous solve of the
                                     batch, or for the first solve by the sum of its rate
                                     constants (results do not depend on the order) */

/*
 * One reaction: reactant slots reac[0..n_reac-1] (a species listed twice is a
 * second-order dependence, e.g. 2A), products prod[0..n_prod-1] with yields.
 * Mass action: r = k~ * prod_s y[reac[s]]; each reactant slot loses r, each
 * product gains yield * r (Background section, per-reaction rate of change).
 */
typedef struct {
  int32_t kind;                   /* CHEM_THERMAL .. CHEM_FALLOFF_SUM */
  int32_t n_reac;                 /* 1..CHEM_MAX_REAC */
  int32_t reac[CHEM_MAX_REAC];
  int32_t n_prod;                 /* 0..CHEM_MAX_PROD */
  int32_t prod[CHEM_MAX_PROD];
  double yield[CHEM_MAX_PROD];
  double A, Ea_over_R, B;         /* Arrhenius term k_a */
  double J;                       /* photolysis rate (s^-1) */
  double A2, Ea2_over_R, B2;      /* Arrhenius term k_b (TROE, PRESSURE_SUM, FALLOFF_SUM) */
  double A3, Ea3_over_R, B3;      /* Arrhenius term k_c (FALLOFF_SUM) */
  double Fc, N;                   /* TROE broadening */
} chem_reaction;

typedef struct chem_mech chem_mech;
typedef struct chem_cells chem_cells;

/* Structure of a compiled mechanism (sizes of its sparse tables and of the
 * per-cell work, and algorithmic FP64 operation counts per kernel step). */
typedef struct {
  int32_t n_species, n_reactions, n_photolysis;
  int32_t nnz_jac;                 /* nonzeros of J plus the diagonal */
  int32_t nnz_lu;                  /* nonzeros after the static-order fill */
  int32_t n_pairs;                 /* (reaction, reactant slot) partials */
  int32_t passes_f, passes_jac, passes_lu, passes_fwd, passes_bwd;  /* warp passes */
  int32_t ops_f, ops_jac, ops_lu, ops_fwd, ops_bwd;                 /* scheduled ops */
  double flops_f, flops_jac, flops_lu, flops_solve;                 /* algorithmic flops */
  int32_t smem_per_cell_fp64, smem_per_cell_fp32;                   /* bytes */
  double flops_adj_iter;           /* adjoint, per corrector iteration walked back: transposed
                                      solve, rates and partials, nu.g, J^T g, theta update, vectors */
  double flops_tan_iter;           /* tangent, per corrector iteration: tangent rates (with a theta
                                      direction), the f program on them, one solve, vectors */
} chem_mech_info;

typedef struct {
  double rtol, atol;
  int32_t max_order;               /* 1..5 (default 5) */
  int32_t max_steps;               /* default 5000 */
  int32_t lu_precision;            /* 64 (default) or 32: LU factor/solve in FP32 */
  int32_t driver;                  /* CHEM_DRIVER_* */
  int32_t cells_per_block;         /* warps (= concurrent cells) per block; 0 = auto: 1 for the
                                      plain driver, the most resident cells per SM for the
                                      persistent one (chem_autotune measures instead) */
  int32_t blocks_per_sm;           /* persistent driver: resident blocks per SM; 0 = auto (as
                                      many as fit); fewer than fit are kept to by padding each
                                      block's shared memory, so the blocks spread over the SMs */
  int32_t record_adjoint;          /* 1: record the tape for chem_sensitivity (needs lu_precision 64) */
  int32_t tape_steps;              /* tape rows per cell: states stored, one per solve, per
                                      refactorisation and per accepted corrector iteration
                                      (0 = 2000, at most CHEM_MAX_TAPE_ROWS); events 3x that + 64 */
  int32_t couple_cells;            /* 1 (default): every cell integrated on its own.  G > 1: the
                                      paper's multi-cell system (Implementations, Multi-cells): cells
                                      integrated in groups of G consecutive cells, each group one ODE
                                      system with shared step size, order and Newton iterations and
                                      one WRMS norm over all its species (the linear systems stay
                                      block-diagonal, one block per cell).  FP64 only, no adjoint;
                                      cells_per_block must be a multiple of G (0: the largest that
                                      fits); a CUDA block holds whole groups; the persistent
                                      driver hands out whole groups, most expensive first by
                                      their cost in the previous solve. */
  int32_t stage_wait;              /* persistent driver, test hook: polls of the bounded wait for a
                                      block's bulk copy of the tables into shared memory.  0 (default):
                                      2^22; -1: none, so every block copies the tables with ordinary
                                      loads instead (the same bytes; results are identical) and
                                      counts a fallback, see chem_staging_fallbacks */
} chem_opts;

/* Per-cell outcome of a solve: status (CHEM_CELL_*), accepted steps, rejected
 * attempts, corrector failures, Newton iterations, f evaluations, Jacobian
 * evaluations (= factorisations), linear solves, the order at the end, the sum
 * over accepted steps of the order each was taken at, and the last step size. */
typedef struct {
  int32_t status, steps, rejects, conv_fails, newton_iters, f_evals, jac_evals, solves,
      final_order, order_sum;
  double final_h;
} chem_cell_stats;

/* Fill opts with the defaults (rtol 1e-4, atol 1e-10, order 5, 5000 steps, FP64 LU,
 * plain driver, automatic launch shape, no adjoint). */
void chem_opts_default(chem_opts *opts);

/* Compile a mechanism.  Paper, Background section: reactions of the general
 * form c1 y1 + ... -> c_{m+1} y_{m+1} + ..., each with a rate r_j that is a
 * function of the state, T and P, contributing -c_i r_j to each reactant and
 * +c_i r_j to each product; the derivative is the sum of the contributions.
 * The rate constants are the CHEM_* kinds above.  Validate the tables
 * (species indices in range, yields finite, rate parameters finite,
 * n_species <= CHEM_MAX_SPECIES), build the
 * Jacobian pattern, a static Markowitz pivot order, the LU fill and the warp
 * programs, and copy them to the current device.  rx: n_reactions entries,
 * borrowed.  *out is owned by the caller and released with
 * chem_mechanism_destroy.  Errors: CHEM_EINVAL, CHEM_ENOMEM, CHEM_ECUDA. */
int chem_mechanism_create(int32_t n_species, int32_t n_reactions, const chem_reaction *rx,
                          chem_mech **out);
void chem_mechanism_destroy(chem_mech *mech);   /* NULL is a no-op */
int chem_mechanism_info(const chem_mech *mech, chem_mech_info *out);
/* Jacobian pattern after the static ordering: position of each species in the
 * pivot order (pos[n_species]) and the LU fill as a dense 0/1 matrix in pivot
 * order (fill[n_species*n_species], row-major; may be NULL). */
int chem_mechanism_structure(const chem_mech *mech, int32_t *pos, uint8_t *fill);

/* Allocate the device state of n_cells cells for a mechanism (which must
 * outlive the batch).  Paper, Background section: every grid cell carries its
 * own temperature, pressure and concentrations and its chemistry is
 * independent of the other cells'; Implementations section (Multi-cells): all
 * cells' data in one structure, with the cell loop inside the solver.  The
 * batch lives on the current device, which is the mechanism's and must be
 * current in every later call on the batch (else CHEM_EINVAL).  opts NULL =
 * defaults.  *out released with chem_cells_destroy.  Errors: CHEM_EINVAL,
 * CHEM_ENOMEM, CHEM_ECUDA. */
int chem_cells_create(const chem_mech *mech, int64_t n_cells, const chem_opts *opts,
                      chem_cells **out);
void chem_cells_destroy(chem_cells *cells);      /* NULL is a no-op */

/* Copy T[n_cells] (K), P[n_cells] (Pa) and y[n_species][n_cells] (mol/mol,
 * cell index unit stride) into the batch (D2D for CHEM_MEM_DEVICE, H2D
 * otherwise), asynchronously on stream; the caller's arrays may be reused once
 * the stream has passed the copies.  Paper, Background section: the state,
 * temperature and pressure of each cell that the rates depend on;
 * Implementations section: the multi-cell state is one array over all cells.
 * Resets the adjoint tape.  Errors: CHEM_EINVAL, CHEM_ECUDA. */
int chem_cells_set_state(chem_cells *cells, const double *T, const double *P, const double *y,
                         int32_t mem, void *stream);
/* Per-cell photolysis rates J[n_photolysis][n_cells] in s^-1 (photolysis
 * reactions in reaction order); NULL reverts to the mechanism's J.  Paper,
 * Background section: a rate is a function of the cell's state (here, its
 * light).  Errors as above. */
int chem_cells_set_photolysis(chem_cells *cells, const double *J, int32_t mem, void *stream);
/* Per-reaction log multipliers theta[n_reactions], shared by all cells:
 * k~_j -> k~_j exp(theta_j).  NULL reverts to theta = 0. */
int chem_cells_set_theta(chem_cells *cells, const double *theta, int32_t mem, void *stream);

/* Integrate every cell over [0, dt] (dt > 0, seconds) on stream; the
 * integrator starts afresh and the new state replaces the old.  Paper,
 * Background section: the chemistry module hands CVODE the derivative and a
 * sparse Jacobian, and CVODE integrates with BDF and Newton iteration; here
 * the whole integration runs on the GPU (variable-order BDF 1-5, modified
 * Newton on I - c J with a static-order sparse LU, error test and step/order
 * control, per cell).  Results do not depend on the driver, the launch shape
 * or the order the persistent queue takes the cells in.  Asynchronous;
 * per-cell outcomes are read with chem_get_stats (a failed cell keeps its
 * input state).  Errors: CHEM_EINVAL, CHEM_ESTATE (before set_state),
 * CHEM_ECUDA; nothing is launched on error. */
int chem_solve_step(chem_cells *cells, double dt, void *stream);
/* n_steps consecutive chem_solve_step calls of dt (1..CHEM_MAX_GRAPH_STEPS) as
 * one CUDA graph launch on stream: the per-step queue resets and solve
 * kernels are captured once, on an internal stream, and the graph is re-used
 * while n_steps, dt, the launch shape and the photolysis/theta sources
 * (per-cell or mechanism J, theta set or not) stay the same; any change
 * re-captures it.  The inputs it reads (T, P, y, J, theta) are the batch's
 * own buffers, so set_state / set_photolysis / set_theta between launches
 * take effect.  Results are identical to n_steps chem_solve_step calls.
 * Asynchronous.  Errors: CHEM_EINVAL, CHEM_ESTATE, CHEM_ECUDA. */
int chem_solve_steps(chem_cells *cells, double dt, int32_t n_steps, void *stream);
/* Choose the launch shape of the batch by measurement: every cells-per-block
 * w the shared memory allows and, for the persistent driver, every resident
 * block count 1..occupancy(w) is timed (CUDA events, best of two) on a scratch
 * copy of the first n_sample cells (0: min(n_cells, CHEM_AUTOTUNE_SAMPLE))
 * integrated over dt; the fastest shape becomes the batch's cells_per_block /
 * blocks_per_sm and is written to the outputs (each may be NULL).  The
 * batch's state is not touched.  Needs set_state.  Allocates scratch and
 * synchronises.  Errors: CHEM_EINVAL, CHEM_ESTATE, CHEM_ENOMEM, CHEM_ECUDA. */
int chem_autotune(chem_cells *cells, double dt, int64_t n_sample, int32_t *cells_per_block,
                  int32_t *blocks_per_sm);

/* Copy the state y[n_species][n_cells] (mol/mol, cell index unit stride) into
 * the caller's y (synchronises stream when mem is CHEM_MEM_HOST).  Paper,
 * Background section: the updated concentrations the chemistry step returns to
 * the model.  Errors: CHEM_EINVAL, CHEM_ECUDA. */
int chem_get_state(const chem_cells *cells, double *y, int32_t mem, void *stream);
/* Copy the per-cell statistics of the last solve (out[n_cells]); synchronises
 * stream when mem is CHEM_MEM_HOST.  The counters are those the paper's
 * Results section compares between its One-cell and Multi-cells forms
 * (solver iterations).  Errors: CHEM_EINVAL, CHEM_ECUDA. */
int chem_get_stats(const chem_cells *cells, chem_cell_stats *out, int32_t mem, void *stream);
/* Staging counters of the last chem_solve_step / chem_solve_steps call on the
 * batch (persistent driver; every step of a graph launch): *fallbacks = blocks
 * whose bulk copy of the tables into shared memory was not seen to land within
 * the bounded wait (they copied the tables with ordinary loads: same results);
 * *unfinished = blocks that exited before such a late copy was seen to land
 * within a second bounded wait.  Both are 0 in normal operation.  With
 * cells NULL: the counters of chem_solve_step_noalloc's last call on the
 * current device.  Reads on stream and synchronises it.  The paper has no
 * counterpart (it is a diagnostic of this library's table staging).  Errors:
 * CHEM_EINVAL, CHEM_ECUDA. */
int chem_staging_fallbacks(const chem_cells *cells, int64_t *fallbacks, int64_t *unfinished, void *stream);

/* Discrete adjoint (needs opts.record_adjoint).  Every solve_step since the
 * last set_state recorded, per cell, everything that determined its result:
 * the initial step, every history rescale, every accepted step with its order,
 * its corrector iteration count and its projections onto y >= 0, and every
 * refactorisation of the iteration matrix, with the states f and J were
 * evaluated at.  For L = sum_{i,c} dL_dy[i][c] * y[i][c] (y the current state)
 * this returns dL_dtheta[n_reactions] (theta: the log multipliers of
 * chem_cells_set_theta, shared by all cells; the sum over cells) and
 * dL_dy0[n_species][n_cells] (the state at set_state).  It is the exact
 * adjoint of the computation the solve made, with its controls frozen: the
 * recorded step sizes, orders, iteration counts and projections, and the
 * iteration matrices M = I - c_M J(y_J) held constant (the paper's CVODE
 * BDF/Newton integration is the map being differentiated; the adjoint itself
 * has no counterpart in the paper).  One warp per cell walks its tape in
 * reverse through transposed sparse LU solves.  Inputs in `mem` space,
 * asynchronous copies on `stream`, then synchronises stream.  Returns 0, a
 * negative error, or the number of cells whose tape overflowed or whose
 * forward solve failed (their dL_dy0 is 0 and they add nothing to
 * dL_dtheta). */
int chem_sensitivity(chem_cells *cells, const double *dL_dy, double *dL_dtheta, double *dL_dy0, int32_t mem,
                     void *stream);
/* The same discrete adjoint over n_steps consecutive solve_step calls of dt,
 * by step checkpointing, for tapes that cannot hold all the steps at once:
 * states[n_steps][n_species][n_cells] holds the state at the start of each
 * step (states[0] the state at set_state, states[k] the result of step k-1),
 * kept by the caller during the forward.  Last step first, the library
 * re-solves step k from states[k] with a fresh tape (or, when last_recorded
 * is nonzero, uses the current tape for the last step: the caller's forward
 * recorded that step alone), runs the adjoint through it with
 * lambda = dL/d(result of step k), and carries the adjoint of its input to the
 * step before; dL_dtheta[n_reactions] receives the sum over steps and cells,
 * dL_dy0[n_species][n_cells] the adjoint of states[0].  The batch's T, P,
 * photolysis rates and theta must be those of the forward.  Afterwards the
 * batch holds the result of re-solving step 0 and its tape that step's.  The
 * paper has no counterpart (it differentiates the Background section's
 * BDF/Newton integration, step by step).  Inputs and outputs in `mem` space;
 * synchronises stream.  Returns 0, a negative error (CHEM_EINVAL, CHEM_ESTATE,
 * CHEM_ECUDA), or the number of (cell, step) pairs whose tape overflowed or
 * whose re-solve failed: those cells' gradients are then incomplete. */
int chem_sensitivity_checkpointed(chem_cells *cells, const double *states, int32_t n_steps, double dt,
                                  int32_t last_recorded, const double *dL_dy, double *dL_dtheta, double *dL_dy0,
                                  int32_t mem, void *stream);
/* Tangent (forward-mode) sensitivity of the same frozen-control map
 * (needs opts.record_adjoint): the directional derivative
 *   dy[n_species][n_cells] = (d y / d y0) dy0 + (d y / d theta) dtheta
 * of the current state along dy0[n_species][n_cells] (a direction in the state
 * at set_state) and dtheta[n_reactions] (a direction in the log multipliers,
 * shared by all cells; NULL = 0).  Its dot product with any dL_dy equals
 * <dL_dy0, dy0> + <dL_dtheta, dtheta> from chem_sensitivity, up to rounding.
 * One warp per cell walks its tape forward: each corrector iteration applies
 * the f program to the tangent rates k~_j sum_s (prod_{s' != s} y) v_s +
 * r_j dtheta_j (that is J v + F_theta dtheta) and one sparse LU solve with the
 * recorded iteration matrix.  The paper has no tangent; it differentiates the
 * paper's BDF/Newton integration.  Inputs and output in `mem` space,
 * asynchronous copies on `stream`, then synchronises stream.  It stages its
 * input and output in the batch's adjoint buffers, so it must not overlap a
 * chem_sensitivity call on the same batch.  Returns 0, a negative error, or
 * the number of cells whose tape overflowed or whose forward solve failed
 * (their dy is 0).  Errors: CHEM_EINVAL, CHEM_ESTATE (no recording, no
 * state), CHEM_ECUDA. */
int chem_tangent(chem_cells *cells, const double *dy0, const double *dtheta, double *dy, int32_t mem, void *stream);
/* The recorded tape of one cell, in host arrays of `capacity` events: kind
 * 0 = INIT (val h0), 1 = RESCALE (q order, val eta), 2 = STEP (q order, val
 * c = h/gamma_q), 3 = PROJECT (q the species the next STEP projects onto 0),
 * 4 = REFACTOR (q its row, val c_M), 5 = ITER (q the iteration of the next
 * STEP).  INIT, REFACTOR and ITER events own one row each, in event order:
 * the state at the start of the solve, y_J, and the iterate f was evaluated
 * at; rows (may be NULL) receives them, [n_rows][n_species].  *n_events and
 * *n_rows receive the lengths; nothing else is copied if capacity < n_events
 * (rows must hold n_rows rows).  Synchronous.  Errors: CHEM_EINVAL,
 * CHEM_ESTATE (no recording), CHEM_ECUDA. */
int chem_get_tape(const chem_cells *cells, int64_t cell, int32_t *kind, int32_t *q, double *val, double *rows,
                  int32_t capacity, int32_t *n_events, int32_t *n_rows);

/* Designs of the derivative f(y) for chem_eval_deriv_design. */
#define CHEM_DERIV_GATHER 0       /* this library's: one warp per cell, the compiled f program, no atomics */
#define CHEM_DERIV_ATOMIC_AOS 1   /* the paper's: one thread per reaction and cell, FP64 atomic adds into f,
                                     reaction data as an array of structures */
#define CHEM_DERIV_ATOMIC_SOA 2   /* the same with the reaction data as a structure of arrays */

/* Derivative only, for comparing kernel designs (the paper's Implementations
 * section describes its GPU Derivative: a thread per reaction and cell adding
 * to f with atomic operations; it has no counterpart of the gather design).
 * f[n_species][n_cells] = f(y) for y[n_species][n_cells] (cell unit stride,
 * `mem` space) with the batch's rate constants k~[n_reactions][n_cells],
 * computed on the GPU on the first call after set_state, set_photolysis or
 * set_theta and kept in a buffer the batch allocates then (8 * n_reactions *
 * n_cells bytes).  The atomic designs sum in an unspecified order (results
 * agree to rounding); the gather design is deterministic.  Asynchronous for
 * device memory; synchronises for host memory.  Errors: CHEM_EINVAL (design,
 * NULL), CHEM_ESTATE (before set_state), CHEM_ENOMEM, CHEM_ECUDA. */
int chem_eval_deriv_design(chem_cells *cells, int32_t design, const double *y, double *f, int32_t mem, void *stream);

/* Diagnostics for kernel-level parity.  For every cell, with the cell's T, P,
 * photolysis rates and theta from the batch (set_state must have been
 * called), evaluate on the GPU with the same device routines the solve uses:
 *   chem_eval_deriv:        f = f(y)                          (step a2)
 *   chem_eval_newton_solve: x = (I - c J(y))^{-1} b           (steps a3-a5,
 *                           in the batch's LU precision)
 * y, b, f, x are [n_species][n_cells].  With CHEM_MEM_HOST the call allocates
 * device scratch, copies, and synchronises stream before returning. */
int chem_eval_deriv(chem_cells *cells, const double *y, double *f, int32_t mem, void *stream);
/* Diagnostic: out[i] = the FP64 reciprocal the solve kernels use (the
 * hardware estimate refined by one cubically convergent Newton-Raphson step,
 * r <- r (1 + e + e^2) with e = 1 - x r) of x[i], for i < n, on the current
 * device.  Defined for normal x with
 * 2^-1022 <= |x| <= 2^1022 (within 1 ulp of 1/x there); the estimate flushes
 * subnormal inputs and results to zero, so outside that range the result is
 * 0 or not finite.  No counterpart in the paper (the pivots of the LU and the
 * error weights 1/(rtol |y| + atol) use it).  With CHEM_MEM_HOST the call
 * allocates device scratch and synchronises stream.  Errors: CHEM_EINVAL,
 * CHEM_ENOMEM, CHEM_ECUDA. */
int chem_eval_reciprocal(const double *x, double *out, int64_t n, int32_t mem, void *stream);
/* Diagnostic: out[g] = the sum the solve kernels form of the 32 doubles
 * x[32 g .. 32 g + 31] (x: n_groups * 32 values, out: n_groups), one warp per
 * group, as they sum the squared weighted terms of the error norms: on the
 * integer pipe, exactly in fixed point relative to the group's largest term,
 * rounded once (within 1.5 ulp of the exact sum).  Defined for terms >= +0;
 * a group with an infinite, NaN or negative term, or with every term below
 * 2^-959, is summed by an FP64 butterfly instead.  No counterpart in the
 * paper (its error norm is the WRMS norm of the Background section's CVODE;
 * this is how the kernels reduce it).  With CHEM_MEM_HOST the call allocates
 * device scratch and synchronises stream.  Errors: CHEM_EINVAL, CHEM_ENOMEM,
 * CHEM_ECUDA. */
int chem_eval_warp_sum(const double *x, double *out, int64_t n_groups, int32_t mem, void *stream);
int chem_eval_newton_solve(chem_cells *cells, double c, const double *y, const double *b, double *x,
                           int32_t mem, void *stream);

/* Solve without any allocation by the library.
 *
 * For callers that must not allocate device memory once they are running: a
 * host model under its own memory manager or a fixed device-memory budget,
 * or a time loop that must never grow the device footprint after start-up.
 * Create the mechanism at start-up (that allocates), then call this entry
 * point with caller-owned DEVICE buffers: T[n_cells], P[n_cells],
 * y[n_species][n_cells] (integrated in place over [0, dt], as
 * chem_solve_step does), stats[n_cells] (written), and optionally
 * J[n_photolysis][n_cells] and theta[n_reactions] (NULL: mechanism J,
 * theta = 0).  Every buffer must be memory of the current device (or
 * managed memory), which must be the mechanism's device; anything else
 * (host memory included) is refused with CHEM_EINVAL before any launch.
 * opts NULL = defaults; the driver is always the persistent work queue, in
 * cell index order; couple_cells > 1 and record_adjoint are refused (both need
 * buffers a batch allocates).  Results equal those of chem_solve_step on a
 * persistent batch with the same inputs and options, bit for bit.  The paper
 * has no counterpart of this entry point.
 *
 * The work-queue counter and the two staging counters (chem_staging_fallbacks
 * with cells NULL reads them) live in a 256-byte static device array inside
 * the library (held by every GPU that loads the library until the process
 * exits); the call clears them on stream before the launch and calls no
 * cudaMalloc/cudaFree.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  All calls on a device share its one array: calls whose
 * work overlaps on that GPU (e.g. launched on two streams) race and must be
 * serialised by the caller.  n_cells beyond CHEM_NOALLOC_MAX_CELLS is
 * rejected with CHEM_EINVAL. */
#define CHEM_NOALLOC_MAX_CELLS 2147483647LL
int chem_solve_step_noalloc(const chem_mech *mech, int64_t n_cells, const double *T, const double *P,
                            const double *J, const double *theta, double *y, chem_cell_stats *stats,
                            double dt, const chem_opts *opts, void *stream);

/*
 * Host-resident state with the chemistry on the GPU, overlapped chunk by
 * chunk.  The paper found that moving the state between host and device
 * every call took about 90% of its GPU time and named overlapping CPU and GPU
 * work with asynchronous transfers as future work (Results and Conclusions
 * sections); this is that overlap for a host model that owns y.  The
 * n_cells cells are split into n_chunks contiguous chunks (sizes differ by at
 * most one, larger first), each with its own device batch (created with
 * opts, which must not ask for record_adjoint or couple_cells) and its own
 * non-blocking stream.  Allocates the batches, streams and events.
 * Errors: CHEM_EINVAL, CHEM_ENOMEM, CHEM_ECUDA.
 */
typedef struct chem_pipeline chem_pipeline;
int chem_pipeline_create(const chem_mech *mech, int64_t n_cells, int32_t n_chunks, const chem_opts *opts,
                         chem_pipeline **out);
void chem_pipeline_destroy(chem_pipeline *p);   /* NULL is a no-op */
/* Called on the thread of chem_pipeline_run once the solved state of cells
 * [c0, c1) for model step `step` is back in the host y.  It may update those
 * columns of y, T, P (and J) -- a transport, emission or deposition stand-in
 * of the host model -- and nothing else of them, while the GPU keeps solving
 * the other chunks.  Return 0 to go on, anything else to stop the run. */
typedef int (*chem_chunk_fn)(int64_t c0, int64_t c1, int32_t step, void *user);
/* n_steps model steps of length dt over host arrays T[n_cells], P[n_cells],
 * y[n_species][n_cells] (cell index unit stride; integrated in place) and
 * optionally J[n_photolysis][n_cells] (NULL: the mechanism's J).  Per chunk
 * and step, on the chunk's stream: T, P, (J,) y columns host -> device (2-D
 * strided copies), the solve, y back device -> host; then, on this thread,
 * fn(c0, c1, step, user) (fn may be NULL), after which that chunk's next step
 * is queued at once, so host work on one chunk overlaps the GPU's work on the
 * others and the copies overlap the solves.  Results equal those of n_steps
 * chem_solve_step calls on one batch with fn applied between them, bit for
 * bit.  The host arrays should be page-locked (cudaHostRegister or a pinned
 * allocation) for the copies to run asynchronously.  stats (may be NULL)
 * receives the statistics of the last step, [n_cells].  Synchronous: returns
 * when every chunk's last step is back and its callback has returned.
 * Returns 0 or a negative error: CHEM_EINVAL, CHEM_ECUDA, CHEM_EABORTED (fn
 * returned nonzero; work already queued is drained first). */
int chem_pipeline_run(chem_pipeline *p, const double *T, const double *P, const double *J, double *y, double dt,
                      int32_t n_steps, chem_chunk_fn fn, void *user, chem_cell_stats *stats);

/* Measured FMA throughput of the CUDA cores in TFLOP/s (precision 64: FP64,
 * 32: FP32), the denominator the solve kernels' arithmetic rooflines are
 * measured against: every thread of a grid that fills all SMs runs 8
 * independent chains of x <- x a + b; *tflops = 2 x chains x iterations x
 * threads / time of one launch (CUDA events on stream, calibrated to about
 * 50 ms, best of three), *ms that time.  No counterpart in the paper.
 * Synchronous.  Errors: CHEM_EINVAL, CHEM_ECUDA. */
int chem_measure_fma_peak(int32_t precision, double *tflops, double *ms, void *stream);

/* Thread-local description of the last error ("" if none). */
const char *chem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
