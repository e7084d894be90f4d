// internal.h -- data structures shared by the mechanism compiler (host) and the
// solve kernels (device).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "chemgpu.h"

namespace chemgpu {

constexpr int QMAX = 5;             // highest BDF order
constexpr int NROW = QMAX + 3;      // history rows D_0 .. D_{QMAX+2}
constexpr int GRID_IMIN = -26;      // step-factor grid g_i = 2^(i/8)
constexpr int GRID_IMAX = 26;
constexpr int GRID_N = GRID_IMAX - GRID_IMIN + 1;
constexpr int WARP = 32;
constexpr int MAX_WARPS_PER_BLOCK = 12;  // cells per block (history and vectors live in registers)
constexpr int ADJ_WARPS_PER_BLOCK = 12;  // most cells per block of the adjoint walk
constexpr int TAN_WARPS_PER_BLOCK = 4;   // ... and of the tangent walk (a larger launch bound costs it
                                         // registers and 70% more instructions)

// A warp program is a sequence of passes of exactly 32 op slots; lane l runs
// slot l of every pass and the warp synchronises between passes.  The
// scheduler guarantees that no location written in a pass is read or written
// by another op of the same pass, so the passes run without intra-pass races.
// On the host an op holds element indices:
//   FMA op:    W[t] = fma(W[a], W[b], W[c])      (NEG program: fma(-W[a], W[b], W[c]))
//   RECIP op:  W[t & 0x7fff] = -1 / W[a]         (t has bit 15 set)
//   empty:     t == 0xffff
// On the device the same op holds BYTE offsets into the cell's work array,
// empty slots become a harmless FMA into a dummy slot, and a RECIP op (or an
// empty slot of a pass with reciprocals) carries c == 0xffff.  A pass with
// reciprocals may hold FMA ops in its other lanes (the interpreter runs such a
// pass as one mixed op per lane).
struct Op {
  uint16_t t, a, b, c;
};
constexpr uint16_t OP_EMPTY = 0xffff;
constexpr uint16_t OP_RECIP = 0x8000;
constexpr uint16_t DEV_RECIP = 0xffff;     // device marker in .w of RECIP passes

// Tables read by every warp of every cell, packed into one 16-byte-aligned
// blob per LU precision so that a block can stage them into shared memory
// with one bulk copy.  Byte offsets of each section within the blob:
struct TableOffsets {
  int f_ops, fwd_ops, bwd_ops;     // ushort4 programs (f on Wd, fwd/bwd on WL)
  int f_runs;                      // uint32 run table of the f program
  int rx_slots;                    // uint2 [R]: byte offsets into Wd of the reactants' y
  int pair_rx;                     // int [n_pairs]
  int pair_other;                  // uint32 [n_pairs]: two 16-bit byte offsets into Wd
  int lu_diag;                     // int [S]: byte offsets into WL of the pivot diagonal
  int dconst_off, dconst_val;      // int [d_nconst] byte offsets into Wd, double values
  int Lconst_off, Lconst_val;      // int [L_nconst] byte offsets into WL, double values
  int thr2, thr3, g;               // step-factor grid: thresholds of the raw squared-norm sums
                                   // (biases 2 and 3), double [7][GRID_N] each, and the factors
                                   // g_i, [GRID_N]
  int lim;                         // double [2][8]: by order q, the raw-sum bounds of the error
                                   // test, S (q+1)^2, and of the corrector, S (0.1 (q+1))^2
  int staged;                      // bytes of the prefix the persistent driver stages in shared
                                   // memory (programs and slots used every Newton iteration or
                                   // refactorisation; constants and the grid stay in global memory)
  int bytes;                       // total, a multiple of 16
};

constexpr int RX_EXT = 8;   // extra rate parameters per reaction

// Everything a solve kernel needs about a mechanism; passed by value.
struct MechDev {
  int S, R, max_reac, n_phot, n_pairs;
  // rate constants (read once per cell)
  const int *rx_kind;      // [R]
  const int *rx_nreac;     // [R]
  const int *rx_phot;      // [R] index among photolysis reactions, or -1
  const double *rx_A, *rx_Ea, *rx_B, *rx_J;
  const double *rx_ext;    // [R][RX_EXT]: A2, Ea2, B2, A3, Ea3, B3, Fc, N (pressure-dependent kinds)
  // reaction data for the derivative-design comparison (chem_eval_deriv_design):
  // the caller's records as uploaded (array of structures), and the same as
  // structure of arrays: reactants [R][3], product counts [R], products and yields [R][8]
  const chem_reaction *rx_aos;
  const int *rx_reac, *rx_nprod, *rx_prod;
  const double *rx_yld;
  // species permutation: position of species s in the pivot order
  const int *sp_pos;       // [S]
  // per-cell double array Wd (element indices)
  int Wd_len, d_Y, d_KT, d_RT, d_F, d_ONE, d_ZERO, d_DUMMY;
  // per-cell LU-precision array WL (element indices)
  int WL_len, L_LU, L_X, L_P, L_ZERO, L_DUMMY, nnz_lu;
  int d_nconst, L_nconst;
  int m_clear;             // WL entries [0, m_clear) are cleared before forming M
  int f_npass, fwd_npass, bwd_npass, m_npass, lu_npass;
  int f_nruns, m_nruns, lu_nruns;  // run tables (f: in the staged blob; M, LU: m_runs, lu_runs)
  const uint32_t *m_runs, *lu_runs;
  // staged tables: blob[0] for an FP64 LU, blob[1] for an FP32 LU (global memory)
  const unsigned char *blob[2];
  TableOffsets tab;
  // programs streamed from global memory, per LU precision (byte-offset ops)
  const ushort4 *m_ops[2], *lu_ops[2];
  // history rescale T(eta)_{im} = sum_p coef[(i-1)*QMAX + m-1][p] eta^p,
  // i, m = 1..QMAX, p = 0..QMAX
  const double *rescale_coef;
  // ---- discrete adjoint (FP64): after the forward's Wd and WL, mu[S], nm[R] =
  // nu_j . mu, jtm[S] = J^T mu, g[R] (theta gradient), temps, constants (up to
  // Wda_len), then pp[n_pairs] = dr_j/dy_l at a_PP; indices from the start of Wd
  int Wda_len, a_MU, a_NM, a_PP, a_JTM, a_G;
  int a_nconst;
  const int *a_const_off;          // byte offsets into the extended Wd
  const double *a_const_val;
  const ushort4 *nudot_ops, *jt_ops;    // programs on the extended Wd
  const ushort4 *fwdT_ops, *bwdT_ops;   // U^T and L^T solves on WL (FP64 byte offsets)
  int nudot_npass, jt_npass, fwdT_npass, bwdT_npass;
  const uint32_t *nudot_runs, *jt_runs, *fwdT_runs, *bwdT_runs;   // their run tables
  int nudot_nruns, jt_nruns, fwdT_nruns, bwdT_nruns;
};

// Kinds of the units a program's passes form, in its run table (one uint32 per
// run of equal units: kind << 28 | units): a single pass of FMAs, a pair of
// consecutive FMA passes whose 64 ops are independent of each other (the
// interpreter loads the operands of both before it stores either result, so a
// lane has two FMAs in flight between warp synchronisations), a pass of
// reciprocals (and FMAs in the lanes the reciprocals leave).
constexpr uint32_t RUN_FMA1 = 0, RUN_FMA2 = 1, RUN_RECIP = 2;

struct HostProgram {
  std::vector<Op> ops;   // n_pass * 32
  std::vector<uint8_t> unit;   // per pass: 0 single FMA pass, 1 / 2 first / second pass of a pair, 3 reciprocals
  int n_ops = 0;
  int n_pass() const { return (int)(ops.size() / WARP); }
  std::vector<uint32_t> runs() const {
    std::vector<uint32_t> r;
    uint32_t kind = 0xf, n = 0;
    for (size_t p = 0; p < unit.size(); ++p) {
      if (unit[p] == 2) continue;
      const uint32_t k = unit[p] == 1 ? RUN_FMA2 : unit[p] == 3 ? RUN_RECIP : RUN_FMA1;
      if (k != kind && n) r.push_back(kind << 28 | n), n = 0;
      kind = k;
      n++;
    }
    if (n) r.push_back(kind << 28 | n);
    return r;
  }
};

// Compiled mechanism (host + device copies).
struct Mechanism {
  int S = 0, R = 0, n_phot = 0, max_reac = 0, n_pairs = 0, nnz_jac = 0, nnz_lu = 0;
  std::vector<int> pos;              // pivot position of each species
  std::vector<uint8_t> fill;         // S*S in pivot order
  HostProgram f_prog, m_prog, lu_prog, fwd_prog, bwd_prog;
  HostProgram nudot_prog, jt_prog, fwdT_prog, bwdT_prog;   // adjoint
  std::vector<double> a_consts_v;
  std::vector<int> a_consts_i;
  double flops_f = 0, flops_jac = 0, flops_lu = 0, flops_solve = 0;
  double flops_adj_iter = 0, flops_tan_iter = 0;   // per corrector iteration of the adjoint / tangent walks
  // host copies of the small tables that upload_mechanism() sends to the device
  std::vector<double> d_consts_v, L_consts_v;
  std::vector<int> d_consts_i, L_consts_i;
  std::vector<int> pair_rx;
  std::vector<std::pair<int, int>> pair_other;   // Wd element indices
  std::vector<int> lu_diag;                      // WL element indices
  std::vector<int> rx_slot_idx;                  // [R][3] Wd element indices of the reactants' y
  std::vector<chem_reaction> rx;
  MechDev dev{};                     // device pointers filled in upload()
  std::vector<void *> allocations;   // device buffers owned
  int device = 0;
};

// Build the mechanism tables (host).  Returns 0 or a CHEM_E* code with msg.
int compile_mechanism(int S, int R, const chem_reaction *rx, Mechanism &m, std::string &msg);
int upload_mechanism(Mechanism &m, std::string &msg);
void free_mechanism(Mechanism &m);

// Launch the solve kernel for all cells (device side in kernels.cu).
struct CellsDev {
  int64_t n_cells;
  const double *T, *P, *J;      // J may be null (mechanism J)
  const double *theta;          // may be null
  double *y;                    // [S][C] in/out
  chem_cell_stats *stats;       // [C]
  unsigned long long *queue;    // persistent driver work counter (may be null)
  const int *order;             // persistent driver: the queue hands out order[0], order[1], ...;
                                // adjoint / tangent: warp slot i takes cell order[i] (NULL: cell i)
                                // (null: cell index order)
  // staging counters (may be null): [0] blocks whose bulk copy of the tables
  // was not seen to land within the first bounded wait (they read the tables
  // from global memory instead), [1] blocks that exited before seeing that
  // late copy land within the final bounded wait
  unsigned long long *stage;
  // adjoint tape (tape_n null: not recording).  Per cell e < tape_cap events,
  // kq = kind | q << 8, val:
  //   0 INIT      val h0,   row y at the start of the solve
  //   1 RESCALE   q order,  val eta
  //   2 STEP      q order,  val c = h/gamma_q (accepted step)
  //   3 PROJECT   q species projected onto y = 0 by the next STEP
  //   4 REFACTOR  q its row index, val c_M; row y_J (M = I - c_M J(y_J))
  //   5 ITER      q iteration k of the next STEP; row y_k, the iterate it
  //               evaluated f at
  // Rows are numbered in event order over the INIT, REFACTOR and ITER events.
  int *tape_kq;
  double *tape_val;
  double *ytape;                // [C][row_cap][S] rows
  int *tape_n;                  // [C] events so far (kept across solve_step calls)
  int *tape_bad;                // [C] nonzero: overflow or a failed solve, no sensitivity
  int *tape_rows;               // [C] rows so far
  int tape_cap, row_cap;
};

enum TapeKind { EV_INIT = 0, EV_RESCALE = 1, EV_STEP = 2, EV_PROJECT = 3, EV_REFACTOR = 4, EV_ITER = 5 };

// Buffers of chem_sensitivity (device, owned by the batch).
struct AdjDev {
  const double *dLdy;           // [S][C]
  double *dLdy0;                // [S][C]
  double *gcell;                // [R][C] per-cell theta gradients
  double *dLdtheta;             // [R]
  int accumulate;               // 0: dLdtheta = the sum over cells; 1: dLdtheta += that sum
};

// Buffers of chem_tangent (device, owned by the batch).
struct TanDev {
  const double *dy0;            // [S][C] direction in the initial state
  const double *dtheta;         // [R] direction in theta (shared by all cells)
  double *dy;                   // [S][C] out: the directional derivative of the state
};

// Iterations of the bounded wait for a block's bulk copy of the tables.
constexpr long long STAGE_WAIT_DEFAULT = 1LL << 22;

struct LaunchCfg {
  int lu_precision;     // 64 / 32
  int driver;           // CHEM_DRIVER_*
  int couple;           // > 1: cells integrated in coupled groups of this many (one block each)
  int warps_per_block;
  int blocks_per_sm;
  double rtol, atol, dt;
  int max_order, max_steps;
  long long stage_wait; // iterations of the first wait for the staged tables (chem_opts.stage_wait)
};

size_t smem_per_cell(const MechDev &m, int lu_precision);
size_t staged_bytes(const MechDev &m, int driver);   // tables staged per block by the driver
cudaError_t set_constants();   // gamma_m, 1/gamma_m into constant memory of the current device
cudaError_t launch_solve(const MechDev &m, const CellsDev &c, const LaunchCfg &cfg, cudaStream_t stream);
// Cells most expensive first for the persistent queue: per cell its cost in
// the batch's previous solve, or for a first solve the sum of its rate
// constants, bucketed linearly in log2 over the batch's range, then a counting
// sort into order[n_cells].  bucket[n_cells] and hist[ORDER_HIST_INTS] are
// scratch.  Stream-ordered (capturable).
constexpr int ORDER_BUCKETS = 256;
constexpr int ORDER_HIST_INTS = 2 * ORDER_BUCKETS + 2;   // counts, cursors, key range
// The same counting sort keyed by tape length (events), longest first: the
// order in which the adjoint and tangent kernels take the cells.
cudaError_t launch_order_tape(const CellsDev &c, int *bucket, int *hist, int *order, cudaStream_t stream);
// ... and keyed by the cost of coupled groups of G cells: order[i] is a group index.
cudaError_t launch_order_groups(const CellsDev &c, int G, int *bucket, int *hist, int *order, cudaStream_t stream);
cudaError_t launch_order(const MechDev &m, const CellsDev &c, double rtol, double atol, int *bucket, int *hist,
                         int *order, cudaStream_t stream);
int max_warps_per_block(const MechDev &m, int lu_precision, int driver);
// resident blocks per SM of the solve kernel for a block of warps_per_block cells
int occupancy(const MechDev &m, int lu_precision, int driver, int warps_per_block);
// cells per block that maximises resident cells per SM (0 if nothing fits)
int best_warps_per_block(const MechDev &m, int lu_precision, int driver);
// diagnostic: mode 0 out = f(y); mode 1 out = (I - c J(y))^{-1} b   (all [S][C] device arrays)
cudaError_t launch_probe(const MechDev &M, const CellsDev &C, int lu_precision, int mode, double c, const double *y,
                         const double *b, double *out, cudaStream_t stream);

// discrete adjoint: replay (exact steps, y rows), backward sweep, theta reduction
cudaError_t launch_adjoint(const MechDev &m, const CellsDev &c, const AdjDev &a, cudaStream_t stream);
cudaError_t launch_tangent(const MechDev &m, const CellsDev &c, const TanDev &t, cudaStream_t stream);
// diagnostic: out[i] = the solve kernels' FP64 reciprocal of x[i] (device arrays)
cudaError_t launch_recip_probe(const double *x, double *out, int64_t n, cudaStream_t stream);
// diagnostic: out[g] = the solve kernels' warp sum of x[32 g .. 32 g + 31] (device arrays)
cudaError_t launch_wsum_probe(const double *x, double *out, int64_t n_groups, cudaStream_t stream);
// *acc += the number of nonzero flags among flag[0..n)
cudaError_t launch_count_flags(const int *flag, int64_t n, unsigned long long *acc, cudaStream_t stream);
// deriv.cu: derivative-only kernels for comparing designs.  kt[R][C] rate
// constants of the batch (launch_rates fills it); y, f [S][C] on the device.
cudaError_t launch_rates(const MechDev &m, const CellsDev &c, double *kt, cudaStream_t stream);
cudaError_t launch_deriv_design(const MechDev &m, const CellsDev &c, int design, const double *kt, const double *y,
                                double *f, cudaStream_t stream);
// kernels.cu: the gather design (one warp per cell, the compiled f program)
cudaError_t launch_deriv_gather(const MechDev &m, const CellsDev &c, const double *kt, const double *y, double *f,
                                cudaStream_t stream);

// sets the thread-local message returned by chem_last_error()
void set_last_error(const std::string &msg);

// noalloc.cu: the staging counters of chem_solve_step_noalloc's last call on
// the current device (read on stream, which is then synchronised); a CHEM_*
// return code
int noalloc_stage_counts(int64_t *fallbacks, int64_t *unfinished, cudaStream_t stream);

}  // namespace chemgpu

// opaque handle of include/chemgpu.h
struct chem_mech {
  chemgpu::Mechanism m;
};
