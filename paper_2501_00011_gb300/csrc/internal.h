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
constexpr int MAX_WARPS_PER_BLOCK = 8;   // cells per block (history and vectors live in registers)

// A warp program is a sequence of passes of exactly 32 op slots; lane l runs
// slot l of every pass and the warp synchronises between passes.  The
// scheduler guarantees that no location written in a pass is read or written
// by another op of the same pass, so the passes run without intra-pass races.
//   FMA op:    W[t] = fma(W[a], W[b], W[c])      (NEG program: fma(-W[a], W[b], W[c]))
//   RECIP op:  W[t & 0x7fff] = -1 / W[a]         (t has bit 15 set)
//   empty:     t == 0xffff
struct Op {
  uint16_t t, a, b, c;
};
constexpr uint16_t OP_EMPTY = 0xffff;
constexpr uint16_t OP_RECIP = 0x8000;

struct ProgramDev {
  const ushort4 *ops;   // n_pass * 32 entries
  int n_pass;
};

// Everything a solve kernel needs about a mechanism; passed by value.
struct MechDev {
  int S, R, max_reac, n_phot, n_pairs;
  // rate constants
  const int *rx_kind;      // [R]
  const int *rx_nreac;     // [R]
  const int *rx_phot;      // [R] index among photolysis reactions, or -1
  const double *rx_A, *rx_Ea, *rx_B, *rx_J;
  // f(y): reactant slots per reaction in Wd index space (missing -> Wd ONE)
  const ushort4 *rx_slots; // [R] x=reac0 y=reac1 z=reac2 (Wd indices of y)
  // Jacobian partials: one per (reaction, reactant slot)
  const int *pair_rx;      // [n_pairs]
  const ushort2 *pair_other;   // [n_pairs] Wd indices of the other reactants' y (ONE if none)
  // species permutation: position of species s in the pivot order
  const int *sp_pos;       // [S]
  // per-cell double array Wd
  int Wd_len, d_Y, d_KT, d_RT, d_F, d_ONE, d_ZERO;
  // per-cell LU-precision array WL
  int WL_len, L_LU, L_NINV, L_X, L_P, L_ZERO, nnz_lu;
  const int *lu_diag;      // [S] WL index of the pivot-order diagonal entries
  // constant slots to initialise in each cell's arrays
  const double *d_const_val; const int *d_const_idx; int d_nconst;
  const double *L_const_val; const int *L_const_idx; int L_nconst;
  // LU slots that are diagonal entries of M (set to 1 before the J terms)
  // and the number of WL entries to clear before forming M ([0, m_clear))
  int m_clear;
  ProgramDev f_prog, m_prog, lu_prog, fwd_prog, bwd_prog;
  // step-factor grid: thr[p][i] for bias 2 (p = 0..6) and bias 3, and g[i]
  const double *grid_thr2, *grid_thr3, *grid_g;
  // history rescale T(eta)_{im} = sum_p coef[(i-1)*QMAX + m-1][p] eta^p,
  // i, m = 1..QMAX, p = 0..QMAX
  const double *rescale_coef;
};

struct HostProgram {
  std::vector<Op> ops;   // n_pass * 32
  int n_ops = 0;
  int n_pass() const { return (int)(ops.size() / WARP); }
};

// Compiled mechanism (host + device copies).
struct Mechanism {
  int S = 0, R = 0, n_phot = 0, max_reac = 0, n_pairs = 0, nnz_jac = 0, nnz_lu = 0;
  std::vector<int> pos;              // pivot position of each species
  std::vector<uint8_t> fill;         // S*S in pivot order
  HostProgram f_prog, m_prog, lu_prog, fwd_prog, bwd_prog;
  double flops_f = 0, flops_jac = 0, flops_lu = 0, flops_solve = 0;
  // host copies of the small tables that upload_mechanism() sends to the device
  std::vector<double> d_consts_v, L_consts_v;
  std::vector<int> d_consts_i, L_consts_i;
  std::vector<int> pair_rx;
  std::vector<std::pair<int, int>> pair_other;
  std::vector<int> lu_diag;
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
  int *queue;                   // persistent driver work counter (may be null)
};

struct LaunchCfg {
  int lu_precision;     // 64 / 32
  int driver;           // CHEM_DRIVER_*
  int warps_per_block;
  int blocks_per_sm;
  double rtol, atol, dt;
  int max_order, max_steps;
};

size_t smem_per_cell(const MechDev &m, int lu_precision);
cudaError_t set_constants();   // gamma_m, 1/gamma_m into constant memory of the current device
cudaError_t launch_solve(const MechDev &m, const CellsDev &c, const LaunchCfg &cfg, cudaStream_t stream);
int max_warps_per_block(const MechDev &m, int lu_precision);
// resident blocks per SM of the solve kernel for a block of warps_per_block cells
int occupancy(const MechDev &m, int lu_precision, int warps_per_block);
// diagnostic: mode 0 out = f(y); mode 1 out = (I - c J(y))^{-1} b   (all [S][C] device arrays)
cudaError_t launch_probe(const MechDev &M, const CellsDev &C, int lu_precision, int mode, double c, const double *y,
                         const double *b, double *out, cudaStream_t stream);

// sets the thread-local message returned by chem_last_error()
void set_last_error(const std::string &msg);

}  // namespace chemgpu

// opaque handle of include/chemgpu.h
struct chem_mech {
  chemgpu::Mechanism m;
};
