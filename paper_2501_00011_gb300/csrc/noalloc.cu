// noalloc.cu -- chem_solve_step_noalloc: the persistent solve on caller-owned
// device buffers, with no allocation by the library.
//
// Who needs it: code that integrates chemistry from inside a context where it
// must not allocate device memory -- a host model running under its own
// memory manager or a fixed memory budget, code that only hands out
// pre-registered device buffers, or a time loop that must never grow the
// device footprint after start-up.  Such callers create the mechanism once at
// start-up and then call this entry point with their own T, P, y and stats
// buffers; the call allocates nothing.
//
// The persistent driver needs one piece of scratch: the device work-queue
// counter that resident warps pop cell indices from.  Here it lives in the
// file-scope array below instead of in a chem_cells batch.  Every GPU that
// loads this library holds the array until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "internal.h"

namespace chemgpu {
namespace {

// Scratch: word 0 is the work-queue counter, word 1 counts blocks whose table
// staging fell back to plain loads; 256 bytes keep them alone in their line.
constexpr int NOALLOC_SCRATCH_WORDS = 32;
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_SCRATCH_WORDS];

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the symbol name is only a host-side stand-in, so the kernel must be
// given this address instead.
constexpr int MAX_DEVICES = 64;
void *g_scratch_addr[MAX_DEVICES] = {nullptr};

int fail(int code, const std::string &msg) {
  set_last_error(msg);
  return code;
}

}  // namespace
}  // namespace chemgpu

using namespace chemgpu;

extern "C" int chem_solve_step_noalloc(const chem_mech *mech, int64_t n_cells, const double *T, const double *P,
                                       const double *J, const double *theta, double *y,
                                       chem_cell_stats *stats, double dt, const chem_opts *opts, void *stream) {
  set_last_error("");
  if (!mech) return fail(CHEM_EINVAL, "mechanism is NULL");
  if (n_cells < 0 || n_cells > CHEM_NOALLOC_MAX_CELLS)
    return fail(CHEM_EINVAL, "n_cells must be in 0..CHEM_NOALLOC_MAX_CELLS (" +
                                 std::to_string((long long)CHEM_NOALLOC_MAX_CELLS) + ")");
  if (n_cells == 0) return 0;
  if (!T || !P || !y || !stats) return fail(CHEM_EINVAL, "T, P, y and stats must be device pointers");
  if (!(dt > 0.0) || !(dt < 1e300)) return fail(CHEM_EINVAL, "dt must be positive and finite");
  chem_opts o;
  if (opts) o = *opts; else chem_opts_default(&o);
  if (!(o.rtol > 0.0) || !(o.atol > 0.0)) return fail(CHEM_EINVAL, "rtol and atol must be > 0");
  if (o.max_order < 1 || o.max_order > QMAX) return fail(CHEM_EINVAL, "max_order must be 1..5");
  if (o.max_steps < 1) return fail(CHEM_EINVAL, "max_steps must be >= 1");
  if (o.lu_precision != 64 && o.lu_precision != 32) return fail(CHEM_EINVAL, "lu_precision must be 64 or 32");
  if (o.cells_per_block < 0 || o.cells_per_block > MAX_WARPS_PER_BLOCK || o.blocks_per_sm < 0)
    return fail(CHEM_EINVAL, "bad launch shape");
  if (o.couple_cells > 1) return fail(CHEM_EINVAL, "coupled cells are not supported here");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CHEM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(CHEM_EINVAL, "device ordinal beyond the supported range");
  if (!g_scratch_addr[dev]) {
    // first call on this device: look up the scratch's device address
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(CHEM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  const int wmax = max_warps_per_block(mech->m.dev, o.lu_precision, CHEM_DRIVER_PERSISTENT);
  if (wmax < 1) return fail(CHEM_EINVAL, "mechanism working set does not fit in shared memory");
  if (o.cells_per_block > wmax) return fail(CHEM_EINVAL, "cells_per_block exceeds the shared-memory limit");
  if (o.cells_per_block == 0) o.cells_per_block = best_warps_per_block(mech->m.dev, o.lu_precision, CHEM_DRIVER_PERSISTENT);
  if (o.cells_per_block < 1) return fail(CHEM_EINVAL, "no launch shape fits on this device");

  cudaStream_t s = (cudaStream_t)stream;
  // the counter must start at zero for every call
  e = cudaMemsetAsync(g_scratch_addr[dev], 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return fail(CHEM_ECUDA, std::string("scratch reset: ") + cudaGetErrorString(e));

  CellsDev cd{};
  cd.n_cells = n_cells;
  cd.T = T;
  cd.P = P;
  cd.J = J;
  cd.theta = theta;
  cd.y = y;
  cd.stats = stats;
  cd.queue = reinterpret_cast<int *>(g_scratch_addr[dev]);
  cd.error = reinterpret_cast<int *>(reinterpret_cast<unsigned long long *>(g_scratch_addr[dev]) + 1);
  LaunchCfg cfg{};
  cfg.lu_precision = o.lu_precision;
  cfg.driver = CHEM_DRIVER_PERSISTENT;
  cfg.warps_per_block = o.cells_per_block;
  cfg.blocks_per_sm = o.blocks_per_sm;
  cfg.rtol = o.rtol;
  cfg.atol = o.atol;
  cfg.dt = dt;
  cfg.max_order = o.max_order;
  cfg.max_steps = o.max_steps;
  e = launch_solve(mech->m.dev, cd, cfg, s);
  if (e != cudaSuccess) return fail(CHEM_ECUDA, std::string("solve kernel launch: ") + cudaGetErrorString(e));
  return 0;
}
