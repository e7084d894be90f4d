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
// The persistent driver needs a few words of scratch: the device work-queue
// counter that resident warps pop cell indices from, and the two staging
// counters.  Here they live in the file-scope array below instead of in a
// chem_cells batch.  Every GPU that loads this library holds the array until
// the process exits.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <mutex>
#include <string>

#include "devbuf.h"
#include "internal.h"

namespace chemgpu {
namespace {

// Scratch: word 0 is the work-queue counter, word 1 counts blocks whose table
// staging fell back to the global tables, word 2 blocks that exited before a
// late staging copy was seen to land; 256 bytes keep them alone in their lines.
constexpr int NOALLOC_SCRATCH_WORDS = 32;
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_SCRATCH_WORDS];

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the symbol name is only a host-side stand-in, so the kernel must be
// given this address instead.  Threads making their first call on a device
// at the same time serialise on the mutex; later calls read the atomic.
constexpr int MAX_DEVICES = 64;
std::atomic<void *> g_scratch_addr[MAX_DEVICES];
std::mutex g_scratch_mu;

int fail(int code, const std::string &msg) {
  set_last_error(msg);
  return code;
}

// The scratch address on the current device (looked up on the first call).
int scratch_address(int dev, unsigned long long **out) {
  void *p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    p = g_scratch_addr[dev].load(std::memory_order_relaxed);
    if (!p) {
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return fail(CHEM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev].store(p, std::memory_order_release);
    }
  }
  *out = static_cast<unsigned long long *>(p);
  return 0;
}

int current_device(int *dev) {
  const cudaError_t e = cudaGetDevice(dev);
  if (e != cudaSuccess) return fail(CHEM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (*dev < 0 || *dev >= MAX_DEVICES) return fail(CHEM_EINVAL, "device ordinal beyond the supported range");
  return 0;
}

// A caller's buffer must be memory of the current device (or managed memory).
int check_device_buffer(const void *p, int dev, const char *name) {
  const std::string why = device_buffer_problem(p, dev, name);
  return why.empty() ? 0 : fail(CHEM_EINVAL, why);
}

}  // namespace

int noalloc_stage_counts(int64_t *fallbacks, int64_t *unfinished, cudaStream_t stream) {
  int dev = 0;
  if (int rc = current_device(&dev)) return rc;
  unsigned long long *scratch = nullptr;
  if (int rc = scratch_address(dev, &scratch)) return rc;
  unsigned long long v[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(v, scratch + 1, sizeof(v), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail(CHEM_ECUDA, std::string("staging counters: ") + cudaGetErrorString(e));
  *fallbacks = (int64_t)v[0];
  *unfinished = (int64_t)v[1];
  return 0;
}

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
  if (o.record_adjoint) return fail(CHEM_EINVAL, "record_adjoint is not supported here (the tape is allocated by a batch)");
  if (o.stage_wait < -1) return fail(CHEM_EINVAL, "stage_wait must be -1, 0 or positive");

  int dev = 0;
  if (int rc = current_device(&dev)) return rc;
  if (dev != mech->m.device)
    return fail(CHEM_EINVAL, "the mechanism belongs to device " + std::to_string(mech->m.device) +
                                 ", which must be current");
  if (int rc = check_device_buffer(T, dev, "T")) return rc;
  if (int rc = check_device_buffer(P, dev, "P")) return rc;
  if (int rc = check_device_buffer(y, dev, "y")) return rc;
  if (int rc = check_device_buffer(stats, dev, "stats")) return rc;
  if (J && mech->m.n_phot > 0)
    if (int rc = check_device_buffer(J, dev, "J")) return rc;
  if (theta)
    if (int rc = check_device_buffer(theta, dev, "theta")) return rc;
  unsigned long long *scratch = nullptr;
  if (int rc = scratch_address(dev, &scratch)) return rc;

  const int wmax = max_warps_per_block(mech->m.dev, o.lu_precision, CHEM_DRIVER_PERSISTENT);
  if (wmax < 1) return fail(CHEM_EINVAL, "mechanism working set does not fit in shared memory");
  if (o.cells_per_block > wmax) return fail(CHEM_EINVAL, "cells_per_block exceeds the shared-memory limit");
  if (o.cells_per_block == 0) o.cells_per_block = best_warps_per_block(mech->m.dev, o.lu_precision, CHEM_DRIVER_PERSISTENT);
  if (o.cells_per_block < 1) return fail(CHEM_EINVAL, "no launch shape fits on this device");

  cudaStream_t s = (cudaStream_t)stream;
  // the queue counter and the staging counters start at zero for every call
  cudaError_t e = cudaMemsetAsync(scratch, 0, 3 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return fail(CHEM_ECUDA, std::string("scratch reset: ") + cudaGetErrorString(e));

  CellsDev cd{};
  cd.n_cells = n_cells;
  cd.T = T;
  cd.P = P;
  cd.J = mech->m.n_phot > 0 ? J : nullptr;
  cd.theta = theta;
  cd.y = y;
  cd.stats = stats;
  cd.queue = scratch;
  cd.stage = scratch + 1;
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
  cfg.stage_wait = o.stage_wait;
  e = launch_solve(mech->m.dev, cd, cfg, s);
  if (e != cudaSuccess) return fail(CHEM_ECUDA, std::string("solve kernel launch: ") + cudaGetErrorString(e));
  return 0;
}
