// capi.cpp -- the extern "C" entry points declared in include/chemgpu.h.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstring>
#include <initializer_list>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "devbuf.h"
#include "internal.h"

using namespace chemgpu;

struct chem_cells {
  const chem_mech *mech = nullptr;
  int64_t n = 0;
  chem_opts opts{};
  double *T = nullptr, *P = nullptr, *y = nullptr, *J = nullptr, *theta = nullptr;
  chem_cell_stats *stats = nullptr;
  // device counters: [0] persistent work queue, [1] staging fallbacks and
  // [2] unfinished staging copies of the last solve call (CellsDev::stage), [3] spare
  unsigned long long *counters = nullptr;
  int *order = nullptr, *order_bucket = nullptr, *order_hist = nullptr;   // persistent driver: queue order
  double *kt = nullptr;       // chem_eval_deriv_design: rate constants [R][C], allocated on first use
  bool kt_valid = false;      // ... and current for the batch's T, P, photolysis and theta
  bool have_state = false, use_J = false, use_theta = false;
  int device = 0;
  // adjoint (record_adjoint)
  int *tape_kq = nullptr, *tape_n = nullptr, *tape_bad = nullptr, *tape_rows = nullptr;
  double *tape_val = nullptr;
  int tape_cap = 0, row_cap = 0;
  // chem_solve_steps: the captured graph and what it was captured for
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0, graph_w = 0, graph_bps = 0;
  double graph_dt = 0.0;
  bool graph_J = false, graph_theta = false;
  double *ytape = nullptr, *gcell = nullptr, *dLdy = nullptr, *dLdy0 = nullptr, *dLdtheta = nullptr;
};

namespace {

thread_local std::string g_err;

// An NVTX range around an entry point, so profilers show the API calls on the
// host timeline (a no-op unless a tool is attached).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return CHEM_ECUDA;
}

cudaMemcpyKind kind_in(int32_t mem) { return mem == CHEM_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int32_t mem) { return mem == CHEM_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

int check_mem(int32_t mem) {
  if (mem != CHEM_MEM_HOST && mem != CHEM_MEM_DEVICE) return fail(CHEM_EINVAL, "mem must be CHEM_MEM_HOST or CHEM_MEM_DEVICE");
  return 0;
}

// With CHEM_MEM_DEVICE the caller's buffers go to the kernels and to
// device-side copies as they are: each one given (NULL entries are skipped)
// must be memory of the current device or managed memory.
int check_buffers(int32_t mem, std::initializer_list<std::pair<const void *, const char *>> bufs) {
  if (mem != CHEM_MEM_DEVICE) return 0;
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CHEM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  for (const auto &b : bufs) {
    if (!b.first) continue;
    const std::string why = device_buffer_problem(b.first, dev, b.second);
    if (!why.empty()) return fail(CHEM_EINVAL, why);
  }
  return 0;
}

// A batch lives on the device that was current when it was created (its
// buffers, and its mechanism's tables and the solver constants, are there):
// every call that touches it must be made with that device current.
int check_device(const chem_cells *c) {
  int dev = -1;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(CHEM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev != c->device)
    return fail(CHEM_EINVAL, "the batch belongs to device " + std::to_string(c->device) + " but device " +
                                 std::to_string(dev) + " is current");
  return 0;
}

}  // namespace

void chemgpu::set_last_error(const std::string &msg) { g_err = msg; }

extern "C" {

void chem_opts_default(chem_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->rtol = 1e-4;
  o->atol = 1e-10;
  o->max_order = 5;
  o->max_steps = 5000;
  o->lu_precision = 64;
  o->couple_cells = 1;
  o->driver = CHEM_DRIVER_PLAIN;
}

const char *chem_last_error(void) { return g_err.c_str(); }

int chem_mechanism_create(int32_t n_species, int32_t n_reactions, const chem_reaction *rx, chem_mech **out) {
  g_err.clear();
  if (!out) return fail(CHEM_EINVAL, "out is NULL");
  *out = nullptr;
  chem_mech *h = new (std::nothrow) chem_mech();
  if (!h) return fail(CHEM_ENOMEM, "host allocation failed");
  std::string msg;
  int rc = compile_mechanism(n_species, n_reactions, rx, h->m, msg);
  if (rc == 0) rc = upload_mechanism(h->m, msg);
  if (rc != 0) {
    delete h;
    return fail(rc, msg);
  }
  *out = h;
  return 0;
}

void chem_mechanism_destroy(chem_mech *h) {
  if (!h) return;
  free_mechanism(h->m);
  delete h;
}

int chem_mechanism_info(const chem_mech *h, chem_mech_info *o) {
  if (!h || !o) return fail(CHEM_EINVAL, "NULL argument");
  const Mechanism &m = h->m;
  std::memset(o, 0, sizeof(*o));
  o->n_species = m.S;
  o->n_reactions = m.R;
  o->n_photolysis = m.n_phot;
  o->nnz_jac = m.nnz_jac;
  o->nnz_lu = m.nnz_lu;
  o->n_pairs = m.n_pairs;
  o->passes_f = m.f_prog.n_pass();
  o->passes_jac = m.m_prog.n_pass();
  o->passes_lu = m.lu_prog.n_pass();
  o->passes_fwd = m.fwd_prog.n_pass();
  o->passes_bwd = m.bwd_prog.n_pass();
  o->ops_f = m.f_prog.n_ops;
  o->ops_jac = m.m_prog.n_ops;
  o->ops_lu = m.lu_prog.n_ops;
  o->ops_fwd = m.fwd_prog.n_ops;
  o->ops_bwd = m.bwd_prog.n_ops;
  o->flops_f = m.flops_f;
  o->flops_jac = m.flops_jac;
  o->flops_lu = m.flops_lu;
  o->flops_solve = m.flops_solve;
  o->smem_per_cell_fp64 = (int32_t)smem_per_cell(m.dev, 64);
  o->smem_per_cell_fp32 = (int32_t)smem_per_cell(m.dev, 32);
  o->flops_adj_iter = m.flops_adj_iter;
  o->flops_tan_iter = m.flops_tan_iter;
  return 0;
}

int chem_mechanism_structure(const chem_mech *h, int32_t *pos, uint8_t *fill) {
  if (!h || !pos) return fail(CHEM_EINVAL, "NULL argument");
  const Mechanism &m = h->m;
  for (int i = 0; i < m.S; ++i) pos[i] = m.pos[i];
  if (fill) std::memcpy(fill, m.fill.data(), m.fill.size());
  return 0;
}

int chem_cells_create(const chem_mech *mech, int64_t n_cells, const chem_opts *opts, chem_cells **out) {
  g_err.clear();
  if (!out) return fail(CHEM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mech) return fail(CHEM_EINVAL, "mechanism is NULL");
  if (n_cells < 0 || n_cells > ((int64_t)1 << 31)) return fail(CHEM_EINVAL, "n_cells must be in 0..2^31");
  {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != mech->m.device)
      return fail(CHEM_EINVAL, "the mechanism belongs to device " + std::to_string(mech->m.device) +
                                   ", which must be current when a batch is created");
  }
  chem_opts o;
  if (opts) o = *opts; else chem_opts_default(&o);
  if (!(o.rtol > 0.0) || !(o.atol > 0.0)) return fail(CHEM_EINVAL, "rtol and atol must be > 0");
  if (o.max_order < 1 || o.max_order > QMAX) return fail(CHEM_EINVAL, "max_order must be 1..5");
  if (o.max_steps < 1) return fail(CHEM_EINVAL, "max_steps must be >= 1");
  if (o.lu_precision != 64 && o.lu_precision != 32) return fail(CHEM_EINVAL, "lu_precision must be 64 or 32");
  if (o.driver != CHEM_DRIVER_PLAIN && o.driver != CHEM_DRIVER_PERSISTENT) return fail(CHEM_EINVAL, "bad driver");
  if (o.cells_per_block < 0 || o.cells_per_block > MAX_WARPS_PER_BLOCK || o.blocks_per_sm < 0) return fail(CHEM_EINVAL, "bad launch shape");
  if (o.couple_cells < 0 || o.couple_cells > MAX_WARPS_PER_BLOCK) return fail(CHEM_EINVAL, "couple_cells out of range");
  if (o.couple_cells == 0) o.couple_cells = 1;
  if (o.couple_cells > 1) {
    if (o.lu_precision != 64) return fail(CHEM_EINVAL, "coupled cells need lu_precision 64");
    if (o.record_adjoint) return fail(CHEM_EINVAL, "coupled cells have no adjoint");
    const int wmax = max_warps_per_block(mech->m.dev, o.lu_precision, o.driver);
    if (o.couple_cells > wmax) return fail(CHEM_EINVAL, "couple_cells exceeds the cells a block can hold");
    if (o.cells_per_block == 0) o.cells_per_block = (wmax / o.couple_cells) * o.couple_cells;   // whole groups per block
    if (o.cells_per_block % o.couple_cells) return fail(CHEM_EINVAL, "cells_per_block must be a multiple of couple_cells");
  }
  const int wmax = max_warps_per_block(mech->m.dev, o.lu_precision, o.driver);
  if (wmax < 1) return fail(CHEM_EINVAL, "mechanism working set does not fit in shared memory");
  if (o.cells_per_block > wmax) return fail(CHEM_EINVAL, "cells_per_block exceeds the shared-memory limit");
  if (o.cells_per_block == 0) o.cells_per_block = best_warps_per_block(mech->m.dev, o.lu_precision, o.driver);
  if (o.cells_per_block < 1) return fail(CHEM_EINVAL, "no launch shape fits on this device");
  if (o.record_adjoint && o.lu_precision != 64)
    return fail(CHEM_EINVAL, "record_adjoint needs lu_precision 64 (the adjoint differentiates the FP64 iteration)");
  if (o.record_adjoint && (o.tape_steps < 0 || o.tape_steps > CHEM_MAX_TAPE_ROWS))
    return fail(CHEM_EINVAL, "tape_steps out of range");
  if (o.stage_wait < -1) return fail(CHEM_EINVAL, "stage_wait must be -1, 0 or positive");

  chem_cells *c = new (std::nothrow) chem_cells();
  if (!c) return fail(CHEM_ENOMEM, "host allocation failed");
  c->mech = mech;
  c->n = n_cells;
  c->opts = o;
  cudaGetDevice(&c->device);
  const int S = mech->m.S, R = mech->m.R;
  const size_t n = (size_t)(n_cells > 0 ? n_cells : 1);
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&c->T, n * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&c->P, n * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&c->y, n * S * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&c->stats, n * sizeof(chem_cell_stats))) != cudaSuccess ||
      (e = cudaMalloc(&c->counters, 4 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&c->theta, (R > 0 ? R : 1) * sizeof(double))) != cudaSuccess ||
      (mech->m.n_phot > 0 && (e = cudaMalloc(&c->J, n * mech->m.n_phot * sizeof(double))) != cudaSuccess)) {
    chem_cells_destroy(c);
    return fail(CHEM_ENOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  if ((o.driver == CHEM_DRIVER_PERSISTENT || o.record_adjoint) &&
      ((e = cudaMalloc(&c->order, n * sizeof(int))) != cudaSuccess ||
       (e = cudaMalloc(&c->order_bucket, n * sizeof(int))) != cudaSuccess ||
       (e = cudaMalloc(&c->order_hist, ORDER_HIST_INTS * sizeof(int))) != cudaSuccess)) {
    chem_cells_destroy(c);
    return fail(CHEM_ENOMEM, std::string("cudaMalloc of the queue order failed: ") + cudaGetErrorString(e));
  }
  if (o.record_adjoint) {
    c->row_cap = o.tape_steps > 0 ? o.tape_steps : 2000;
    c->tape_cap = 3 * c->row_cap + 64;
    const size_t E = (size_t)c->tape_cap, RC = (size_t)c->row_cap;
    if ((e = cudaMalloc(&c->tape_kq, n * E * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&c->tape_val, n * E * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&c->tape_n, n * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&c->tape_rows, n * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&c->tape_bad, n * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&c->ytape, n * RC * S * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&c->gcell, n * (R > 0 ? R : 1) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&c->dLdy, n * S * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&c->dLdy0, n * S * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&c->dLdtheta, (R > 0 ? R : 1) * sizeof(double))) != cudaSuccess) {
      chem_cells_destroy(c);
      return fail(CHEM_ENOMEM, std::string("cudaMalloc of the adjoint tape failed: ") + cudaGetErrorString(e));
    }
    if ((e = cudaMemset(c->tape_n, 0, n * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(c->tape_rows, 0, n * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(c->tape_bad, 0, n * sizeof(int))) != cudaSuccess) {
      chem_cells_destroy(c);
      return cuda_fail(e, "cudaMemset");
    }
  }
  if ((e = cudaMemset(c->stats, 0, n * sizeof(chem_cell_stats))) != cudaSuccess ||
      (e = cudaMemset(c->counters, 0, 4 * sizeof(unsigned long long))) != cudaSuccess) {
    chem_cells_destroy(c);
    return cuda_fail(e, "cudaMemset");
  }
  *out = c;
  return 0;
}

void chem_cells_destroy(chem_cells *c) {
  if (!c) return;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  cudaFree(c->T);
  cudaFree(c->P);
  cudaFree(c->y);
  cudaFree(c->J);
  cudaFree(c->theta);
  cudaFree(c->stats);
  cudaFree(c->counters);
  cudaFree(c->order);
  cudaFree(c->order_bucket);
  cudaFree(c->order_hist);
  cudaFree(c->kt);
  cudaFree(c->tape_kq);
  cudaFree(c->tape_val);
  cudaFree(c->tape_n);
  cudaFree(c->tape_rows);
  cudaFree(c->tape_bad);
  cudaFree(c->ytape);
  cudaFree(c->gcell);
  cudaFree(c->dLdy);
  cudaFree(c->dLdy0);
  cudaFree(c->dLdtheta);
  delete c;
}

int chem_cells_set_state(chem_cells *c, const double *T, const double *P, const double *y, int32_t mem, void *stream) {
  Range range("chem_cells_set_state");
  g_err.clear();
  if (!c || !T || !P || !y) return fail(CHEM_EINVAL, "NULL argument");
  if (int rc = check_device(c)) return rc;
  c->kt_valid = false;
  if (int rc = check_mem(mem)) return rc;
  if (int rc = check_buffers(mem, {{T, "T"}, {P, "P"}, {y, "y"}})) return rc;
  if (c->n == 0) { c->have_state = true; return 0; }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)c->n, S = (size_t)c->mech->m.S;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->T, T, n * sizeof(double), kind_in(mem), s)) != cudaSuccess) return cuda_fail(e, "set_state T");
  if ((e = cudaMemcpyAsync(c->P, P, n * sizeof(double), kind_in(mem), s)) != cudaSuccess) return cuda_fail(e, "set_state P");
  if ((e = cudaMemcpyAsync(c->y, y, n * S * sizeof(double), kind_in(mem), s)) != cudaSuccess) return cuda_fail(e, "set_state y");
  if (c->tape_n) {   // a new state starts a new tape
    if ((e = cudaMemsetAsync(c->tape_n, 0, n * sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->tape_rows, 0, n * sizeof(int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->tape_bad, 0, n * sizeof(int), s)) != cudaSuccess)
      return cuda_fail(e, "set_state tape reset");
  }
  c->have_state = true;
  return 0;
}

int chem_cells_set_photolysis(chem_cells *c, const double *J, int32_t mem, void *stream) {
  g_err.clear();
  if (!c) return fail(CHEM_EINVAL, "NULL argument");
  if (int rc = check_device(c)) return rc;
  c->kt_valid = false;
  if (!J) { c->use_J = false; return 0; }
  if (int rc = check_mem(mem)) return rc;
  if (int rc = check_buffers(mem, {{J, "J"}})) return rc;
  const size_t np = (size_t)c->mech->m.n_phot;
  if (np == 0 || c->n == 0) { c->use_J = false; return 0; }
  cudaError_t e = cudaMemcpyAsync(c->J, J, np * (size_t)c->n * sizeof(double), kind_in(mem), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_photolysis");
  c->use_J = true;
  return 0;
}

int chem_cells_set_theta(chem_cells *c, const double *theta, int32_t mem, void *stream) {
  g_err.clear();
  if (!c) return fail(CHEM_EINVAL, "NULL argument");
  if (int rc = check_device(c)) return rc;
  c->kt_valid = false;
  if (!theta) { c->use_theta = false; return 0; }
  if (int rc = check_mem(mem)) return rc;
  if (int rc = check_buffers(mem, {{theta, "theta"}})) return rc;
  const size_t R = (size_t)c->mech->m.R;
  if (R == 0) return 0;
  cudaError_t e = cudaMemcpyAsync(c->theta, theta, R * sizeof(double), kind_in(mem), (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "set_theta");
  c->use_theta = true;
  return 0;
}

}  // extern "C"

namespace {

CellsDev solve_dev(chem_cells *c) {
  CellsDev cd{};
  cd.n_cells = c->n;
  cd.T = c->T;
  cd.P = c->P;
  cd.J = c->use_J ? c->J : nullptr;
  cd.theta = c->use_theta ? c->theta : nullptr;
  cd.y = c->y;
  cd.stats = c->stats;
  cd.queue = nullptr;
  cd.stage = c->counters + 1;
  cd.tape_kq = c->tape_kq;
  cd.ytape = c->ytape;
  cd.tape_val = c->tape_val;
  cd.tape_n = c->tape_n;
  cd.tape_rows = c->tape_rows;
  cd.tape_bad = c->tape_bad;
  cd.tape_cap = c->tape_cap;
  cd.row_cap = c->row_cap;
  return cd;
}

LaunchCfg launch_cfg(const chem_opts &o, double dt) {
  LaunchCfg cfg{};
  cfg.lu_precision = o.lu_precision;
  cfg.driver = o.driver;
  cfg.couple = o.couple_cells;
  cfg.warps_per_block = o.cells_per_block;
  cfg.blocks_per_sm = o.blocks_per_sm;
  cfg.rtol = o.rtol;
  cfg.atol = o.atol;
  cfg.dt = dt;
  cfg.max_order = o.max_order;
  cfg.max_steps = o.max_steps;
  cfg.stage_wait = o.stage_wait;
  return cfg;
}

// One solve of every cell on stream s: queue reset (persistent driver) and
// the solve kernel.  Stream-ordered calls only, so it can be captured.
cudaError_t enqueue_solve(chem_cells *c, double dt, cudaStream_t s) {
  CellsDev cd = solve_dev(c);
  if (c->opts.driver == CHEM_DRIVER_PERSISTENT) {
    cudaError_t e = cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    cd.queue = c->counters;
    // most expensive cells first, so the longest solves do not start last
    // (coupled groups are fixed sets of consecutive cells, handed out whole)
    if (c->opts.couple_cells > 1) {
      if ((e = launch_order_groups(cd, c->opts.couple_cells, c->order_bucket, c->order_hist, c->order, s)) != cudaSuccess)
        return e;
      cd.order = c->order;
    } else {
      if ((e = launch_order(c->mech->m.dev, cd, c->opts.rtol, c->opts.atol, c->order_bucket, c->order_hist, c->order,
                            s)) != cudaSuccess)
        return e;
      cd.order = c->order;
    }
  }
  return launch_solve(c->mech->m.dev, cd, launch_cfg(c->opts, dt), s);
}

int check_solve_args(chem_cells *c, double dt) {
  if (!c) return fail(CHEM_EINVAL, "NULL argument");
  if (!(dt > 0.0) || !(dt < 1e300)) return fail(CHEM_EINVAL, "dt must be positive and finite");
  if (!c->have_state) return fail(CHEM_ESTATE, "solve before set_state");
  return check_device(c);
}

// the staging counters report on one solve call (all its steps)
cudaError_t clear_stage_counters(chem_cells *c, cudaStream_t s) {
  return cudaMemsetAsync(c->counters + 1, 0, 2 * sizeof(unsigned long long), s);
}

}  // namespace

extern "C" {

int chem_solve_step(chem_cells *c, double dt, void *stream) {
  Range range("chem_solve_step");
  g_err.clear();
  if (int rc = check_solve_args(c, dt)) return rc;
  if (c->n == 0) return 0;
  cudaError_t e = clear_stage_counters(c, (cudaStream_t)stream);
  if (e == cudaSuccess) e = enqueue_solve(c, dt, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "solve kernel launch");
  return 0;
}

int chem_solve_steps(chem_cells *c, double dt, int32_t n_steps, void *stream) {
  Range range("chem_solve_steps");
  g_err.clear();
  if (int rc = check_solve_args(c, dt)) return rc;
  if (n_steps < 1 || n_steps > CHEM_MAX_GRAPH_STEPS) return fail(CHEM_EINVAL, "n_steps out of range");
  if (c->n == 0) return 0;
  cudaError_t e;
  const bool same = c->graph && c->graph_steps == n_steps && c->graph_dt == dt &&
                    c->graph_w == c->opts.cells_per_block && c->graph_bps == c->opts.blocks_per_sm &&
                    c->graph_J == c->use_J && c->graph_theta == c->use_theta;
  if (!same) {
    if (c->graph) {
      cudaGraphExecDestroy(c->graph);
      c->graph = nullptr;
    }
    if (!c->capture_stream && (e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "capture stream");
    // relaxed mode: the launch path may query and set kernel attributes while capturing
    if ((e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
      return cuda_fail(e, "begin capture");
    cudaError_t le = clear_stage_counters(c, c->capture_stream);
    for (int k = 0; k < n_steps && le == cudaSuccess; ++k) le = enqueue_solve(c, dt, c->capture_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->capture_stream, &g);
    if (le != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(le, "capture of the solve steps");
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->graph = nullptr;
      return cuda_fail(e, "graph instantiate");
    }
    c->graph_steps = n_steps;
    c->graph_dt = dt;
    c->graph_w = c->opts.cells_per_block;
    c->graph_bps = c->opts.blocks_per_sm;
    c->graph_J = c->use_J;
    c->graph_theta = c->use_theta;
  }
  if ((e = cudaGraphLaunch(c->graph, (cudaStream_t)stream)) != cudaSuccess) return cuda_fail(e, "graph launch");
  return 0;
}

int chem_autotune(chem_cells *c, double dt, int64_t n_sample, int32_t *cells_per_block, int32_t *blocks_per_sm) {
  Range range("chem_autotune");
  g_err.clear();
  if (int rc = check_solve_args(c, dt)) return rc;
  if (n_sample < 0) return fail(CHEM_EINVAL, "n_sample must be >= 0");
  if (c->opts.couple_cells > 1) return fail(CHEM_EINVAL, "a coupled batch's launch shape is its group size");
  if (c->n == 0) return 0;
  const int64_t ns = (n_sample == 0 || n_sample > c->n) ? (c->n < CHEM_AUTOTUNE_SAMPLE ? c->n : CHEM_AUTOTUNE_SAMPLE) : n_sample;
  const MechDev &M = c->mech->m.dev;
  const size_t S = (size_t)M.S, NP = (size_t)M.n_phot;
  const int prec = c->opts.lu_precision, drv = c->opts.driver;
  // scratch copy of the first ns cells with stride ns
  double *T = nullptr, *P = nullptr, *y = nullptr, *y0 = nullptr, *J = nullptr;
  chem_cell_stats *st = nullptr;
  long long *q = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s = nullptr;
  int rc = 0;
  cudaError_t e;
  auto cleanup = [&]() {
    cudaFree(T); cudaFree(P); cudaFree(y); cudaFree(y0); cudaFree(J); cudaFree(st); cudaFree(q);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
  };
  if ((e = cudaMalloc(&T, ns * sizeof(double))) != cudaSuccess || (e = cudaMalloc(&P, ns * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&y, ns * S * sizeof(double))) != cudaSuccess || (e = cudaMalloc(&y0, ns * S * sizeof(double))) != cudaSuccess ||
      (c->use_J && NP > 0 && (e = cudaMalloc(&J, ns * NP * sizeof(double))) != cudaSuccess) ||
      (e = cudaMalloc(&st, ns * sizeof(chem_cell_stats))) != cudaSuccess ||
      (e = cudaMalloc(&q, 4 * sizeof(long long))) != cudaSuccess) {
    cleanup();
    return fail(CHEM_ENOMEM, std::string("autotune scratch: ") + cudaGetErrorString(e));
  }
  if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess || (e = cudaEventCreate(&e0)) != cudaSuccess ||
      (e = cudaEventCreate(&e1)) != cudaSuccess ||
      (e = cudaMemcpyAsync(T, c->T, ns * sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(P, c->P, ns * sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpy2DAsync(y0, ns * sizeof(double), c->y, c->n * sizeof(double), ns * sizeof(double), S,
                             cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
      (J && (e = cudaMemcpy2DAsync(J, ns * sizeof(double), c->J, c->n * sizeof(double), ns * sizeof(double), NP,
                                   cudaMemcpyDeviceToDevice, s)) != cudaSuccess) ||
      (e = cudaMemsetAsync(q, 0, 4 * sizeof(long long), s)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "autotune setup");
  }
  CellsDev cd{};
  cd.n_cells = ns;
  cd.T = T;
  cd.P = P;
  cd.J = J;
  cd.theta = c->use_theta ? c->theta : nullptr;
  cd.y = y;
  cd.stats = st;
  cd.stage = reinterpret_cast<unsigned long long *>(q + 1);
  const int wmax = max_warps_per_block(M, prec, drv);
  float best = 0.0f;
  int best_w = 0, best_b = 0;
  for (int w = 1; w <= wmax && rc == 0; ++w) {
    const int occ = occupancy(M, prec, drv, w);
    if (occ < 1) continue;
    const int nb = drv == CHEM_DRIVER_PERSISTENT ? occ : 1;
    for (int b = 1; b <= nb && rc == 0; ++b) {
      LaunchCfg cfg = launch_cfg(c->opts, dt);
      cfg.warps_per_block = w;
      cfg.blocks_per_sm = drv == CHEM_DRIVER_PERSISTENT ? b : 0;
      float t_min = 0.0f;
      for (int rep = 0; rep < 2; ++rep) {
        if ((e = cudaMemcpyAsync(y, y0, ns * S * sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) break;
        cd.queue = nullptr;
        if (drv == CHEM_DRIVER_PERSISTENT) {
          if ((e = cudaMemsetAsync(q, 0, sizeof(long long), s)) != cudaSuccess) break;
          cd.queue = reinterpret_cast<unsigned long long *>(q);
        }
        float ms = 0.0f;
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess || (e = launch_solve(M, cd, cfg, s)) != cudaSuccess ||
            (e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
          break;
        if (rep == 0 || ms < t_min) t_min = ms;
      }
      if (e != cudaSuccess) {
        rc = cuda_fail(e, "autotune trial");
        break;
      }
      if (best_w == 0 || t_min < best) {
        best = t_min;
        best_w = w;
        best_b = cfg.blocks_per_sm;
      }
    }
  }
  cleanup();
  if (rc) return rc;
  if (best_w == 0) return fail(CHEM_EINVAL, "no launch shape fits on this device");
  c->opts.cells_per_block = best_w;
  c->opts.blocks_per_sm = best_b;
  if (cells_per_block) *cells_per_block = best_w;
  if (blocks_per_sm) *blocks_per_sm = best_b;
  return 0;
}

int chem_staging_fallbacks(const chem_cells *c, int64_t *fallbacks, int64_t *unfinished, void *stream) {
  g_err.clear();
  if (!fallbacks || !unfinished) return fail(CHEM_EINVAL, "NULL argument");
  if (!c) return noalloc_stage_counts(fallbacks, unfinished, (cudaStream_t)stream);
  if (int rc = check_device(c)) return rc;
  unsigned long long v[2] = {0, 0};
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(v, c->counters + 1, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "staging counters");
  *fallbacks = (int64_t)v[0];
  *unfinished = (int64_t)v[1];
  return 0;
}

int chem_get_state(const chem_cells *c, double *y, int32_t mem, void *stream) {
  Range range("chem_get_state");
  g_err.clear();
  if (!c || !y) return fail(CHEM_EINVAL, "NULL argument");
  if (int rc = check_mem(mem)) return rc;
  if (int rc = check_device(c)) return rc;
  if (int rc = check_buffers(mem, {{y, "y"}})) return rc;
  if (c->n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(y, c->y, (size_t)c->n * c->mech->m.S * sizeof(double), kind_out(mem), s);
  if (e != cudaSuccess) return cuda_fail(e, "get_state");
  if (mem == CHEM_MEM_HOST && (e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "get_state sync");
  return 0;
}

int chem_get_stats(const chem_cells *c, chem_cell_stats *out, int32_t mem, void *stream) {
  g_err.clear();
  if (!c || !out) return fail(CHEM_EINVAL, "NULL argument");
  if (int rc = check_mem(mem)) return rc;
  if (int rc = check_device(c)) return rc;
  if (int rc = check_buffers(mem, {{out, "out"}})) return rc;
  if (c->n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(out, c->stats, (size_t)c->n * sizeof(chem_cell_stats), kind_out(mem), s);
  if (e != cudaSuccess) return cuda_fail(e, "get_stats");
  if (mem == CHEM_MEM_HOST && (e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "get_stats sync");
  return 0;
}

namespace {

CellsDev cells_dev(chem_cells *c) {
  CellsDev cd{};
  cd.n_cells = c->n;
  cd.T = c->T;
  cd.P = c->P;
  cd.J = c->use_J ? c->J : nullptr;
  cd.theta = c->use_theta ? c->theta : nullptr;
  cd.y = c->y;
  cd.stats = c->stats;
  cd.queue = nullptr;
  cd.stage = c->counters + 1;
  cd.tape_kq = nullptr;
  cd.ytape = nullptr;
  cd.tape_val = nullptr;
  cd.tape_n = nullptr;
  cd.tape_rows = nullptr;
  cd.tape_bad = nullptr;
  cd.tape_cap = cd.row_cap = 0;
  return cd;
}

int probe(chem_cells *c, int mode, double cc, const double *y, const double *b, double *out, int32_t mem, void *stream) {
  g_err.clear();
  if (!c || !y || !out || (mode == 1 && !b)) return fail(CHEM_EINVAL, "NULL argument");
  if (int rc = check_mem(mem)) return rc;
  if (!c->have_state) return fail(CHEM_ESTATE, "diagnostic before set_state");
  if (int rc = check_device(c)) return rc;
  if (int rc = check_buffers(mem, {{y, "y"}, {b, "b"}, {out, "out"}})) return rc;
  if (c->n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)c->n * c->mech->m.S * sizeof(double);
  const double *dy = y, *db = b;
  double *dout = out, *tmp = nullptr;
  cudaError_t e = cudaSuccess;
  if (mem == CHEM_MEM_HOST) {
    if ((e = cudaMalloc(&tmp, 3 * bytes)) != cudaSuccess) return fail(CHEM_ENOMEM, "cudaMalloc for diagnostic scratch");
    double *ty = tmp, *tb = tmp + bytes / sizeof(double), *to = tmp + 2 * (bytes / sizeof(double));
    if ((e = cudaMemcpyAsync(ty, y, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (b && (e = cudaMemcpyAsync(tb, b, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)) {
      cudaFree(tmp);
      return cuda_fail(e, "diagnostic copy-in");
    }
    dy = ty;
    db = b ? tb : nullptr;
    dout = to;
  }
  e = launch_probe(c->mech->m.dev, cells_dev(c), c->opts.lu_precision, mode, cc, dy, db, dout, s);
  if (e == cudaSuccess && mem == CHEM_MEM_HOST) {
    e = cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "diagnostic kernel");
  return 0;
}

}  // namespace

int chem_eval_deriv(chem_cells *c, const double *y, double *f, int32_t mem, void *stream) {
  return probe(c, 0, 0.0, y, nullptr, f, mem, stream);
}

int chem_eval_newton_solve(chem_cells *c, double cc, const double *y, const double *b, double *x, int32_t mem,
                           void *stream) {
  return probe(c, 1, cc, y, b, x, mem, stream);
}

int chem_eval_reciprocal(const double *x, double *out, int64_t n, int32_t mem, void *stream) {
  g_err.clear();
  if (n < 0 || (n > 0 && (!x || !out))) return fail(CHEM_EINVAL, "bad argument");
  if (int rc = check_mem(mem)) return rc;
  if (n == 0) return 0;
  if (int rc = check_buffers(mem, {{x, "x"}, {out, "out"}})) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)n * sizeof(double);
  double *tmp = nullptr;
  const double *dx = x;
  double *dout = out;
  cudaError_t e = cudaSuccess;
  if (mem == CHEM_MEM_HOST) {
    if (cudaMalloc(&tmp, 2 * bytes) != cudaSuccess) return fail(CHEM_ENOMEM, "cudaMalloc for diagnostic scratch");
    dx = tmp;
    dout = tmp + n;
    e = cudaMemcpyAsync(tmp, x, bytes, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = launch_recip_probe(dx, dout, n, s);
  if (e == cudaSuccess && mem == CHEM_MEM_HOST) {
    e = cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "reciprocal diagnostic");
  return 0;
}

int chem_eval_warp_sum(const double *x, double *out, int64_t n_groups, int32_t mem, void *stream) {
  g_err.clear();
  if (n_groups < 0 || (n_groups > 0 && (!x || !out))) return fail(CHEM_EINVAL, "bad argument");
  if (int rc = check_mem(mem)) return rc;
  if (n_groups == 0) return 0;
  if (int rc = check_buffers(mem, {{x, "x"}, {out, "out"}})) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t in_bytes = (size_t)n_groups * WARP * sizeof(double), out_bytes = (size_t)n_groups * sizeof(double);
  double *tmp = nullptr;
  const double *dx = x;
  double *dout = out;
  cudaError_t e = cudaSuccess;
  if (mem == CHEM_MEM_HOST) {
    if (cudaMalloc(&tmp, in_bytes + out_bytes) != cudaSuccess) return fail(CHEM_ENOMEM, "cudaMalloc for diagnostic scratch");
    dx = tmp;
    dout = tmp + (size_t)n_groups * WARP;
    e = cudaMemcpyAsync(tmp, x, in_bytes, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = launch_wsum_probe(dx, dout, n_groups, s);
  if (e == cudaSuccess && mem == CHEM_MEM_HOST) {
    e = cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "warp-sum diagnostic");
  return 0;
}

int chem_eval_deriv_design(chem_cells *c, int32_t design, const double *y, double *f, int32_t mem, void *stream) {
  Range range("chem_eval_deriv_design");
  g_err.clear();
  if (!c || !y || !f) return fail(CHEM_EINVAL, "NULL argument");
  if (design != CHEM_DERIV_GATHER && design != CHEM_DERIV_ATOMIC_AOS && design != CHEM_DERIV_ATOMIC_SOA)
    return fail(CHEM_EINVAL, "unknown derivative design");
  if (int rc = check_mem(mem)) return rc;
  if (!c->have_state) return fail(CHEM_ESTATE, "derivative before set_state");
  if (int rc = check_device(c)) return rc;
  if (int rc = check_buffers(mem, {{y, "y"}, {f, "f"}})) return rc;
  if (c->n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  const MechDev &M = c->mech->m.dev;
  cudaError_t e;
  if (!c->kt && (e = cudaMalloc(&c->kt, (size_t)c->n * (M.R > 0 ? M.R : 1) * sizeof(double))) != cudaSuccess) {
    c->kt = nullptr;
    return fail(CHEM_ENOMEM, std::string("cudaMalloc of the rate constants failed: ") + cudaGetErrorString(e));
  }
  if (!c->kt_valid) {
    if ((e = launch_rates(M, cells_dev(c), c->kt, s)) != cudaSuccess) return cuda_fail(e, "rate constants");
    c->kt_valid = true;
  }
  const size_t bytes = (size_t)c->n * M.S * sizeof(double);
  const double *dy = y;
  double *df = f, *tmp = nullptr;
  if (mem == CHEM_MEM_HOST) {
    if ((e = cudaMalloc(&tmp, 2 * bytes)) != cudaSuccess) return fail(CHEM_ENOMEM, "cudaMalloc for derivative scratch");
    if ((e = cudaMemcpyAsync(tmp, y, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
      cudaFree(tmp);
      return cuda_fail(e, "derivative copy-in");
    }
    dy = tmp;
    df = tmp + bytes / sizeof(double);
  }
  e = launch_deriv_design(M, cells_dev(c), design, c->kt, dy, df, s);
  if (e == cudaSuccess && mem == CHEM_MEM_HOST) {
    e = cudaMemcpyAsync(f, df, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "derivative kernels");
  return 0;
}

int chem_sensitivity(chem_cells *c, const double *dL_dy, double *dL_dtheta, double *dL_dy0, int32_t mem, void *stream) {
  Range range("chem_sensitivity");
  g_err.clear();
  if (!c || !dL_dy || !dL_dtheta || !dL_dy0) return fail(CHEM_EINVAL, "NULL argument");
  if (int rc = check_mem(mem)) return rc;
  if (!c->tape_n) return fail(CHEM_ESTATE, "the batch was created without record_adjoint");
  if (!c->have_state) return fail(CHEM_ESTATE, "sensitivity before set_state");
  if (int rc = check_device(c)) return rc;
  if (int rc = check_buffers(mem, {{dL_dy, "dL_dy"}, {dL_dtheta, "dL_dtheta"}, {dL_dy0, "dL_dy0"}})) return rc;
  const size_t n = (size_t)c->n, S = (size_t)c->mech->m.S, R = (size_t)c->mech->m.R;
  if (n == 0) {
    if (mem == CHEM_MEM_HOST) std::memset(dL_dtheta, 0, R * sizeof(double));
    else cudaMemsetAsync(dL_dtheta, 0, R * sizeof(double), (cudaStream_t)stream);
    return 0;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->dLdy, dL_dy, n * S * sizeof(double), kind_in(mem), s)) != cudaSuccess)
    return cuda_fail(e, "sensitivity copy-in");
  CellsDev cd{};
  cd.n_cells = c->n;
  cd.T = c->T;
  cd.P = c->P;
  cd.J = c->use_J ? c->J : nullptr;
  cd.theta = c->use_theta ? c->theta : nullptr;
  cd.y = c->y;
  cd.stats = c->stats;
  cd.queue = nullptr;
  cd.stage = nullptr;
  cd.tape_kq = c->tape_kq;
  cd.ytape = c->ytape;
  cd.tape_val = c->tape_val;
  cd.tape_n = c->tape_n;
  cd.tape_rows = c->tape_rows;
  cd.tape_bad = c->tape_bad;
  cd.tape_cap = c->tape_cap;
  cd.row_cap = c->row_cap;
  AdjDev ad{};
  ad.dLdy = c->dLdy;
  ad.dLdy0 = c->dLdy0;
  ad.gcell = c->gcell;
  ad.dLdtheta = c->dLdtheta;
  ad.accumulate = 0;
  // the longest tapes first, popped from the batch's work counter
  if ((e = launch_order_tape(cd, c->order_bucket, c->order_hist, c->order, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long), s)) != cudaSuccess)
    return cuda_fail(e, "adjoint order");
  cd.order = c->order;
  cd.queue = c->counters;
  if ((e = launch_adjoint(c->mech->m.dev, cd, ad, s)) != cudaSuccess) return cuda_fail(e, "adjoint kernels");
  if ((e = cudaMemcpyAsync(dL_dy0, c->dLdy0, n * S * sizeof(double), kind_out(mem), s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dL_dtheta, c->dLdtheta, R * sizeof(double), kind_out(mem), s)) != cudaSuccess)
    return cuda_fail(e, "sensitivity copy-out");
  std::vector<int> bad(n);
  if ((e = cudaMemcpyAsync(bad.data(), c->tape_bad, n * sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "sensitivity sync");
  int n_bad = 0;
  for (int v : bad) n_bad += v != 0;
  return n_bad;
}

int chem_sensitivity_checkpointed(chem_cells *c, const double *states, int32_t n_steps, double dt,
                                  int32_t last_recorded, const double *dL_dy, double *dL_dtheta, double *dL_dy0,
                                  int32_t mem, void *stream) {
  Range range("chem_sensitivity_checkpointed");
  g_err.clear();
  if (!c || !states || !dL_dy || !dL_dtheta || !dL_dy0) return fail(CHEM_EINVAL, "NULL argument");
  if (int rc = check_mem(mem)) return rc;
  if (!c->tape_n) return fail(CHEM_ESTATE, "the batch was created without record_adjoint");
  if (!c->have_state) return fail(CHEM_ESTATE, "sensitivity before set_state");
  if (int rc = check_device(c)) return rc;
  if (int rc = check_buffers(mem, {{states, "states"}, {dL_dy, "dL_dy"}, {dL_dtheta, "dL_dtheta"}, {dL_dy0, "dL_dy0"}}))
    return rc;
  if (n_steps < 1 || n_steps > CHEM_MAX_GRAPH_STEPS) return fail(CHEM_EINVAL, "n_steps out of range");
  if (!(dt > 0.0) || !(dt < 1e300)) return fail(CHEM_EINVAL, "dt must be positive and finite");
  const size_t n = (size_t)c->n, S = (size_t)c->mech->m.S, R = (size_t)c->mech->m.R;
  cudaStream_t s = (cudaStream_t)stream;
  if (n == 0) {
    if (mem == CHEM_MEM_HOST) std::memset(dL_dtheta, 0, R * sizeof(double));
    else cudaMemsetAsync(dL_dtheta, 0, R * sizeof(double), s);
    return 0;
  }
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->dLdy, dL_dy, n * S * sizeof(double), kind_in(mem), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->counters + 3, 0, sizeof(unsigned long long), s)) != cudaSuccess)
    return cuda_fail(e, "sensitivity copy-in");
  CellsDev cd = solve_dev(c);
  cd.stage = nullptr;
  // lambda ping-pongs between the batch's two adjoint vectors
  double *lin = c->dLdy, *lout = c->dLdy0;
  for (int k = n_steps - 1; k >= 0; --k) {
    if (!(last_recorded && k == n_steps - 1)) {
      // re-run step k from its kept state with a fresh tape
      if ((e = cudaMemcpyAsync(c->y, states + (size_t)k * S * n, n * S * sizeof(double), kind_in(mem), s)) != cudaSuccess ||
          (e = cudaMemsetAsync(c->tape_n, 0, n * sizeof(int), s)) != cudaSuccess ||
          (e = cudaMemsetAsync(c->tape_rows, 0, n * sizeof(int), s)) != cudaSuccess ||
          (e = cudaMemsetAsync(c->tape_bad, 0, n * sizeof(int), s)) != cudaSuccess ||
          (e = enqueue_solve(c, dt, s)) != cudaSuccess)
        return cuda_fail(e, "checkpointed re-solve");
    }
    CellsDev ca = cd;
    if ((e = launch_order_tape(ca, c->order_bucket, c->order_hist, c->order, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long), s)) != cudaSuccess)
      return cuda_fail(e, "adjoint order");
    ca.order = c->order;
    ca.queue = c->counters;
    AdjDev ad{};
    ad.dLdy = lin;
    ad.dLdy0 = lout;
    ad.gcell = c->gcell;
    ad.dLdtheta = c->dLdtheta;
    ad.accumulate = k != n_steps - 1;
    if ((e = launch_adjoint(c->mech->m.dev, ca, ad, s)) != cudaSuccess ||
        (e = launch_count_flags(c->tape_bad, c->n, c->counters + 3, s)) != cudaSuccess)
      return cuda_fail(e, "adjoint kernels");
    std::swap(lin, lout);
  }
  unsigned long long n_bad = 0;
  if ((e = cudaMemcpyAsync(dL_dy0, lin, n * S * sizeof(double), kind_out(mem), s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dL_dtheta, c->dLdtheta, R * sizeof(double), kind_out(mem), s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&n_bad, c->counters + 3, sizeof(n_bad), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "sensitivity copy-out");
  return n_bad > (unsigned long long)INT32_MAX ? INT32_MAX : (int)n_bad;
}

int chem_tangent(chem_cells *c, const double *dy0, const double *dtheta, double *dy, int32_t mem, void *stream) {
  Range range("chem_tangent");
  g_err.clear();
  if (!c || !dy0 || !dy) return fail(CHEM_EINVAL, "NULL argument");
  if (int rc = check_mem(mem)) return rc;
  if (!c->tape_n) return fail(CHEM_ESTATE, "the batch was created without record_adjoint");
  if (!c->have_state) return fail(CHEM_ESTATE, "tangent before set_state");
  if (int rc = check_device(c)) return rc;
  if (int rc = check_buffers(mem, {{dy0, "dy0"}, {dtheta, "dtheta"}, {dy, "dy"}})) return rc;
  const size_t n = (size_t)c->n, S = (size_t)c->mech->m.S, R = (size_t)c->mech->m.R;
  if (n == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  // the adjoint's buffers hold the tangent's input and output
  if ((e = cudaMemcpyAsync(c->dLdy, dy0, n * S * sizeof(double), kind_in(mem), s)) != cudaSuccess ||
      (dtheta && R > 0 && (e = cudaMemcpyAsync(c->dLdtheta, dtheta, R * sizeof(double), kind_in(mem), s)) != cudaSuccess))
    return cuda_fail(e, "tangent copy-in");
  CellsDev cd{};
  cd.n_cells = c->n;
  cd.T = c->T;
  cd.P = c->P;
  cd.J = c->use_J ? c->J : nullptr;
  cd.theta = c->use_theta ? c->theta : nullptr;
  cd.y = c->y;
  cd.stats = c->stats;
  cd.tape_kq = c->tape_kq;
  cd.ytape = c->ytape;
  cd.tape_val = c->tape_val;
  cd.tape_n = c->tape_n;
  cd.tape_rows = c->tape_rows;
  cd.tape_bad = c->tape_bad;
  cd.tape_cap = c->tape_cap;
  cd.row_cap = c->row_cap;
  TanDev td;
  td.dy0 = c->dLdy;
  td.dtheta = (dtheta && R > 0) ? c->dLdtheta : nullptr;
  td.dy = c->dLdy0;
  if ((e = launch_order_tape(cd, c->order_bucket, c->order_hist, c->order, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long), s)) != cudaSuccess)
    return cuda_fail(e, "tangent order");
  cd.order = c->order;
  cd.queue = c->counters;
  if ((e = launch_tangent(c->mech->m.dev, cd, td, s)) != cudaSuccess) return cuda_fail(e, "tangent kernel");
  if ((e = cudaMemcpyAsync(dy, c->dLdy0, n * S * sizeof(double), kind_out(mem), s)) != cudaSuccess)
    return cuda_fail(e, "tangent copy-out");
  std::vector<int> bad(n);
  if ((e = cudaMemcpyAsync(bad.data(), c->tape_bad, n * sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "tangent sync");
  int n_bad = 0;
  for (int v : bad) n_bad += v != 0;
  return n_bad;
}

int chem_get_tape(const chem_cells *c, int64_t cell, int32_t *kind, int32_t *q, double *val, double *rows,
                  int32_t capacity, int32_t *n_events, int32_t *n_rows) {
  g_err.clear();
  if (!c || !n_events || !n_rows) return fail(CHEM_EINVAL, "NULL argument");
  if (!c->tape_n) return fail(CHEM_ESTATE, "the batch was created without record_adjoint");
  if (cell < 0 || cell >= c->n) return fail(CHEM_EINVAL, "cell index out of range");
  if (int rc = check_device(c)) return rc;
  int n = 0, nr = 0;
  cudaError_t e;
  if ((e = cudaMemcpy(&n, c->tape_n + cell, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(&nr, c->tape_rows + cell, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "get_tape");
  *n_events = n;
  *n_rows = nr;
  if (capacity < n || !kind || !q || !val) return 0;
  std::vector<int> kq(n);
  if ((e = cudaMemcpy(kq.data(), c->tape_kq + cell * (int64_t)c->tape_cap, n * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(val, c->tape_val + cell * (int64_t)c->tape_cap, n * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "get_tape");
  const size_t S = (size_t)c->mech->m.S;
  if (rows && nr > 0 &&
      (e = cudaMemcpy(rows, c->ytape + cell * (int64_t)c->row_cap * S, (size_t)nr * S * sizeof(double),
                      cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "get_tape rows");
  for (int i = 0; i < n; ++i) {
    kind[i] = kq[i] & 0xff;
    q[i] = kq[i] >> 8;
  }
  return 0;
}

// ---------------------------------------------------------------- pipeline
// Host-resident state, chunked: per chunk its own batch and stream, so the
// copies of one chunk overlap the solves of the others and the host's work on
// a chunk that is back overlaps the GPU's work on the rest.

struct chem_pipeline {
  const chem_mech *mech = nullptr;
  int64_t n = 0;
  std::vector<int64_t> c0;                 // chunk k is cells [c0[k], c0[k + 1])
  std::vector<chem_cells *> sub;
  std::vector<cudaStream_t> stream;
  std::vector<cudaEvent_t> done;
};

void chem_pipeline_destroy(chem_pipeline *p) {
  if (!p) return;
  for (cudaStream_t s : p->stream)
    if (s) cudaStreamSynchronize(s);
  for (cudaEvent_t e : p->done)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : p->stream)
    if (s) cudaStreamDestroy(s);
  for (chem_cells *c : p->sub) chem_cells_destroy(c);
  delete p;
}

int chem_pipeline_create(const chem_mech *mech, int64_t n_cells, int32_t n_chunks, const chem_opts *opts,
                         chem_pipeline **out) {
  g_err.clear();
  if (!out) return fail(CHEM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mech) return fail(CHEM_EINVAL, "mechanism is NULL");
  if (n_cells < 0 || n_cells > ((int64_t)1 << 31)) return fail(CHEM_EINVAL, "n_cells must be in 0..2^31");
  if (n_chunks < 1 || n_chunks > 64) return fail(CHEM_EINVAL, "n_chunks must be in 1..64");
  if (n_cells > 0 && n_chunks > n_cells) return fail(CHEM_EINVAL, "more chunks than cells");
  if (opts && (opts->record_adjoint || opts->couple_cells > 1))
    return fail(CHEM_EINVAL, "a pipeline takes neither record_adjoint nor couple_cells");
  chem_pipeline *p = new (std::nothrow) chem_pipeline();
  if (!p) return fail(CHEM_ENOMEM, "host allocation failed");
  p->mech = mech;
  p->n = n_cells;
  const int K = n_cells > 0 ? n_chunks : 1;
  const int64_t base = n_cells / K, extra = n_cells % K;
  p->c0.push_back(0);
  for (int k = 0; k < K; ++k) p->c0.push_back(p->c0.back() + base + (k < extra ? 1 : 0));
  p->sub.assign(K, nullptr);
  p->stream.assign(K, nullptr);
  p->done.assign(K, nullptr);
  for (int k = 0; k < K; ++k) {
    if (int rc = chem_cells_create(mech, p->c0[k + 1] - p->c0[k], opts, &p->sub[k])) {
      const std::string msg = g_err;
      chem_pipeline_destroy(p);
      return fail(rc, msg);
    }
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&p->stream[k], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p->done[k], cudaEventDisableTiming)) != cudaSuccess) {
      chem_pipeline_destroy(p);
      return cuda_fail(e, "pipeline streams");
    }
  }
  *out = p;
  return 0;
}

namespace {

// chunk k, one model step: inputs in, the solve, y out, then the chunk's event
cudaError_t pipeline_enqueue(chem_pipeline *p, int k, const double *T, const double *P, const double *J, double *y,
                             double dt) {
  chem_cells *c = p->sub[k];
  const cudaStream_t s = p->stream[k];
  const int64_t c0 = p->c0[k], nk = c->n;
  const size_t S = (size_t)p->mech->m.S, np = (size_t)p->mech->m.n_phot;
  const size_t ld = (size_t)p->n * sizeof(double), w = (size_t)nk * sizeof(double);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->T, T + c0, w, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(c->P, P + c0, w, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpy2DAsync(c->y, w, y + c0, ld, w, S, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  c->use_J = J && np > 0;
  if (c->use_J && (e = cudaMemcpy2DAsync(c->J, w, J + c0, ld, w, np, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  c->have_state = true;
  c->kt_valid = false;
  if ((e = enqueue_solve(c, dt, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpy2DAsync(y + c0, ld, c->y, w, w, S, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
  return cudaEventRecord(p->done[k], s);
}

}  // namespace

int chem_pipeline_run(chem_pipeline *p, const double *T, const double *P, const double *J, double *y, double dt,
                      int32_t n_steps, chem_chunk_fn fn, void *user, chem_cell_stats *stats) {
  Range range("chem_pipeline_run");
  g_err.clear();
  if (!p || !T || !P || !y) return fail(CHEM_EINVAL, "NULL argument");
  if (!(dt > 0.0) || !(dt < 1e300)) return fail(CHEM_EINVAL, "dt must be positive and finite");
  if (n_steps < 0) return fail(CHEM_EINVAL, "n_steps must be >= 0");
  if (p->n == 0 || n_steps == 0) return 0;
  const int K = (int)p->sub.size();
  cudaError_t e = cudaSuccess;
  int rc = 0;
  for (int k = 0; k < K && e == cudaSuccess; ++k) e = pipeline_enqueue(p, k, T, P, J, y, dt);
  // visit the chunks in queue order; a chunk's next step goes in as soon as its callback returns
  for (int step = 0; step < n_steps && e == cudaSuccess && rc == 0; ++step)
    for (int k = 0; k < K && e == cudaSuccess && rc == 0; ++k) {
      if ((e = cudaEventSynchronize(p->done[k])) != cudaSuccess) break;
      int stop = 0;
      if (fn) {
        Range cb("chem_pipeline host work");
        stop = fn(p->c0[k], p->c0[k + 1], step, user);
      }
      if (stop != 0) {
        rc = fail(CHEM_EABORTED, "a chunk callback stopped the pipeline");
        break;
      }
      if (step + 1 < n_steps) e = pipeline_enqueue(p, k, T, P, J, y, dt);
    }
  // drain whatever is still queued, also on the error paths
  for (int k = 0; k < K; ++k) {
    const cudaError_t es = cudaStreamSynchronize(p->stream[k]);
    if (e == cudaSuccess) e = es;
  }
  if (e != cudaSuccess) return cuda_fail(e, "pipeline");
  if (rc) return rc;
  if (stats)
    for (int k = 0; k < K; ++k)
      if ((e = cudaMemcpy(stats + p->c0[k], p->sub[k]->stats, (size_t)p->sub[k]->n * sizeof(chem_cell_stats),
                          cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "pipeline stats");
  return 0;
}

}  // extern "C"
