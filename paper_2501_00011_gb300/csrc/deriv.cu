// deriv.cu -- derivative-only kernels for comparing designs of f(y) on the GPU.
//
// The paper's GPU work is the Derivative function (Implementations section):
// one GPU thread per reaction and cell computes the reaction's rate and adds
// its contributions to the species' rates of change with atomic additions;
// reorganising the reaction data for the GPU gave a further speedup.  This
// file builds that design (reaction data as an array of structures or as a
// structure of arrays) so it can be measured against this library's gather,
// one warp per cell running the compiled f program (kernels.cu), on the same
// inputs: the rate constants of the batch computed once, y and f in HBM.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "internal.h"

namespace chemgpu {

namespace {

constexpr int DERIV_THREADS = 256;

// a1 for every (cell, reaction): kt[j][c], cells fastest
__global__ void rates_kernel(const __grid_constant__ MechDev M, const CellsDev C, double *kt) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (c >= C.n_cells) return;
  const double Tc = C.T[c], Pc = C.P[c];
  kt[(int64_t)j * C.n_cells + c] = rate_constant(M, C, j, c, Tc, air_number_density(Tc, Pc));
}

// a2, reaction-parallel: thread (j, c) forms r_j = k~_j prod y and adds -r_j
// to each reactant and yield * r_j to each product of reaction j in cell c.
template <bool AOS>
__global__ void deriv_atomic_kernel(const __grid_constant__ MechDev M, const int64_t NC, const double *kt,
                                    const double *y, double *f) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (c >= NC) return;
  double r = kt[(int64_t)j * NC + c];
  if (AOS) {
    const chem_reaction &rx = M.rx_aos[j];
    const int nr = rx.n_reac, np = rx.n_prod;
    for (int s = 0; s < nr; ++s) r *= y[(int64_t)rx.reac[s] * NC + c];
    for (int s = 0; s < nr; ++s) atomicAdd(f + (int64_t)rx.reac[s] * NC + c, -r);
    for (int p = 0; p < np; ++p) atomicAdd(f + (int64_t)rx.prod[p] * NC + c, rx.yield[p] * r);
  } else {
    const int nr = __ldg(M.rx_nreac + j), np = __ldg(M.rx_nprod + j);
    for (int s = 0; s < nr; ++s) r *= y[(int64_t)__ldg(M.rx_reac + j * CHEM_MAX_REAC + s) * NC + c];
    for (int s = 0; s < nr; ++s) atomicAdd(f + (int64_t)__ldg(M.rx_reac + j * CHEM_MAX_REAC + s) * NC + c, -r);
    for (int p = 0; p < np; ++p)
      atomicAdd(f + (int64_t)__ldg(M.rx_prod + j * CHEM_MAX_PROD + p) * NC + c, __ldg(M.rx_yld + j * CHEM_MAX_PROD + p) * r);
  }
}

}  // namespace

cudaError_t launch_rates(const MechDev &M, const CellsDev &C, double *kt, cudaStream_t stream) {
  if (C.n_cells <= 0 || M.R == 0) return cudaSuccess;
  if (M.R > 65535) return cudaErrorInvalidValue;     // one grid row per reaction
  const dim3 grid((unsigned)((C.n_cells + DERIV_THREADS - 1) / DERIV_THREADS), (unsigned)M.R);
  rates_kernel<<<grid, DERIV_THREADS, 0, stream>>>(M, C, kt);
  return cudaGetLastError();
}

cudaError_t launch_deriv_design(const MechDev &M, const CellsDev &C, int design, const double *kt, const double *y,
                                double *f, cudaStream_t stream) {
  if (C.n_cells <= 0) return cudaSuccess;
  if (design == CHEM_DERIV_GATHER) return launch_deriv_gather(M, C, kt, y, f, stream);
  if (design != CHEM_DERIV_ATOMIC_AOS && design != CHEM_DERIV_ATOMIC_SOA) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(f, 0, (size_t)C.n_cells * M.S * sizeof(double), stream);
  if (e != cudaSuccess || M.R == 0) return e;
  if (M.R > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((C.n_cells + DERIV_THREADS - 1) / DERIV_THREADS), (unsigned)M.R);
  if (design == CHEM_DERIV_ATOMIC_AOS)
    deriv_atomic_kernel<true><<<grid, DERIV_THREADS, 0, stream>>>(M, C.n_cells, kt, y, f);
  else
    deriv_atomic_kernel<false><<<grid, DERIV_THREADS, 0, stream>>>(M, C.n_cells, kt, y, f);
  return cudaGetLastError();
}

}  // namespace chemgpu
