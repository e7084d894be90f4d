// device_common.cuh -- device functions shared by the CUDA translation units.
#pragma once

#include "internal.h"

namespace chemgpu {

// number density of air in molecules per cm^3 at T (K), P (Pa): P / (k_B T) * 1e-6
__device__ __forceinline__ double air_number_density(const double Tc, const double Pc) {
  constexpr double K_BOLTZMANN = 1.380649e-23;   // J/K (exact, SI 2019)
  return Pc / (K_BOLTZMANN * Tc) * 1e-6;
}

// a1: the rate constant k~_j of one cell (Background: each reaction's rate is
// a function of temperature and pressure).  Thermal: A exp(-Ea/T) (T/300)^B
// times n_air^(n_reac - 1) so that rates act on mixing ratios; photolysis:
// the cell's J (or the mechanism's); both times exp(theta_j) when theta is set.
__device__ __forceinline__ double rate_constant(const MechDev &M, const CellsDev &C, const int j, const int64_t cell,
                                                const double Tc, const double n_air) {
  double kj;
  if (__ldg(M.rx_kind + j) == CHEM_PHOTOLYSIS) {
    kj = C.J ? C.J[(int64_t)__ldg(M.rx_phot + j) * C.n_cells + cell] : __ldg(M.rx_J + j);
  } else {
    kj = __ldg(M.rx_A + j) * exp(-__ldg(M.rx_Ea + j) / Tc) * pow(Tc / 300.0, __ldg(M.rx_B + j));
    const int nr = __ldg(M.rx_nreac + j);
    for (int r = 1; r < nr; ++r) kj *= n_air;
  }
  if (C.theta) kj *= exp(C.theta[j]);
  return kj;
}

}  // namespace chemgpu
