// device_common.cuh -- device functions shared by the CUDA translation units.
#pragma once

#include "internal.h"

namespace chemgpu {

// number density of air in molecules per cm^3 at T (K), P (Pa): P / (k_B T) * 1e-6
__device__ __forceinline__ double air_number_density(const double Tc, const double Pc) {
  constexpr double K_BOLTZMANN = 1.380649e-23;   // J/K (exact, SI 2019)
  return Pc / (K_BOLTZMANN * Tc) * 1e-6;
}

__device__ __forceinline__ double arrhenius(const double A, const double Ea, const double B, const double Tc) {
  return A * exp(-Ea / Tc) * pow(Tc / 300.0, B);
}

// a1: the rate constant k~_j of one cell (Background: each reaction's rate is
// a function of temperature and pressure).  Thermal: A exp(-Ea/T) (T/300)^B;
// the pressure-dependent kinds combine up to three such terms with the air
// number density [M] (Troe fall-off, k_a + k_b [M], k_a + k_c [M] / (1 + k_c [M] / k_b));
// all thermal kinds times n_air^(n_reac - 1) so that rates act on mixing
// ratios; photolysis: the cell's J (or the mechanism's); every kind times
// exp(theta_j) when theta is set.
__device__ __forceinline__ double rate_constant(const MechDev &M, const CellsDev &C, const int j, const int64_t cell,
                                                const double Tc, const double n_air) {
  double kj;
  const int kind = __ldg(M.rx_kind + j);
  if (kind == CHEM_PHOTOLYSIS) {
    kj = C.J ? C.J[(int64_t)__ldg(M.rx_phot + j) * C.n_cells + cell] : __ldg(M.rx_J + j);
  } else {
    kj = arrhenius(__ldg(M.rx_A + j), __ldg(M.rx_Ea + j), __ldg(M.rx_B + j), Tc);
    if (kind != CHEM_THERMAL) {
      const double *e = M.rx_ext + (size_t)j * RX_EXT;
      const double kb = arrhenius(__ldg(e + 0), __ldg(e + 1), __ldg(e + 2), Tc);
      if (kind == CHEM_TROE) {
        const double k0m = kj * n_air;            // low-pressure limit times [M]
        const double x = k0m / kb;
        const double lx = log10(x) / __ldg(e + 7);
        kj = k0m / (1.0 + x) * pow(__ldg(e + 6), 1.0 / (1.0 + lx * lx));
      } else if (kind == CHEM_PRESSURE_SUM) {
        kj += kb * n_air;
      } else {                                    // CHEM_FALLOFF_SUM
        const double kcm = arrhenius(__ldg(e + 3), __ldg(e + 4), __ldg(e + 5), Tc) * n_air;
        kj += kcm / (1.0 + kcm / kb);
      }
    }
    const int nr = __ldg(M.rx_nreac + j);
    for (int r = 1; r < nr; ++r) kj *= n_air;
  }
  if (C.theta) kj *= exp(C.theta[j]);
  return kj;
}

}  // namespace chemgpu
