"""Pins of the oracle's pressure-dependent rate constants.

The rate of a reaction is a function of the whole state, temperature and
pressure included (Background section).  The oracle's fall-off and
pressure-sum kinds are pinned here by properties the physics fixes, not by
their formulas: the Troe broadening equals Fc at the centre of the fall-off
curve and Fc^(1/2) one decade (N = 1) or two decades (N = 2) either side of
it, and is symmetric in log10(k0 [M] / kinf); with Fc = 1 the rate
constant is the harmonic combination 1/k = 1/(k0 [M]) + 1/kinf and tends to
k0 [M] and kinf at the low- and high-pressure ends; a pressure sum is linear
in [M] with slope and intercept equal to thermal reactions with the same
Arrhenius parameters; a fall-off sum runs from k_a + k_c [M] to k_a + k_b and
passes k_a + k_b / 2 where k_c [M] = k_b.  [M] is the air number density
P / (k_B T) with the exact SI k_B.
"""
import math

import numpy as np
import pytest

from paper_2501_00011_gb300 import synth

K_B = 1.380649e-23


def n_air(T, P):
    return P / (K_B * T) * 1e-6


def p_for(T, nm):
    """Pressure (Pa) at which the air number density is nm (cm^-3)."""
    return nm * 1e6 * K_B * T


def _kt(oracle_lib, rxs, T, P, theta=None):
    m = synth.mechanism_from_list(3, rxs, name="ratelaw")
    return oracle_lib.rate_constants(m, T, P, theta=theta)


def _troe(n_reac=2, **kw):
    reac = [0, 1][:n_reac]
    return dict(reac=reac, prod=[2], kind=synth.TROE, **kw)


@pytest.mark.parametrize("Fc", [0.6, 0.35, 1.0])
def test_troe_centre_of_falloff(oracle_lib, Fc):
    # k0 [M] = kinf: k = (kinf / 2) Fc
    T, k0, kinf = 300.0, 1e-30, 1e-11
    P = p_for(T, kinf / k0)
    kt = _kt(oracle_lib, [_troe(A=k0, A2=kinf, Fc=Fc)], T, P)
    # bimolecular: k~ = k n_air (mixing-ratio units)
    assert kt[0] / n_air(T, P) == pytest.approx(0.5 * Fc * kinf, rel=1e-13)


@pytest.mark.parametrize("N", [1.0, 2.0])
def test_troe_broadening_decades(oracle_lib, N):
    # with N, log10 x = +-N gives F = Fc^(1/2); F(x) = F(1/x)
    T, k0, kinf, Fc = 300.0, 1e-30, 1e-11, 0.6
    rx_fc = _troe(A=k0, A2=kinf, Fc=Fc, N=N)
    rx_1 = _troe(A=k0, A2=kinf, Fc=1.0, N=N)
    F = {}
    for dec in (-N, N, -2.7, 2.7):
        P = p_for(T, kinf / k0 * 10.0 ** dec)
        kt = _kt(oracle_lib, [rx_fc, rx_1], T, P)
        F[dec] = kt[0] / kt[1]
    assert F[N] == pytest.approx(math.sqrt(Fc), rel=1e-13)
    assert F[-N] == pytest.approx(math.sqrt(Fc), rel=1e-13)
    assert F[2.7] == pytest.approx(F[-2.7], rel=1e-13)
    assert math.sqrt(Fc) < F[2.7] < 1.0           # F -> 1 away from the centre


def test_troe_lindemann_limits(oracle_lib):
    T, kinf = 250.0, 3e-11
    rx = _troe(A=2e-30, B=-3.0, A2=kinf, B2=-0.5, Fc=1.0)
    k0 = 2e-30 * (T / 300.0) ** -3.0            # thermal twins carry the same temperature laws
    twins = [dict(reac=[0, 1], prod=[2], A=2e-30, B=-3.0), dict(reac=[0, 1], prod=[2], A=kinf, B=-0.5)]
    for P in (1.0, 3e3, 1e5, 1e9):
        nm = n_air(T, P)
        kt = _kt(oracle_lib, [rx] + twins, T, P)
        k, k0_t, kinf_t = (v / nm for v in kt)        # per-molecule rate constants
        assert k0_t == pytest.approx(k0, rel=1e-14)
        low = k0_t * nm
        assert 1.0 / k == pytest.approx(1.0 / low + 1.0 / kinf_t, rel=1e-13)
    # ends of the curve
    nm = n_air(T, 1e-6)
    k = _kt(oracle_lib, [rx], T, 1e-6)[0] / nm
    assert k == pytest.approx(k0 * nm, rel=1e-9)
    nm = n_air(T, 1e13)
    k = _kt(oracle_lib, [rx], T, 1e13)[0] / nm
    assert k == pytest.approx(kinf * (T / 300.0) ** -0.5, rel=1e-9)


def test_unimolecular_troe_has_no_number_density_factor(oracle_lib):
    # a thermal decomposition A (+M) -> products: k in s^-1 at the centre is kinf Fc / 2
    T, k0, kinf = 300.0, 1e-19, 1e-1
    P = p_for(T, kinf / k0)
    kt = _kt(oracle_lib, [_troe(n_reac=1, A=k0, A2=kinf, Fc=0.45)], T, P)
    assert kt[0] == pytest.approx(0.5 * 0.45 * kinf, rel=1e-13)


def test_pressure_sum_is_linear_in_number_density(oracle_lib):
    T = 260.0
    sum_rx = dict(reac=[0, 1], prod=[2], kind=synth.PRESSURE_SUM, A=3e-13, Ea=-460.0, B=0.5,
                  A2=2e-33, Ea2=-920.0, B2=-1.0)
    twin_a = dict(reac=[0, 1], prod=[2], A=3e-13, Ea=-460.0, B=0.5)
    twin_b = dict(reac=[0, 1], prod=[2], A=2e-33, Ea=-920.0, B=-1.0)
    ks = []
    for P in (1e3, 5e4, 1e5):
        nm = n_air(T, P)
        kt = _kt(oracle_lib, [sum_rx, twin_a, twin_b], T, P) / nm
        ks.append((nm, kt[0], kt[1], kt[2]))
    (n1, s1, a, b), (n2, s2, _, _), (n3, s3, _, _) = ks
    assert (s2 - s1) / (n2 - n1) == pytest.approx(b, rel=1e-9)
    assert (s3 - s2) / (n3 - n2) == pytest.approx(b, rel=1e-9)
    assert s1 - b * n1 == pytest.approx(a, rel=1e-9)


def test_falloff_sum_limits_and_midpoint(oracle_lib):
    T = 280.0
    rx = dict(reac=[0, 1], prod=[2], kind=synth.FALLOFF_SUM, A=2.4e-14, Ea=-460.0,
              A2=2.7e-17, Ea2=-2199.0, A3=6.5e-34, Ea3=-1335.0)
    twins = [dict(reac=[0, 1], prod=[2], A=2.4e-14, Ea=-460.0), dict(reac=[0, 1], prod=[2], A=2.7e-17, Ea=-2199.0),
             dict(reac=[0, 1], prod=[2], A=6.5e-34, Ea=-1335.0)]
    nm1 = n_air(T, 1e5)
    _, ka, kb, kc = _kt(oracle_lib, [rx] + twins, T, 1e5) / nm1
    # k_c [M] = k_b
    P = p_for(T, kb / kc)
    k = _kt(oracle_lib, [rx], T, P)[0] / n_air(T, P)
    assert k == pytest.approx(ka + 0.5 * kb, rel=1e-13)
    k = _kt(oracle_lib, [rx], T, 1e-4)[0] / n_air(T, 1e-4)
    assert k == pytest.approx(ka + kc * n_air(T, 1e-4), rel=1e-12)
    k = _kt(oracle_lib, [rx], T, 1e12)[0] / n_air(T, 1e12)
    assert k == pytest.approx(ka + kb, rel=1e-9)


def test_theta_scales_every_kind(oracle_lib):
    T, P = 270.0, 4e4
    rxs = [_troe(A=1e-30, A2=1e-11), dict(reac=[0, 1], prod=[2], kind=synth.PRESSURE_SUM, A=1e-13, A2=1e-33),
           dict(reac=[0, 1], prod=[2], kind=synth.FALLOFF_SUM, A=1e-14, A2=1e-17, A3=1e-33)]
    th = np.array([0.3, -0.2, 0.7])
    k0 = _kt(oracle_lib, rxs, T, P)
    k1 = _kt(oracle_lib, rxs, T, P, theta=th)
    np.testing.assert_allclose(k1, k0 * np.exp(th), rtol=1e-15)


def test_pressure_workload_spans_the_falloff(oracle_lib):
    # the workload's Troe reactions run from below the centre of their curves to above it
    wl = synth.workload_pressure(200)
    m = wl.mech
    troe = np.nonzero(m.kind == synth.TROE)[0]
    assert troe.size == 12 and np.count_nonzero(m.kind == synth.PRESSURE_SUM) == 3
    assert np.count_nonzero(m.kind == synth.FALLOFF_SUM) == 3
    x = []
    for c in range(wl.cells.n_cells):
        T, P = wl.cells.T[c], wl.cells.P[c]
        x.append(m.A[troe] * (T / 300.0) ** m.B[troe] * n_air(T, P)
                 / (m.ext[troe, synth.EXT_A2] * (T / 300.0) ** m.ext[troe, synth.EXT_B2]))
    x = np.array(x)
    assert x.min() < 0.1 and x.max() > 10.0


def test_hand_worked_rate_constants(oracle_lib):
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "pressure_rate_laws.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, *v = line.split()
                vals[k] = np.array([float(x) for x in v])
    rxs = [dict(reac=[0, 1], prod=[2], kind=synth.TROE, A=1e-30, A2=1e-11, Fc=0.64, N=1.0),
           dict(reac=[0, 1], prod=[2], kind=synth.PRESSURE_SUM, A=1e-12, A2=1e-32),
           dict(reac=[0, 1], prod=[2], kind=synth.FALLOFF_SUM, A=1e-13, A2=1e-12, A3=1e-32)]
    kt = _kt(oracle_lib, rxs, float(vals["T"][0]), float(vals["P"][0]))
    # P is given to 7 digits, so n_air (and each k~) carries a relative error of about 1e-8
    np.testing.assert_allclose(kt, vals["kt"], rtol=1e-7)
