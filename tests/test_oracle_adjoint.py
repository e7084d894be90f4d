"""Pins of the oracle's discrete adjoint.

The adjoint is the exact adjoint of the frozen-control map of a tape: the
integrator's own arithmetic with its step sizes, orders, corrector iteration
counts, iteration matrices and projections held fixed.  It is checked against
things other than itself: the map against the integrator it replays (they must
agree bit for bit), the tangent-linear model through the dot-product identity
<lam, T v> = <T^T lam, v>, central finite differences of the map, and the
closed form of backward Euler with a fixed step on A -> B
(A_n = A_0 (1 + h k)^-n).
"""
import math

import numpy as np
import pytest

from paper_2501_00011_gb300 import synth


def _setup(mech, n_steps, rtol, atol, seed, c=0):
    import oracle
    cells = synth.random_cells(mech.n_species, 3, T_range=(230.0, 300.0), P_range=(3e4, 1e5), seed=seed)
    theta0 = np.zeros(mech.n_reactions)
    kt = oracle.rate_constants(mech, cells.T[c], cells.P[c], theta=theta0)
    y0 = cells.y[:, c].copy()
    y, stats, tape = oracle.integrate_steps(mech, kt, y0, 600.0, n_steps, rtol, atol)
    assert all(s["status"] == 0 for s in stats)
    return cells, kt, y0, y, tape


@pytest.mark.parametrize("which", ["small", "tropo"])
def test_replay_reproduces_forward(oracle_lib, which):
    m = synth.mechanism_small() if which == "small" else synth.mechanism_tropo()
    cells, kt, y0, y, tape = _setup(m, 3, 1e-6 if which == "small" else 1e-4, 1e-14 if which == "small" else 1e-10,
                                    seed=21)
    assert np.any(tape.kind == 4) and np.any(tape.kind == 5)
    yr, ys = oracle_lib.replay(m, kt, y0, tape, keep_steps=True)
    # the same operations in the same order: identical bits
    assert np.array_equal(yr, y)
    steps = np.flatnonzero(tape.kind == 2)
    assert np.array_equal(ys[steps], tape.y[steps])


@pytest.mark.parametrize("which", ["small", "tropo"])
def test_adjoint_dot_product_identity(oracle_lib, which):
    m = synth.mechanism_small() if which == "small" else synth.mechanism_tropo()
    cells, kt, y0, y, tape = _setup(m, 2 if which == "small" else 1, 1e-5 if which == "small" else 1e-4,
                                    1e-14 if which == "small" else 1e-10, seed=22)
    rng = np.random.default_rng(3)
    lam = rng.standard_normal(m.n_species)
    dy0 = rng.standard_normal(m.n_species) * y0
    dth = rng.standard_normal(m.n_reactions)
    Tv = oracle_lib.tangent(m, kt, y0, tape, dy0, dth)
    ly0, g = oracle_lib.adjoint(m, kt, y0, tape, lam)
    lhs = lam @ Tv
    rhs = ly0 @ dy0 + g @ dth
    scale = np.abs(lam) @ np.abs(Tv) + np.abs(ly0) @ np.abs(dy0) + np.abs(g) @ np.abs(dth)
    assert abs(lhs - rhs) <= 1e-10 * scale


def test_adjoint_matches_central_differences_small(oracle_lib):
    m = synth.mechanism_small()
    n_steps = 4
    cells, kt, y0, y, tape = _setup(m, n_steps, 1e-5, 1e-14, seed=23)
    w = synth.loss_weights(m.n_species, 1)[:, 0]
    ly0, g = oracle_lib.adjoint(m, kt, y0, tape, w)
    T, P = cells.T[0], cells.P[0]
    eps = 1e-6
    # rounding floor of a central difference of L = w . y (and of the replay's
    # rounding-level convergence): a few hundred eps * |L| / step
    L0 = abs(w @ y)
    floor_th = 1e3 * np.finfo(float).eps * L0 / eps
    for j in range(m.n_reactions):
        th = np.zeros(m.n_reactions)
        th[j] = eps
        lp = w @ oracle_lib.replay(m, oracle_lib.rate_constants(m, T, P, theta=th), y0, tape, kt_M=kt)
        th[j] = -eps
        lm = w @ oracle_lib.replay(m, oracle_lib.rate_constants(m, T, P, theta=th), y0, tape, kt_M=kt)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[j]) <= 1e-5 * abs(g[j]) + floor_th, (j, fd, g[j])
    for i in range(m.n_species):
        e = eps * abs(y0[i])
        yp, ym = y0.copy(), y0.copy()
        yp[i] += e
        ym[i] -= e
        fd = (w @ oracle_lib.replay(m, kt, yp, tape) - w @ oracle_lib.replay(m, kt, ym, tape)) / (2 * e)
        assert abs(fd - ly0[i]) <= 1e-5 * abs(ly0[i]) + 1e3 * np.finfo(float).eps * L0 / e, (i, fd, ly0[i])


def test_adjoint_directional_differences_tropo(oracle_lib):
    m = synth.mechanism_tropo()
    cells, kt, y0, y, tape = _setup(m, 2, 1e-4, 1e-10, seed=24)
    w = synth.loss_weights(m.n_species, 1)[:, 0]
    ly0, g = oracle_lib.adjoint(m, kt, y0, tape, w)
    T, P = cells.T[0], cells.P[0]
    rng = np.random.default_rng(5)
    eps = 1e-6
    for _ in range(2):
        v = rng.standard_normal(m.n_reactions)
        lp = w @ oracle_lib.replay(m, oracle_lib.rate_constants(m, T, P, theta=eps * v), y0, tape, kt_M=kt)
        lm = w @ oracle_lib.replay(m, oracle_lib.rate_constants(m, T, P, theta=-eps * v), y0, tape, kt_M=kt)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g @ v) <= 1e-5 * np.abs(g) @ np.abs(v)
        u = rng.standard_normal(m.n_species) * y0
        fd = (w @ oracle_lib.replay(m, kt, y0 + eps * u, tape) - w @ oracle_lib.replay(m, kt, y0 - eps * u, tape)) / (2 * eps)
        assert abs(fd - ly0 @ u) <= 1e-5 * np.abs(ly0) @ np.abs(u)


def test_adjoint_backward_euler_closed_form(oracle_lib):
    # A -> B with rate k, backward Euler with fixed h: A_n = A_0 (1 + h k)^-n, so
    # dA_n/dA_0 = (1 + hk)^-n and dA_n/dtheta = -n h k A_n / (1 + h k).
    k = 0.05
    m = synth.mechanism_from_list(2, [dict(reac=[0], prod=[1], A=k)])
    kt = oracle_lib.rate_constants(m, 300.0, 1e5)
    y0 = np.array([0.7, 0.1])
    h, n = 4.0, 25
    y, st, tape = oracle_lib.integrate(m, kt, y0, n * h, 1e-6, 1e-12, fixed_h=h, fixed_order=1,
                                       newton_tol=1e-8, newton_maxiter=10, tape_cap=200)
    An = y0[0] * (1 + h * k) ** (-n)
    assert y[0] == pytest.approx(An, rel=1e-12)
    ly0, g = oracle_lib.adjoint(m, kt, y0, tape, np.array([1.0, 0.0]))
    assert ly0[0] == pytest.approx((1 + h * k) ** (-n), rel=1e-11)
    assert abs(ly0[1]) <= 1e-14
    assert g[0] == pytest.approx(-n * h * k * An / (1 + h * k), rel=1e-10)


def test_binding_accepts_strided_inputs(oracle_lib):
    # column slices of [S, C] arrays are not contiguous: the binding must pass
    # copies that stay alive for the whole call
    m = synth.mechanism_small()
    cells, kt, y0, y, tape = _setup(m, 2, 1e-6, 1e-14, seed=25)
    w = synth.loss_weights(m.n_species, 3)
    Y = np.stack([y0, y0, y0], axis=1)
    ref = oracle_lib.adjoint(m, kt, y0, tape, w[:, 1].copy())
    got = oracle_lib.adjoint(m, kt, Y[:, 1], tape, w[:, 1])
    assert np.array_equal(ref[0], got[0]) and np.array_equal(ref[1], got[1])
    dv = np.stack([y0, y0], axis=1) * 1e-3
    t_ref = oracle_lib.tangent(m, kt, y0, tape, dv[:, 0].copy(), np.zeros(m.n_reactions))
    t_got = oracle_lib.tangent(m, kt, Y[:, 2], tape, dv[:, 0], np.zeros(m.n_reactions))
    assert np.array_equal(t_ref, t_got)
    assert np.array_equal(oracle_lib.replay(m, kt, Y[:, 0], tape), y)
