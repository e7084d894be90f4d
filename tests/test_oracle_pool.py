"""The oracle run over cell shards in spawned worker processes gives exactly
the single-process oracle's results (cells are independent), with and without
host work between steps, and the pooled adjoint equals the per-cell one."""
import numpy as np

from oracle import pool
from paper_2501_00011_gb300 import synth


def _between(y, T, step):
    # a host step acting on each cell alone (module level, so workers can unpickle it)
    y *= 0.95 + 0.01 * step
    T += 1.0


def test_pool_solve_equals_sequential(oracle_lib):
    wl = synth.workload_batching(37)
    ys, ss = oracle_lib.solve_cells(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol)
    yp, sp = pool.solve(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol, workers=3, chunks_per_worker=2)
    assert np.array_equal(ys, yp) and np.array_equal(ss, sp)


def test_pool_solve_steps_with_host_work(oracle_lib):
    wl = synth.workload_tropo(23)
    cur = synth.subset(wl.cells, np.arange(23))
    for k in range(3):
        cur.y, st = oracle_lib.solve_cells(wl.mech, cur, wl.dt, wl.rtol, wl.atol)
        if k < 2:
            _between(cur.y, cur.T, k)
    yp, sp = pool.solve(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol, n_steps=3, between=_between, workers=2)
    assert np.array_equal(cur.y, yp) and np.array_equal(st, sp)
    # the caller's arrays are not modified
    assert np.array_equal(wl.cells.T, synth.workload_tropo(23).cells.T)


def test_pool_adjoint_equals_per_cell(oracle_lib):
    wl = synth.workload_adjoint(5)
    tapes, lam = [], synth.loss_weights(wl.mech.n_species, 5)
    for k in range(5):
        kt = oracle_lib.rate_constants(wl.mech, wl.cells.T[k], wl.cells.P[k])
        _, _, tape = oracle_lib.integrate_steps(wl.mech, kt, wl.cells.y[:, k], wl.dt, 2, wl.rtol, wl.atol)
        tapes.append(tape)
    ly0, g = pool.adjoint(wl.mech, wl.cells, tapes, lam, workers=2, chunks_per_worker=1)
    for k in range(5):
        kt = oracle_lib.rate_constants(wl.mech, wl.cells.T[k], wl.cells.P[k])
        l1, g1 = oracle_lib.adjoint(wl.mech, kt, wl.cells.y[:, k], tapes[k], lam[:, k])
        assert np.array_equal(ly0[:, k], l1) and np.array_equal(g[k], g1)


def test_pool_workers_reused_and_forward_adjoint(oracle_lib):
    wl = synth.workload_adjoint(6)
    lam = synth.loss_weights(wl.mech.n_species, 6)
    with pool.Workers(2) as ex:
        y1, s1 = pool.solve(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol, executor=ex)
        y2, s2 = pool.solve(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol, executor=ex)
        ly0, g = pool.forward_adjoint(wl.mech, wl.cells, wl.dt, 2, wl.rtol, wl.atol, lam, executor=ex)
    assert np.array_equal(y1, y2) and np.array_equal(s1, s2)
    g_ref = np.zeros(wl.mech.n_reactions)
    for k in range(6):
        kt = oracle_lib.rate_constants(wl.mech, wl.cells.T[k], wl.cells.P[k])
        _, _, tape = oracle_lib.integrate_steps(wl.mech, kt, wl.cells.y[:, k], wl.dt, 2, wl.rtol, wl.atol)
        l1, g1 = oracle_lib.adjoint(wl.mech, kt, wl.cells.y[:, k], tape, lam[:, k])
        assert np.array_equal(ly0[:, k], l1)
        g_ref += g1
    np.testing.assert_allclose(g, g_ref, rtol=1e-13, atol=0)
