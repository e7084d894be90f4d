"""Host-resident state through the chunked pipeline (chem_pipeline_*).

The pipeline must give, bit for bit, what one device batch gives over the
same steps with the host's work applied between them: cells are independent,
so how they are split into chunks, streams and launches cannot change a
result.  Also: the callback sees every chunk of every step once, in order;
a callback can stop the run, and an exception in it reaches the caller.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_00011_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_00011_gb300 import build, chemgpu
    build.build()
    torch.cuda.init()
    chemgpu.load()
    return chemgpu


@pytest.fixture(scope="module")
def tropo(cg):
    return cg.Mechanism(synth.mechanism_tropo())


def _host_step(y, T, c0, c1, step):
    """A stand-in for the host model's work on a chunk between chemistry steps."""
    y[:, c0:c1] *= 0.9 + 0.01 * step
    y[:5, c0:c1] += 1e-9
    T[c0:c1] += 1.5


def _host_step_cells(y, T, step):
    """The same host work on every column of a batch (the oracle's runs)."""
    _host_step(y, T, 0, y.shape[1], step)


def _reference(cg, mech, wl, cells, n_steps, driver, J=None, prec=64):
    c = cg.Cells(mech, cells.n_cells, rtol=wl.rtol, atol=wl.atol, driver=driver, lu_precision=prec)
    y, T, P = cells.y.copy(), cells.T.copy(), cells.P.copy()
    st = None
    for step in range(n_steps):
        c.set_state(T, P, y)
        if J is not None:
            c.set_photolysis(J)
        c.solve_step(wl.dt)
        y = c.get_state()
        st = c.get_stats()
        _host_step(y, T, 0, cells.n_cells, step)
    c.close()
    return y, T, st


@pytest.mark.parametrize("n,K,driver,prec", [(301, 4, "persistent", 64), (301, 3, "plain", 64), (7, 7, "persistent", 64),
                                             (50, 1, "persistent", 64), (120, 3, "persistent", 32)])
def test_pipeline_equals_one_batch(cg, tropo, n, K, driver, prec):
    wl = synth.workload_tropo(n)
    n_steps = 3
    yr, Tr, sr = _reference(cg, tropo, wl, wl.cells, n_steps, driver, prec=prec)
    y = cg.pinned_empty(wl.cells.y.shape)
    y[:] = wl.cells.y
    T, P = wl.cells.T.copy(), wl.cells.P.copy()
    seen = []

    def fn(c0, c1, step):
        seen.append((step, c0, c1))
        _host_step(y, T, c0, c1, step)

    p = cg.Pipeline(tropo, n, K, rtol=wl.rtol, atol=wl.atol, driver=driver, lu_precision=prec)
    st = p.run(T, P, y, wl.dt, n_steps, fn=fn, stats=True)
    p.close()
    assert np.array_equal(y, yr) and np.array_equal(T, Tr) and np.array_equal(st, sr)
    # every chunk of every step once, steps in order, chunks in order within a step
    assert [s for s, _, _ in seen] == sorted(s for s, _, _ in seen)
    for step in range(n_steps):
        chunks = [(a, b) for s, a, b in seen if s == step]
        assert chunks[0][0] == 0 and chunks[-1][1] == n and len(chunks) == K
        assert all(b == a2 for (_, b), (a2, _) in zip(chunks, chunks[1:]))
        sizes = [b - a for a, b in chunks]
        assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("K,driver", [(4, "persistent"), (3, "plain")])
def test_pipeline_matches_oracle(oracle_lib, cg, tropo, K, driver):
    # the pipeline with the host's work between chemistry steps, cell by cell against
    # the oracle applying the same work between its own solves: solve, host work,
    # solve, host work, solve (per-cell photolysis), by the parity rules
    from parity_util import compare
    wl = synth.workload_batching(301)
    n_steps = 3
    y = cg.pinned_empty(wl.cells.y.shape)
    y[:] = wl.cells.y
    T, P, J = wl.cells.T.copy(), wl.cells.P.copy(), wl.cells.J.copy()

    def fn(c0, c1, step):
        if step + 1 < n_steps:
            _host_step(y, T, c0, c1, step)

    p = cg.Pipeline(tropo, wl.cells.n_cells, K, rtol=wl.rtol, atol=wl.atol, driver=driver)
    st = p.run(T, P, y, wl.dt, n_steps, fn=fn, J=J, stats=True)
    p.close()
    from parity_util import oracle_steps
    yo, so = oracle_steps(oracle_lib, wl, wl.cells, n_steps, between=_host_step_cells)
    rep = compare(np.array(y), st, yo, so, oracle_lib, wl, wl.cells, n_steps=n_steps, between=_host_step_cells,
                  label=f"pipeline {K} chunks {driver}")
    print(f"pipeline, {K} chunks, {driver}, host work between 3 steps:", rep.summary())


def test_pipeline_per_cell_photolysis_and_pageable_memory(cg, tropo):
    wl = synth.workload_batching(97)
    yr, Tr, sr = _reference(cg, tropo, wl, wl.cells, 2, "persistent", J=wl.cells.J)
    y, T, P = wl.cells.y.copy(), wl.cells.T.copy(), wl.cells.P.copy()     # pageable host memory
    p = cg.Pipeline(tropo, 97, 5, rtol=wl.rtol, atol=wl.atol)
    st = p.run(T, P, y, wl.dt, 2, fn=lambda c0, c1, s: _host_step(y, T, c0, c1, s), J=wl.cells.J.copy(), stats=True)
    assert np.array_equal(y, yr) and np.array_equal(st, sr)


def test_pipeline_without_callback_and_stop(cg, tropo):
    wl = synth.workload_tropo(40)
    y0 = wl.cells.y.copy()
    y, T, P = y0.copy(), wl.cells.T.copy(), wl.cells.P.copy()
    p = cg.Pipeline(tropo, 40, 4, rtol=wl.rtol, atol=wl.atol)
    p.run(T, P, y, wl.dt, 2)
    c = cg.Cells(tropo, 40, rtol=wl.rtol, atol=wl.atol, driver="persistent")
    c.set_state(wl.cells.T, wl.cells.P, y0)
    c.solve_step(wl.dt)
    c.solve_step(wl.dt)
    assert np.array_equal(y, c.get_state())
    # a callback that asks to stop, and one that raises
    with pytest.raises(cg.ChemError, match="stopped"):
        p.run(T, P, y, wl.dt, 3, fn=lambda c0, c1, s: s == 1 and c0 > 0)

    def boom(c0, c1, s):
        raise ValueError("host model failed")
    with pytest.raises(ValueError, match="host model failed"):
        p.run(T, P, y, wl.dt, 2, fn=boom)
    # the pipeline is still usable afterwards
    p.run(T, P, y, wl.dt, 1)
    assert np.all(np.isfinite(y))


def test_pipeline_argument_checks(cg, tropo):
    with pytest.raises(cg.ChemError):
        cg.Pipeline(tropo, 3, 4)                 # more chunks than cells
    with pytest.raises(cg.ChemError):
        cg.Pipeline(tropo, 10, 0)
    p = cg.Pipeline(tropo, 0, 1)
    p.run(np.zeros(0), np.zeros(0), np.zeros((72, 0)), 600.0, 1)
    p = cg.Pipeline(tropo, 8, 2)
    wl = synth.workload_tropo(8)
    with pytest.raises(cg.ChemError):
        p.run(wl.cells.T, wl.cells.P, np.asfortranarray(wl.cells.y), 600.0, 1)   # not C-contiguous
    with pytest.raises(cg.ChemError):
        p.run(wl.cells.T, wl.cells.P, wl.cells.y.copy(), -1.0, 1)
