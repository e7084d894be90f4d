"""Full-size workloads on the GPU, checked on sampled cells against the oracle.

Each test runs a whole batch at its benchmark size and launch configuration
(10,000 cells, persistent FP64; 50,000 cells with per-cell photolysis over six
graph-captured steps with an autotuned launch shape; 50,000 cells with the
FP32 LU; 2,048 cells through the discrete adjoint) and compares a sample of
cells, which the oracle computes one by one, with the parity rules of
parity_util.  Properties that hold at any size (every cell solved; graph and
single steps identical; launch shape without effect on results) are checked
on the whole batch.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_00011_gb300 import synth  # noqa: E402

from parity_util import FLOOR, compare, oracle_steps, sample_cells  # noqa: E402


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


def _batch(cg, mech, wl, **opts):
    c = cg.Cells(mech, wl.cells.n_cells, rtol=wl.rtol, atol=wl.atol, **opts)
    c.set_state(wl.cells.T, wl.cells.P, wl.cells.y)
    if wl.cells.J is not None:
        c.set_photolysis(wl.cells.J)
    return c


def test_tropo_10k_persistent(oracle_lib, cg, tropo):
    wl = synth.workload_tropo(10_000)
    c = _batch(cg, tropo, wl, driver="persistent")
    c.solve_step(wl.dt)
    y, st = c.get_state(), c.get_stats()
    assert np.all(st["status"] == 0)
    idx = sample_cells(wl.cells.n_cells, 64, seed=1)
    sub = synth.subset(wl.cells, idx)
    yo, so = oracle_steps(oracle_lib, wl, sub, 1)
    err, flips, odd = compare(y[:, idx], st[idx], yo, so, oracle_lib, wl, sub)
    print(f"10k persistent FP64, {idx.size} sampled cells: max rel err {err:.2e}, flips {flips}, rounding-limited {odd}")


def test_one_million_cells(oracle_lib, cg, tropo):
    # a batch 100x the benchmark's (y alone 576 MB): one persistent launch, a million
    # queue pops; sampled cells against the oracle, every cell converged and finite
    wl = synth.workload_tropo(1_000_000)
    c = _batch(cg, tropo, wl, driver="persistent")
    c.solve_step(wl.dt)
    y, st = c.get_state(), c.get_stats()
    assert np.all(st["status"] == 0) and np.all(np.isfinite(y))
    idx = sample_cells(wl.cells.n_cells, 12, seed=7)
    sub = synth.subset(wl.cells, idx)
    yo, so = oracle_steps(oracle_lib, wl, sub, 1)
    compare(y[:, idx], st[idx], yo, so, oracle_lib, wl, sub)
    c.close()


def test_batching_50k_graph_autotuned(oracle_lib, cg, tropo):
    wl = synth.workload_batching(50_000)
    c = _batch(cg, tropo, wl, driver="persistent")
    w, b = c.autotune(wl.dt)
    assert 1 <= w <= 12 and b >= 1
    c.solve_steps(wl.dt, wl.n_steps)
    y, st = c.get_state(), c.get_stats()
    assert np.all(st["status"] == 0)
    # uneven work: night cells and warm/cold cells take very different step counts
    assert st["steps"].max() >= 2 * max(1, np.percentile(st["steps"], 5))
    idx = sample_cells(wl.cells.n_cells, 40, seed=2)
    sub = synth.subset(wl.cells, idx)
    yo, so = oracle_steps(oracle_lib, wl, sub, wl.n_steps)
    err, flips, odd = compare(y[:, idx], st[idx], yo, so, oracle_lib, wl, sub, n_steps=wl.n_steps)
    print(f"50k batching, 6 graph steps, shape w={w} b={b}: max rel err {err:.2e}, flips {flips}, "
          f"rounding-limited {odd}; steps per cell (last step) min/median/max "
          f"{st['steps'].min()}/{int(np.median(st['steps']))}/{st['steps'].max()}")


@pytest.mark.parametrize("driver", ["plain", "persistent"])
def test_graph_equals_single_steps(cg, tropo, driver):
    wl = synth.workload_batching(3001)
    a = _batch(cg, tropo, wl, driver=driver)
    a.solve_steps(wl.dt, 3)
    ya, sa = a.get_state(), a.get_stats()
    b = _batch(cg, tropo, wl, driver=driver)
    for _ in range(3):
        b.solve_step(wl.dt)
    assert np.array_equal(ya, b.get_state()) and np.array_equal(sa, b.get_stats())
    # replaying the captured graph on a reset state gives the same result again
    a.set_state(wl.cells.T, wl.cells.P, wl.cells.y)
    a.solve_steps(wl.dt, 3)
    assert np.array_equal(ya, a.get_state())
    # a different step count re-captures
    a.set_state(wl.cells.T, wl.cells.P, wl.cells.y)
    a.solve_steps(wl.dt, 1)
    b.set_state(wl.cells.T, wl.cells.P, wl.cells.y)
    b.solve_step(wl.dt)
    assert np.array_equal(a.get_state(), b.get_state())


def test_autotune_keeps_state_and_results(cg, tropo):
    wl = synth.workload_batching(5000)
    a = _batch(cg, tropo, wl, driver="persistent")
    y_before = a.get_state()
    w, b = a.autotune(wl.dt, 2000)
    assert np.array_equal(a.get_state(), y_before)
    a.solve_step(wl.dt)
    ref = _batch(cg, tropo, wl, driver="persistent", cells_per_block=1, blocks_per_sm=1)
    ref.solve_step(wl.dt)
    assert np.array_equal(a.get_state(), ref.get_state())
    p = _batch(cg, tropo, wl, driver="plain")
    wp, bp = p.autotune(wl.dt, 2000)
    assert bp == 0 and wp >= 1
    p.solve_step(wl.dt)
    assert np.array_equal(p.get_state(), ref.get_state())


def test_fp32_lu_50k(oracle_lib, cg, tropo):
    # accuracy bound of the FP32-LU form (see test_gpu_parity): within 50
    # tolerance units of the FP64 oracle and as accurate as it against a tight
    # reference, on a sample of the full 50,000-cell batch
    wl = synth.workload_precision(50_000)
    c32 = _batch(cg, tropo, wl, driver="persistent", lu_precision=32)
    c32.solve_step(wl.dt)
    y, st = c32.get_state(), c32.get_stats()
    c64 = _batch(cg, tropo, wl, driver="persistent", lu_precision=64)
    c64.solve_step(wl.dt)
    st64 = c64.get_stats()
    assert np.all(st["status"] == 0) and np.all(st64["status"] == 0)
    idx = sample_cells(wl.cells.n_cells, 40, seed=3)
    sub = synth.subset(wl.cells, idx)
    yo, so = oracle_lib.solve_cells(wl.mech, sub, wl.dt, wl.rtol, wl.atol)
    yt, stt = oracle_lib.solve_cells(wl.mech, sub, wl.dt, 1e-10, 1e-18)
    assert np.all(stt["status"] == 0)
    ys = y[:, idx]
    tol = wl.rtol * np.abs(yo) + wl.atol
    assert (np.abs(ys - yo) / tol).max() <= 50.0
    acc32 = (np.abs(ys - yt) / (wl.rtol * np.abs(yt) + wl.atol)).max(axis=0)
    acc64 = (np.abs(yo - yt) / (wl.rtol * np.abs(yt) + wl.atol)).max(axis=0)
    assert acc32.max() <= 1.25 * acc64.max() and np.median(acc32) <= 1.1 * np.median(acc64)
    # the cells where the two forms differ most: there too FP32 is as accurate as FP64
    y64 = c64.get_state()
    diff = (np.abs(y - y64) / (wl.rtol * np.abs(y64) + wl.atol)).max(axis=0)
    worst = np.argsort(-diff)[:10]
    ywt, swt = oracle_lib.solve_cells(wl.mech, synth.subset(wl.cells, worst), wl.dt, 1e-10, 1e-18)
    assert np.all(swt["status"] == 0)
    unit = wl.rtol * np.abs(ywt) + wl.atol
    w32 = (np.abs(y[:, worst] - ywt) / unit).max(axis=0)
    w64 = (np.abs(y64[:, worst] - ywt) / unit).max(axis=0)
    assert w32.max() <= 1.25 * w64.max() and np.median(w32) <= 1.1 * np.median(w64), (w32, w64)
    assert diff.max() <= 50.0
    rel = np.where(np.abs(yo) > FLOOR, np.abs(ys - yo) / np.maximum(np.abs(yo), 1e-300), 0.0).max(axis=1)
    print(f"fp32 LU 50k: per-species max rel err vs FP64 oracle on {idx.size} cells: median {np.median(rel):.2e}, "
          f"max {rel.max():.2e}; Newton iterations {st['newton_iters'].sum() / st64['newton_iters'].sum():.3f}x "
          f"the FP64 GPU path's over all cells")


def test_adjoint_2048_sampled(oracle_lib, cg, tropo):
    # the whole 2,048-cell batch runs forward (4 steps) and backward; the loss
    # weights are nonzero on sampled cells only, so dL/dtheta is their sum and
    # the oracle adjoint of each sampled cell's GPU tape gives it exactly
    wl = synth.workload_adjoint(2048)
    c = _batch(cg, tropo, wl, driver="persistent", record_adjoint=True)
    for _ in range(wl.n_steps):
        c.solve_step(wl.dt)
    idx = sample_cells(wl.cells.n_cells, 8, seed=4)
    w = np.zeros((wl.mech.n_species, wl.cells.n_cells))
    w[:, idx] = synth.loss_weights(wl.mech.n_species, wl.cells.n_cells)[:, idx]
    gth, gy0, n_bad = c.sensitivity(w)
    assert n_bad == 0
    assert np.all(gy0[:, np.setdiff1d(np.arange(wl.cells.n_cells), idx)] == 0.0)
    g_sum = np.zeros(wl.mech.n_reactions)
    for k in idx:
        kind, q, val, rows = c.get_tape(k)
        has_row = (kind == 0) | (kind == 4) | (kind == 5)
        yrow = np.zeros((kind.size, wl.mech.n_species))
        yrow[has_row] = rows
        tape = oracle_lib.Tape(kind, q, val, yrow)
        kt = oracle_lib.rate_constants(wl.mech, wl.cells.T[k], wl.cells.P[k])
        ly0, g = oracle_lib.adjoint(wl.mech, kt, wl.cells.y[:, k], tape, w[:, k])
        g_sum += g
        assert np.all(np.abs(gy0[:, k] - ly0) <= 1e-8 * np.abs(ly0) + 1e-12 * np.abs(ly0).max()), k
    assert np.all(np.abs(gth - g_sum) <= 1e-8 * np.abs(g_sum) + 1e-12 * np.abs(g_sum).max())
