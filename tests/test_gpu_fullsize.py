"""Full-size workloads on the GPU, every cell checked against the oracle.

Each test runs a whole batch at its benchmark size and launch configuration
(10,000 cells, persistent FP64; 50,000 cells with per-cell photolysis over six
graph-captured steps with an autotuned launch shape; 50,000 cells with the
FP32 LU; 2,048 cells through the discrete adjoint) and compares every cell
with the oracle, which runs on all host cores (oracle.pool), by the parity
rules of parity_util.  The counts of flipped and rounding-limited cells are
part of every assertion message and printed.  A batch of a million cells is
checked on a sample (the oracle would need minutes of every core for it).
Properties that hold at any size (every cell solved; graph and single steps
identical; launch shape without effect on results) are checked on the whole
batch.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import pool  # noqa: E402
from paper_2501_00011_gb300 import synth  # noqa: E402

from parity_util import FLOOR, compare, oracle_steps, sample_cells  # noqa: E402

# Flipped plus rounding-limited cells allowed at full size: 0.6% of the cells.
# Measured: 34 of the 10,000 headline cells (0.34%), 107 of the 50,000 batching
# cells after six steps (0.21%), 8 of the 2,048 adjoint cells (0.39%).
MAX_ODD_FRAC = 0.006


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


def test_tropo_10k_persistent_all_cells(oracle_lib, cg, tropo):
    wl = synth.workload_tropo(10_000)
    c = _batch(cg, tropo, wl, driver="persistent")
    c.solve_step(wl.dt)
    y, st = c.get_state(), c.get_stats()
    assert np.all(st["status"] == 0)
    yo, so = oracle_steps(oracle_lib, wl, wl.cells, 1)
    rep = compare(y, st, yo, so, oracle_lib, wl, wl.cells, max_odd_frac=MAX_ODD_FRAC, label="10k persistent FP64")
    print("10k persistent FP64, all cells:", rep.summary())


def test_one_million_cells(oracle_lib, cg, tropo):
    # a batch 100x the benchmark's (y alone 576 MB): one persistent launch, a million
    # queue pops; sampled cells against the oracle, every cell converged and finite
    wl = synth.workload_tropo(1_000_000)
    c = _batch(cg, tropo, wl, driver="persistent")
    c.solve_step(wl.dt)
    y, st = c.get_state(), c.get_stats()
    assert np.all(st["status"] == 0) and np.all(np.isfinite(y))
    idx = sample_cells(wl.cells.n_cells, 64, seed=7)
    sub = synth.subset(wl.cells, idx)
    yo, so = oracle_steps(oracle_lib, wl, sub, 1)
    compare(y[:, idx], st[idx], yo, so, oracle_lib, wl, sub, label="1M sampled")
    c.close()


def test_batching_50k_graph_autotuned_all_cells(oracle_lib, cg, tropo):
    wl = synth.workload_batching(50_000)
    c = _batch(cg, tropo, wl, driver="persistent")
    w, b = c.autotune(wl.dt)
    assert 1 <= w <= 12 and b >= 1
    c.solve_steps(wl.dt, wl.n_steps)
    y, st = c.get_state(), c.get_stats()
    assert np.all(st["status"] == 0)
    # uneven work: night cells and warm/cold cells take very different step counts
    assert st["steps"].max() >= 2 * max(1, np.percentile(st["steps"], 5))
    yo, so = oracle_steps(oracle_lib, wl, wl.cells, wl.n_steps)
    rep = compare(y, st, yo, so, oracle_lib, wl, wl.cells, n_steps=wl.n_steps, max_odd_frac=MAX_ODD_FRAC,
                  label="50k batching, 6 graph steps")
    print(f"50k batching, 6 graph steps, shape w={w} b={b}, all cells: {rep.summary()}; steps per cell "
          f"(last step) min/median/max {st['steps'].min()}/{int(np.median(st['steps']))}/{st['steps'].max()}")


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


def test_staging_fallback_counter(cg, tropo):
    # stage_wait = -1: every block skips its bounded wait for the staged tables and
    # reads them from global memory (the same bytes): identical results, one
    # fallback per block (5 cells per block, one block per SM), counted per call
    # over all its steps; no copy is left unfinished
    wl = synth.workload_batching(3001)
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = min(n_sm, -(-wl.cells.n_cells // 5))
    a = _batch(cg, tropo, wl, driver="persistent", cells_per_block=5, blocks_per_sm=1)
    a.solve_step(wl.dt)
    assert a.staging_fallbacks() == (0, 0)
    b = _batch(cg, tropo, wl, driver="persistent", cells_per_block=5, blocks_per_sm=1, stage_wait=-1)
    b.solve_step(wl.dt)
    assert b.staging_fallbacks() == (blocks, 0)
    assert np.array_equal(a.get_state(), b.get_state()) and np.array_equal(a.get_stats(), b.get_stats())
    b.set_state(wl.cells.T, wl.cells.P, wl.cells.y)
    b.solve_steps(wl.dt, 3)
    assert b.staging_fallbacks() == (3 * blocks, 0)
    a.set_state(wl.cells.T, wl.cells.P, wl.cells.y)
    a.solve_steps(wl.dt, 3)
    assert a.staging_fallbacks() == (0, 0)
    assert np.array_equal(a.get_state(), b.get_state())


def test_fp32_lu_50k_all_cells(oracle_lib, cg, tropo):
    # The FP32-LU form's stated bound: no less accurate than the FP64 oracle
    # against a tight reference (the oracle at rtol 1e-10), max over cells within
    # 1.25x and median within 1.1x of the FP64 oracle's error, on the 100 cells
    # where the FP32 form differs most from the FP64 oracle and on 100 random
    # cells.  The per-species relative-error distribution against the FP64
    # oracle over all 50,000 cells is printed beside it (a 1e-6 bar cannot hold:
    # the FP32 factor changes the corrector iterates, so borderline decisions
    # flip and step sequences differ).
    wl = synth.workload_precision(50_000)
    c32 = _batch(cg, tropo, wl, driver="persistent", lu_precision=32)
    c32.solve_step(wl.dt)
    y, st = c32.get_state(), c32.get_stats()
    c64 = _batch(cg, tropo, wl, driver="persistent", lu_precision=64)
    c64.solve_step(wl.dt)
    st64 = c64.get_stats()
    assert np.all(st["status"] == 0) and np.all(st64["status"] == 0)
    yo, so = pool.solve(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol)
    assert np.all(so["status"] == 0)
    tol = wl.rtol * np.abs(yo) + wl.atol
    units = (np.abs(y - yo) / tol).max(axis=0)
    rng = np.random.default_rng(3)
    idx = np.unique(np.concatenate([np.argsort(-units)[:100], rng.integers(0, wl.cells.n_cells, 100)]))
    sub = synth.subset(wl.cells, idx)
    yt, stt = pool.solve(wl.mech, sub, wl.dt, 1e-10, 1e-18, max_steps=200_000)
    assert np.all(stt["status"] == 0)
    unit_t = wl.rtol * np.abs(yt) + wl.atol
    acc32 = (np.abs(y[:, idx] - yt) / unit_t).max(axis=0)
    acc64 = (np.abs(yo[:, idx] - yt) / unit_t).max(axis=0)
    msg = (f"FP32 LU vs tight reference on {idx.size} cells: max {acc32.max():.2f} (FP64 oracle {acc64.max():.2f}), "
           f"median {np.median(acc32):.2f} (FP64 oracle {np.median(acc64):.2f}) tolerance units")
    assert acc32.max() <= 1.25 * acc64.max() and np.median(acc32) <= 1.1 * np.median(acc64), msg
    mask = np.abs(yo) > FLOOR
    rel = np.where(mask, np.abs(y - yo) / np.where(mask, np.abs(yo), 1.0), 0.0)
    per_species = rel.max(axis=1)
    per_cell = rel.max(axis=0)
    print(f"fp32 LU 50k, all cells against the FP64 oracle: per-species max rel err median "
          f"{np.median(per_species):.2e}, max {per_species.max():.2e}; per-cell max rel err percentiles "
          f"50/90/99/99.9/100: {np.percentile(per_cell, [50, 90, 99, 99.9, 100])}; tolerance units max "
          f"{units.max():.1f}, cells above 10 units {int(np.sum(units > 10))}; {msg}; Newton iterations "
          f"{st['newton_iters'].sum() / st64['newton_iters'].sum():.4f}x the FP64 GPU path's")


def _adjoint_spread(wl, cells, tapes, lam, n=16):
    """Per cell, the largest relative move of the oracle adjoint's dL/dy0 (on
    entries above 1e-6 of the cell's largest) when the states recorded on its
    tape and y0 are perturbed by 1e-15 relative (rounding-level noise)."""
    C = cells.n_cells
    rep = np.repeat(np.arange(C), n)
    sub = synth.subset(cells, rep)
    rng = np.random.default_rng(17)
    sub.y = sub.y * (1 + 1e-15 * rng.standard_normal(sub.y.shape))
    import oracle
    tp = []
    for i in rep:
        t = tapes[i]
        tp.append(oracle.Tape(t.kind, t.q, t.val, t.y * (1 + 1e-15 * rng.standard_normal(t.y.shape))))
    lp, _ = pool.adjoint(wl.mech, sub, tp, np.ascontiguousarray(lam[:, rep]))
    l0, _ = pool.adjoint(wl.mech, cells, tapes, lam)
    out = np.zeros(C)
    for i in range(C):
        ref = l0[:, i]
        big = np.abs(ref) > 1e-6 * np.abs(ref).max()
        out[i] = (np.abs(lp[:, i * n:(i + 1) * n] - ref[:, None])[big] / np.abs(ref[big])[:, None]).max()
    return out


def test_adjoint_2048_all_cells(oracle_lib, cg, tropo):
    # The whole 2,048-cell batch forward (4 steps, tape recorded) and backward with
    # the workload's loss weights on every cell; the oracle adjoint of every
    # cell's GPU tape gives dL/dy0 per cell and dL/dtheta as their sum.  Bar: 1e-8
    # relative on entries above 1e-6 of the cell's largest (1e-12 of it below).
    # The GPU's sparse static-order LU and the oracle's dense pivoted LU round
    # differently in the transposed solves; where the iteration matrices are
    # ill-conditioned that is amplified, so a cell above the bar must lie within
    # 10x the oracle adjoint's own spread under rounding-level noise on its tape
    # and within the workload's differentiation bar, 1e-5 relative.
    wl = synth.workload_adjoint(2048)
    c = _batch(cg, tropo, wl, driver="persistent", record_adjoint=True)
    for _ in range(wl.n_steps):
        c.solve_step(wl.dt)
    w = synth.loss_weights(wl.mech.n_species, wl.cells.n_cells)
    gth, gy0, n_bad = c.sensitivity(w)
    assert n_bad == 0
    tapes = []
    for k in range(wl.cells.n_cells):
        kind, q, val, rows = c.get_tape(k)
        has_row = (kind == 0) | (kind == 4) | (kind == 5)
        yrow = np.zeros((kind.size, wl.mech.n_species))
        yrow[has_row] = rows
        tapes.append(oracle_lib.Tape(kind, q, val, yrow))
    ly0, g = pool.adjoint(wl.mech, wl.cells, tapes, w)
    scale = np.abs(ly0).max(axis=0)
    big = np.abs(ly0) > 1e-6 * scale
    rel = np.where(big, np.abs(gy0 - ly0) / np.maximum(np.abs(ly0), 1e-300), 0.0).max(axis=0)
    small_ok = np.all(big | (np.abs(gy0 - ly0) <= 1e-12 * scale), axis=0)
    assert np.all(small_ok), f"entries below 1e-6 of the cell's largest beyond 1e-12 of it: {np.nonzero(~small_ok)[0][:8]}"
    odd = np.nonzero(rel > 1e-8)[0]
    detail = ""
    if odd.size:
        sub = synth.subset(wl.cells, odd)
        sp = _adjoint_spread(wl, sub, [tapes[i] for i in odd], np.ascontiguousarray(w[:, odd]))
        detail = [(int(i), float(rel[i]), float(s)) for i, s in zip(odd, sp)]
        beyond = [d for d in detail if d[1] > 10 * d[2] or d[1] > 1e-5]
        assert not beyond, f"dL/dy0 beyond 10x the oracle adjoint's rounding spread or 1e-5 (cell, rel, spread): {beyond}"
    assert odd.size <= max(2, MAX_ODD_FRAC * wl.cells.n_cells), detail
    # dL/dtheta sums every cell's contribution: each may carry its cell's error,
    # 1e-8 of its size, or up to the differentiation bar for a rounding-limited cell
    g_sum = g.sum(axis=0)
    is_odd = np.zeros(wl.cells.n_cells, bool)
    is_odd[odd] = True
    allow = 1e-8 * np.abs(g[~is_odd]).sum(axis=0) + 1e-5 * np.abs(g[is_odd]).sum(axis=0)
    excess = np.abs(gth - g_sum) / np.maximum(allow, 1e-300)
    assert np.all(excess <= 1.0), (int(np.argmax(excess)), float(excess.max()))
    print(f"adjoint 2048 cells, all cells: dL/dy0 max rel diff {rel[rel <= 1e-8].max():.2e} on {2048 - odd.size} "
          f"cells, rounding-limited {odd.size} (cell, rel, oracle spread): {detail}; dL/dtheta max diff "
          f"{(np.abs(gth - g_sum) / np.abs(g).sum(axis=0)).max():.2e} of the summed contributions' magnitude")
