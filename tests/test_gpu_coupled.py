"""GPU coupled (multi-cell) solve against the oracle's coupled system.

couple_cells = G integrates every group of G consecutive cells as one ODE
system (the paper's Multi-cells): one step size, order and Newton iteration
and one WRMS norm over the group.  The oracle integrates the same group
written out as one mechanism (oracle.solve_coupled).  Parity rules are those
of parity_util, applied per group: within 1e-6 relative above 1e-10 mol/mol;
where the group's result moves more than that under 1e-15 perturbations of
its inputs, within 10x that spread and the integration tolerance; groups
whose step sequence differs, within the integration tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_00011_gb300 import synth  # noqa: E402

from parity_util import FLOOR, REL  # noqa: E402


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


def _solve(cg, mech, wl, cells, G, driver):
    c = cg.Cells(mech, cells.n_cells, rtol=wl.rtol, atol=wl.atol, driver=driver, couple_cells=G)
    c.set_state(cells.T, cells.P, cells.y)
    if cells.J is not None:
        c.set_photolysis(cells.J)
    c.solve_step(wl.dt)
    return c.get_state(), c.get_stats()


def _group_spread(oracle_lib, wl, cells, idx, n=3):
    sub = synth.subset(cells, idx)
    yo, _ = oracle_lib.solve_coupled(wl.mech, sub, wl.dt, wl.rtol, wl.atol, len(idx))
    worst = 0.0
    for r in range(n):
        p = synth.subset(cells, idx)
        p.y = p.y * (1 + 1e-15 * np.random.default_rng(100 + r).standard_normal(p.y.shape))
        yp, _ = oracle_lib.solve_coupled(wl.mech, p, wl.dt, wl.rtol, wl.atol, len(idx))
        mask = np.abs(yo) > FLOOR
        worst = max(worst, float((np.abs(yp - yo)[mask] / np.abs(yo[mask])).max()))
    return worst


def _compare_groups(oracle_lib, wl, cells, G, y, st):
    yo, so = oracle_lib.solve_coupled(wl.mech, cells, wl.dt, wl.rtol, wl.atol, G)
    assert np.array_equal(st["status"], so["status"])
    tol = wl.rtol * np.abs(yo) + wl.atol
    odd = 0
    n_groups = 0
    for c0 in range(0, cells.n_cells, G):
        idx = np.arange(c0, min(cells.n_cells, c0 + G))
        n_groups += 1
        # one system: every cell of a group shares the group's counts
        assert np.all(st["steps"][idx] == st["steps"][idx[0]]) and np.all(st["newton_iters"][idx] == st["newton_iters"][idx[0]])
        if so["status"][idx[0]] != 0:
            continue
        same = st["steps"][idx[0]] == so["steps"][idx[0]] and st["newton_iters"][idx[0]] == so["newton_iters"][idx[0]]
        ug = np.abs(y[:, idx] - yo[:, idx]) / tol[:, idx]
        if not same:
            odd += 1
            assert ug.max() <= 10.0, c0
            continue
        mask = np.abs(yo[:, idx]) > FLOOR
        e = float((np.abs(y[:, idx] - yo[:, idx])[mask] / np.abs(yo[:, idx][mask])).max())
        if e <= REL:
            continue
        odd += 1
        sp = _group_spread(oracle_lib, wl, cells, idx)
        assert e <= 10 * sp, (c0, e, sp)
        assert ug.max() <= 1.0, c0
    assert odd <= max(2, 0.05 * n_groups), odd


@pytest.mark.parametrize("G,n,driver", [(4, 26, "plain"), (4, 26, "persistent"), (10, 23, "persistent")])
def test_coupled_matches_oracle(oracle_lib, cg, tropo, G, n, driver):
    wl = synth.workload_batching(n)          # per-cell photolysis, T in [200, 320] K: uneven cells in a group
    y, st = _solve(cg, tropo, wl, wl.cells, G, driver)
    assert np.all(st["status"] == 0)
    _compare_groups(oracle_lib, wl, wl.cells, G, y, st)


def test_coupled_copies_equal_the_single_cell(cg, tropo):
    wl = synth.workload_tropo(5)
    one = synth.subset(wl.cells, [3])
    group = synth.subset(wl.cells, [3, 3, 3, 3])
    y1, s1 = _solve(cg, tropo, wl, one, 1, "plain")
    yg, sg = _solve(cg, tropo, wl, group, 4, "plain")
    assert np.all(sg["steps"] == s1["steps"][0]) and np.all(sg["newton_iters"] == s1["newton_iters"][0])
    mask = np.abs(y1[:, 0]) > 1e-20
    for c in range(4):
        assert np.all(np.abs(yg[mask, c] - y1[mask, 0]) <= 1e-10 * np.abs(y1[mask, 0]))


def test_coupled_options_rejected(cg, tropo):
    with pytest.raises(cg.ChemError):
        cg.Cells(tropo, 8, couple_cells=4, lu_precision=32)
    with pytest.raises(cg.ChemError):
        cg.Cells(tropo, 8, couple_cells=4, record_adjoint=True)
    with pytest.raises(cg.ChemError):
        cg.Cells(tropo, 8, couple_cells=4, cells_per_block=2)
    c = cg.Cells(tropo, 8, couple_cells=4, driver="persistent")
    wl = synth.workload_tropo(8)
    c.set_state(wl.cells.T, wl.cells.P, wl.cells.y)
    with pytest.raises(cg.ChemError):
        c.autotune(600.0)


def test_coupled_group_order_does_not_change_results(cg, tropo):
    # the persistent queue hands out groups by their previous cost (a second solve of the
    # same batch runs in another order than the first); results equal the plain driver's
    wl = synth.workload_batching(97)
    ref, sref = _solve(cg, tropo, wl, wl.cells, 4, "plain")
    c = cg.Cells(tropo, wl.cells.n_cells, rtol=wl.rtol, atol=wl.atol, driver="persistent", couple_cells=4)
    for _ in range(2):
        c.set_state(wl.cells.T, wl.cells.P, wl.cells.y)
        c.set_photolysis(wl.cells.J)
        c.solve_step(wl.dt)
        assert np.array_equal(c.get_state(), ref) and np.array_equal(c.get_stats(), sref)
