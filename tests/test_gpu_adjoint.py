"""GPU discrete adjoint against the oracle adjoint and finite differences.

The GPU's own recorded tape (step sizes, orders, iteration counts,
projections, and the states its iteration matrices and iterates were
evaluated at) is read back and given to the oracle, so both differentiate
the same frozen-control map.  The oracle replays that map: it must reproduce
the GPU's final state to rounding (1e-9 relative: the GPU's sparse LU and the
oracle's dense pivoted LU round differently).  The GPU's dL/dy0 and
dL/dtheta must match the oracle adjoint to 1e-8 relative, and central
differences (step 1e-6) of the oracle's replay must match the GPU gradient
to 1e-5 relative, the differentiation bar of the workload.
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


def _tape_for(oracle_lib, kind, q, val, rows):
    """The GPU tape in the oracle's layout: one state per event (rows go, in
    order, to the INIT, REFACTOR and ITER events; the others get zeros)."""
    has_row = (kind == 0) | (kind == 4) | (kind == 5)
    assert has_row.sum() == rows.shape[0]
    y = np.zeros((kind.size, rows.shape[1]))
    y[has_row] = rows
    return oracle_lib.Tape(kind.astype(np.int32), q.astype(np.int32), val.astype(np.float64), y)


def _run(cg, wl, n_cells, n_steps):
    m = cg.Mechanism(wl.mech)
    cells = synth.subset(wl.cells, np.arange(n_cells))
    c = cg.Cells(m, n_cells, rtol=wl.rtol, atol=wl.atol, record_adjoint=True)
    c.set_state(cells.T, cells.P, cells.y)
    for _ in range(n_steps):
        c.solve_step(wl.dt)
    w = synth.loss_weights(wl.mech.n_species, n_cells)
    gth, gy0, n_bad = c.sensitivity(w)
    assert n_bad == 0
    return m, c, cells, w, gth, gy0


@pytest.mark.parametrize("name,n_steps", [("small", 2), ("tropo", 4)])
def test_gpu_adjoint_matches_oracle_adjoint(oracle_lib, cg, name, n_steps):
    wl = synth.workload_small() if name == "small" else synth.workload_adjoint(12)
    n_cells = 6
    m, c, cells, w, gth, gy0 = _run(cg, wl, n_cells, n_steps)
    g_sum = np.zeros(wl.mech.n_reactions)
    y_gpu = c.get_state()
    for k in range(n_cells):
        kind, q, val, rows = c.get_tape(k)
        assert (kind == 0).sum() == n_steps
        assert np.all(np.isin(kind, [0, 1, 2, 3, 4, 5]))
        tape = _tape_for(oracle_lib, kind, q, val, rows)
        kt = oracle_lib.rate_constants(wl.mech, cells.T[k], cells.P[k])
        yr = oracle_lib.replay(wl.mech, kt, cells.y[:, k], tape)
        big = np.abs(y_gpu[:, k]) > 1e-10 * np.abs(y_gpu[:, k]).max()
        assert np.all(np.abs(yr - y_gpu[:, k])[big] <= 1e-9 * np.abs(y_gpu[:, k])[big]), k
        ly0, g = oracle_lib.adjoint(wl.mech, kt, cells.y[:, k], tape, w[:, k])
        g_sum += g
        scale = np.abs(ly0).max()
        assert np.all(np.abs(gy0[:, k] - ly0) <= 1e-8 * np.abs(ly0) + 1e-12 * scale), k
    scale = np.abs(g_sum).max()
    assert np.all(np.abs(gth - g_sum) <= 1e-8 * np.abs(g_sum) + 1e-12 * scale)


def test_gpu_adjoint_matches_finite_differences(oracle_lib, cg):
    wl = synth.workload_adjoint(8)
    n_cells, n_steps = 3, 4
    m, c, cells, w, gth, gy0 = _run(cg, wl, n_cells, n_steps)
    rng = np.random.default_rng(11)
    eps = 1e-6
    tapes = [_tape_for(oracle_lib, *c.get_tape(k)) for k in range(n_cells)]
    kts = [oracle_lib.rate_constants(wl.mech, cells.T[k], cells.P[k]) for k in range(n_cells)]

    def loss(theta, dy0=None):
        # the iteration matrices stay those of the recorded run (kt_M)
        tot = 0.0
        for k in range(n_cells):
            kt = oracle_lib.rate_constants(wl.mech, cells.T[k], cells.P[k], theta=theta)
            y0 = cells.y[:, k] if dy0 is None else cells.y[:, k] + dy0[:, k]
            tot += w[:, k] @ oracle_lib.replay(wl.mech, kt, y0, tapes[k], kt_M=kts[k])
        return tot

    R = wl.mech.n_reactions
    for _ in range(2):
        v = rng.standard_normal(R)
        fd = (loss(eps * v) - loss(-eps * v)) / (2 * eps)
        assert abs(fd - gth @ v) <= 1e-5 * (np.abs(gth) @ np.abs(v))
        u = rng.standard_normal(cells.y.shape) * cells.y
        fd = (loss(np.zeros(R), eps * u) - loss(np.zeros(R), -eps * u)) / (2 * eps)
        assert abs(fd - np.sum(gy0 * u)) <= 1e-5 * np.sum(np.abs(gy0 * u))


def test_gpu_adjoint_per_component_fd(oracle_lib, cg):
    # component by component: central differences (step 1e-6) of the oracle's
    # replay of the GPU tapes, the iteration matrices held at the recorded run's,
    # against the GPU gradient to 1e-5 relative, on 20 log rate constants (the 12
    # with the largest |dL/dtheta_j| and 8 more drawn at random above 1e-2 of the
    # largest) and, per cell, on the 20 initial concentrations through which L
    # moves most (largest |dL/dy0_i y0_i|; the step is 1e-6 y0_i).  The floor:
    # the loss is evaluated to a few ulp, so the difference quotient carries an
    # error of about 4e-16 |L| / 2e-6 = 2e-10 |L|; here the largest |dL/dtheta_j|
    # is about 0.017 |L|, so 1e-5 relative is checkable from 1e-2 of it up
    # (observed: 1.3e-5 at about 1e-3 of the largest, 2.8e-6 at 1.7e-3).
    wl = synth.workload_adjoint(8)
    n_cells, n_steps = 3, 4
    m, c, cells, w, gth, gy0 = _run(cg, wl, n_cells, n_steps)
    eps = 1e-6
    tapes = [_tape_for(oracle_lib, *c.get_tape(k)) for k in range(n_cells)]
    kts = [oracle_lib.rate_constants(wl.mech, cells.T[k], cells.P[k]) for k in range(n_cells)]

    def cell_loss(k, theta=None, y0=None):
        kt = kts[k] if theta is None else oracle_lib.rate_constants(wl.mech, cells.T[k], cells.P[k], theta=theta)
        y0 = cells.y[:, k] if y0 is None else y0
        return w[:, k] @ oracle_lib.replay(wl.mech, kt, y0, tapes[k], kt_M=kts[k])

    R = wl.mech.n_reactions
    rng = np.random.default_rng(5)
    order = np.argsort(-np.abs(gth))
    above = np.nonzero(np.abs(gth) >= 1e-2 * np.abs(gth).max())[0]
    pick = np.unique(np.concatenate([order[:12], rng.choice(np.setdiff1d(above, order[:12]), 8, replace=False)]))
    worst = 0.0
    for j in pick:
        e = np.zeros(R)
        e[j] = eps
        fd = sum(cell_loss(k, e) - cell_loss(k, -e) for k in range(n_cells)) / (2 * eps)
        err = abs(fd - gth[j]) / abs(gth[j])
        worst = max(worst, err)
        assert err <= 1e-5, (int(j), fd, gth[j], err)
    for k in range(n_cells):
        y0 = cells.y[:, k]
        for i in np.argsort(-np.abs(gy0[:, k] * y0))[:20]:
            h = eps * y0[i]
            yp, ym = y0.copy(), y0.copy()
            yp[i] += h
            ym[i] -= h
            fd = (cell_loss(k, y0=yp) - cell_loss(k, y0=ym)) / (2 * h)
            err = abs(fd - gy0[i, k]) / abs(gy0[i, k])
            worst = max(worst, err)
            assert err <= 1e-5, (k, int(i), fd, gy0[i, k], err)
    print(f"per-component central differences, {pick.size} theta_j and {20 * n_cells} y0 entries: "
          f"max rel err {worst:.2e}")


def test_autograd_function_matches_sensitivity(cg):
    wl = synth.workload_adjoint(16)
    dev = torch.device("cuda")
    m = cg.Mechanism(wl.mech)
    c = cg.Cells(m, 16, rtol=wl.rtol, atol=wl.atol, record_adjoint=True)
    theta = torch.zeros(wl.mech.n_reactions, dtype=torch.float64, device=dev, requires_grad=True)
    y0 = torch.from_numpy(wl.cells.y[:, :16].copy()).to(dev).requires_grad_(True)
    T = torch.from_numpy(wl.cells.T[:16].copy()).to(dev)
    P = torch.from_numpy(wl.cells.P[:16].copy()).to(dev)
    w = torch.from_numpy(synth.loss_weights(wl.mech.n_species, 16)).to(dev)
    y = cg.solve_with_grad(c, theta, y0, T, P, wl.dt, 2)
    (w * y).sum().backward()
    gth, gy0, n_bad = c.sensitivity(w.cpu().numpy())
    assert n_bad == 0
    np.testing.assert_allclose(theta.grad.cpu().numpy(), gth, rtol=1e-12, atol=0)
    np.testing.assert_allclose(y0.grad.cpu().numpy(), gy0, rtol=1e-12, atol=0)


def _rows_needed(cg, m, wl, T, P, y0, n_steps):
    """Largest tape (rows) any cell needs for all n_steps, and for any single step."""
    c = cg.Cells(m, y0.shape[1], rtol=wl.rtol, atol=wl.atol, record_adjoint=True)
    c.set_state(T, P, y0)
    states = [y0]
    for _ in range(n_steps):
        c.solve_step(wl.dt)
        states.append(c.get_state())
    rows_all = max(c.get_tape(k)[3].shape[0] for k in range(y0.shape[1]))
    rows_one = 0
    for s in states[:-1]:
        c.set_state(T, P, s)
        c.solve_step(wl.dt)
        rows_one = max(rows_one, max(c.get_tape(k)[3].shape[0] for k in range(y0.shape[1])))
    return rows_all, rows_one


@pytest.mark.parametrize("mode", ["checkpoint", "overflow_fallback"])
def test_step_checkpointing_matches_full_tape(cg, mode):
    # per-step recording (forced, or the automatic fallback after a tape
    # overflow) chains the adjoint through re-run steps: same gradients as
    # one tape over all steps, up to the order of the theta sums
    wl = synth.workload_adjoint(16)
    dev = torch.device("cuda")
    m = cg.Mechanism(wl.mech)
    T = torch.from_numpy(wl.cells.T[:16].copy()).to(dev)
    P = torch.from_numpy(wl.cells.P[:16].copy()).to(dev)
    w = torch.from_numpy(synth.loss_weights(wl.mech.n_species, 16)).to(dev)
    tape_small = 0
    if mode == "overflow_fallback":
        rows_all, rows_one = _rows_needed(cg, m, wl, wl.cells.T[:16], wl.cells.P[:16], wl.cells.y[:, :16].copy(),
                                          wl.n_steps)
        assert rows_one < rows_all
        tape_small = rows_one          # holds any one step, not all of them
    grads = []
    for kind in ("full", mode):
        tape = tape_small if kind == "overflow_fallback" else 0
        c = cg.Cells(m, 16, rtol=wl.rtol, atol=wl.atol, record_adjoint=True, tape_steps=tape)
        theta = torch.zeros(wl.mech.n_reactions, dtype=torch.float64, device=dev, requires_grad=True)
        y0 = torch.from_numpy(wl.cells.y[:, :16].copy()).to(dev).requires_grad_(True)
        y = cg.solve_with_grad(c, theta, y0, T, P, wl.dt, wl.n_steps, checkpoint=(kind == "checkpoint"))
        (w * y).sum().backward()
        grads.append((y.detach().cpu().numpy(), theta.grad.cpu().numpy(), y0.grad.cpu().numpy()))
        if kind == "overflow_fallback":
            c.set_state(T, P, y0.detach())
            for _ in range(wl.n_steps):
                c.solve_step(wl.dt)
            assert c.sensitivity(w.cpu().numpy())[2] > 0      # the whole tape does not fit
    (ya, ga, ha), (yb, gb, hb) = grads
    assert np.array_equal(ya, yb)
    np.testing.assert_allclose(gb, ga, rtol=1e-11, atol=1e-14 * np.abs(ga).max())
    np.testing.assert_allclose(hb, ha, rtol=1e-11, atol=1e-14 * np.abs(ha).max())


def test_tape_overflow_is_reported(cg):
    wl = synth.workload_adjoint(4)
    m = cg.Mechanism(wl.mech)
    c = cg.Cells(m, 4, rtol=wl.rtol, atol=wl.atol, record_adjoint=True, tape_steps=8)
    c.set_state(wl.cells.T[:4], wl.cells.P[:4], wl.cells.y[:, :4])
    c.solve_step(wl.dt)
    gth, gy0, n_bad = c.sensitivity(np.ones((wl.mech.n_species, 4)))
    assert n_bad == 4
    assert np.all(gy0 == 0.0) and np.all(gth == 0.0)


def test_recording_needs_fp64_lu(cg):
    wl = synth.workload_adjoint(4)
    m = cg.Mechanism(wl.mech)
    with pytest.raises(cg.ChemError):
        cg.Cells(m, 4, record_adjoint=True, lu_precision=32)


def test_sensitivity_requires_recording(cg):
    wl = synth.workload_adjoint(4)
    m = cg.Mechanism(wl.mech)
    c = cg.Cells(m, 4)
    c.set_state(wl.cells.T[:4], wl.cells.P[:4], wl.cells.y[:, :4])
    c.solve_step(wl.dt)
    with pytest.raises(cg.ChemError):
        c.sensitivity(np.ones((wl.mech.n_species, 4)))


def test_sensitivity_checkpointed_host_arrays(cg):
    # the library's checkpointed backward called directly with host arrays: the
    # kept states of a 3-step forward, every step re-solved from its state, the
    # adjoint chained through them, against one tape over all three steps
    wl = synth.workload_adjoint(24)
    m = cg.Mechanism(wl.mech)
    cells = synth.subset(wl.cells, np.arange(24))
    w = synth.loss_weights(wl.mech.n_species, 24)
    c = cg.Cells(m, 24, rtol=wl.rtol, atol=wl.atol, record_adjoint=True, driver="persistent")
    c.set_state(cells.T, cells.P, cells.y)
    states = [cells.y.copy()]
    for _ in range(3):
        c.solve_step(wl.dt)
        states.append(c.get_state())
    g_full, l_full, n_bad = c.sensitivity(w)
    assert n_bad == 0
    g_ck, l_ck, n_bad = c.sensitivity_checkpointed(np.stack(states[:-1]), wl.dt, w)
    assert n_bad == 0
    np.testing.assert_allclose(g_ck, g_full, rtol=1e-11, atol=1e-14 * np.abs(g_full).max())
    np.testing.assert_allclose(l_ck, l_full, rtol=1e-11, atol=1e-14 * np.abs(l_full).max())
    # the batch holds the re-solved first step afterwards
    assert np.array_equal(c.get_state(), states[1])
