"""GPU tangent (forward-mode) sensitivities against the oracle tangent.

As for the adjoint, the GPU's own recorded tape is read back and given to the
oracle, so both differentiate the same frozen-control map.  The GPU tangent
dy = (dy/dy0) dy0 + (dy/dtheta) dtheta must match the oracle tangent to 1e-8
relative (plus 1e-12 of the cell's largest component: the sparse LU and the
oracle's dense pivoted LU round differently), and must satisfy the adjoint
identity <w, dy> = <dL/dy0, dy0> + <dL/dtheta, dtheta> with the GPU adjoint
to 1e-9 of the sum of absolute terms, at every size.
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
    has_row = (kind == 0) | (kind == 4) | (kind == 5)
    assert has_row.sum() == rows.shape[0]
    y = np.zeros((kind.size, rows.shape[1]))
    y[has_row] = rows
    return oracle_lib.Tape(kind.astype(np.int32), q.astype(np.int32), val.astype(np.float64), y)


def _directions(mech, cells, seed):
    rng = np.random.default_rng(seed)
    dy0 = rng.standard_normal(cells.y.shape) * cells.y
    dth = rng.standard_normal(mech.n_reactions)
    return dy0, dth


def _solved(cg, wl, cells, n_steps, theta=None):
    m = cg.Mechanism(wl.mech)
    c = cg.Cells(m, cells.n_cells, rtol=wl.rtol, atol=wl.atol, record_adjoint=True)
    c.set_state(cells.T, cells.P, cells.y)
    if cells.J is not None:
        c.set_photolysis(cells.J)
    if theta is not None:
        c.set_theta(theta)
    for _ in range(n_steps):
        c.solve_step(wl.dt)
    return m, c


@pytest.mark.parametrize("name,n_steps,with_theta", [("small", 2, False), ("tropo", 4, False), ("tropo", 2, True),
                                                    ("pressure", 2, True)])
def test_gpu_tangent_matches_oracle_tangent(oracle_lib, cg, name, n_steps, with_theta):
    # "pressure": the Troe / pressure-sum kinds, 1e3..1.05e5 Pa (theta scales every kind alike)
    wl = {"small": synth.workload_small, "tropo": lambda: synth.workload_adjoint(12),
          "pressure": lambda: synth.workload_pressure(12)}[name]()
    n_cells = 6
    cells = synth.subset(wl.cells, np.arange(n_cells))
    theta = np.random.default_rng(5).uniform(-0.3, 0.3, wl.mech.n_reactions) if with_theta else None
    m, c = _solved(cg, wl, cells, n_steps, theta)
    dy0, dth = _directions(wl.mech, cells, 21)
    dy, n_bad = c.tangent(dy0, dth)
    assert n_bad == 0
    for k in range(n_cells):
        tape = _tape_for(oracle_lib, *c.get_tape(k))
        jp = None if cells.J is None else cells.J[:, k]
        kt = oracle_lib.rate_constants(wl.mech, cells.T[k], cells.P[k], jphot=jp, theta=theta)
        ref = oracle_lib.tangent(wl.mech, kt, cells.y[:, k], tape, dy0[:, k], dth)
        scale = np.abs(ref).max()
        assert np.all(np.abs(dy[:, k] - ref) <= 1e-8 * np.abs(ref) + 1e-12 * scale), k


def test_tangent_adjoint_identity_full_size(oracle_lib, cg):
    """The 2,048-cell, four-step differentiation workload: the identity on every
    cell, the oracle tangent on a sample of cells."""
    wl = synth.workload_adjoint()
    n = wl.cells.n_cells
    m, c = _solved(cg, wl, wl.cells, wl.n_steps)
    w = synth.loss_weights(wl.mech.n_species, n)
    gth, gy0, n_bad = c.sensitivity(w)
    assert n_bad == 0
    dy0, dth = _directions(wl.mech, wl.cells, 22)
    dy, n_bad = c.tangent(dy0, dth)
    assert n_bad == 0
    lhs = np.sum(w * dy)
    rhs = np.sum(gy0 * dy0) + gth @ dth
    mag = np.sum(np.abs(w * dy)) + np.sum(np.abs(gy0 * dy0)) + np.abs(gth) @ np.abs(dth)
    assert abs(lhs - rhs) <= 1e-9 * mag
    # per cell: the adjoint's theta gradient is summed over cells, so check y0 alone
    dyy, _ = c.tangent(dy0)
    per_cell = np.sum(w * dyy, axis=0) - np.sum(gy0 * dy0, axis=0)
    assert np.all(np.abs(per_cell) <= 1e-9 * (np.sum(np.abs(w * dyy), axis=0) + np.sum(np.abs(gy0 * dy0), axis=0)))
    for k in np.linspace(0, n - 1, 6).astype(int):
        tape = _tape_for(oracle_lib, *c.get_tape(k))
        kt = oracle_lib.rate_constants(wl.mech, wl.cells.T[k], wl.cells.P[k])
        ref = oracle_lib.tangent(wl.mech, kt, wl.cells.y[:, k], tape, dy0[:, k], dth)
        assert np.all(np.abs(dy[:, k] - ref) <= 1e-8 * np.abs(ref) + 1e-12 * np.abs(ref).max()), k


def test_walks_do_not_depend_on_batch_size_or_launch_shape(cg):
    """Each cell's walk is its own: the first 48 cells of a batch large enough
    for the walks' full occupancy (two or more cells per warp at 8 warps per
    SM) and the same 48 cells alone (walked at no more than 8 warps per SM)
    give bitwise equal final states, dL/dy0 and tangents."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    n_big, n = 2 * 8 * n_sm + 97, 48
    wl = synth.workload_adjoint(n_big)
    S = wl.mech.n_species
    w = synth.loss_weights(S, n_big)
    dy0, dth = _directions(wl.mech, wl.cells, 23)
    out = []
    for cells, ww, d0 in ((wl.cells, w, dy0), (synth.subset(wl.cells, np.arange(n)), w[:, :n], dy0[:, :n])):
        m, c = _solved(cg, wl, cells, wl.n_steps)
        y = c.get_state()
        gth, gy0, n_bad = c.sensitivity(ww)
        dy, n_bad_t = c.tangent(d0, dth)
        assert n_bad == 0 and n_bad_t == 0
        out.append((y[:, :n], gy0[:, :n], dy[:, :n]))
        c.close()
    for big, small in zip(*out):
        assert np.array_equal(big, small)


def test_tangent_options_and_devices(cg):
    wl = synth.workload_adjoint(10)
    m, c = _solved(cg, wl, wl.cells, 1)
    dy0, dth = _directions(wl.mech, wl.cells, 23)
    a, _ = c.tangent(dy0)
    b, _ = c.tangent(dy0, np.zeros(wl.mech.n_reactions))
    assert np.array_equal(a, b)
    # linear in the direction
    d1, _ = c.tangent(dy0, dth)
    d2, _ = c.tangent(np.zeros_like(dy0), dth)
    assert np.allclose(d1, a + d2, rtol=1e-10, atol=1e-10 * np.abs(d1).max())
    # device tensors in and out give the host result
    dev = torch.device("cuda")
    out = torch.zeros(dy0.shape, dtype=torch.float64, device=dev)
    t, _ = c.tangent(torch.from_numpy(dy0).to(dev), torch.from_numpy(dth).to(dev), out)
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy(), d1)
    with pytest.raises(cg.ChemError):
        c.tangent(torch.from_numpy(dy0).to(dev), dth)
    plain = cg.Cells(m, 4, rtol=wl.rtol, atol=wl.atol)
    with pytest.raises(cg.ChemError):
        plain.tangent(np.zeros((wl.mech.n_species, 4)))


def test_tangent_and_adjoint_at_128_species(oracle_lib, cg):
    # the maximum species count (four register slots per lane): the GPU tangent and
    # adjoint of the GPU tape against the oracle's
    m = synth.random_mechanism(128, 330, 100, 34, name="synthetic_128sp_330rx")
    cells = synth.random_cells(128, 5, T_range=(220.0, 310.0), P_range=(2e4, 1e5))
    wl = synth.Workload(m.name, m, cells, 600.0, 1, 1e-4, 1e-10)
    mech, c = _solved(cg, wl, cells, 1)
    dy0, dth = _directions(m, cells, 24)
    dy, n_bad = c.tangent(dy0, dth)
    assert n_bad == 0
    w = synth.loss_weights(128, cells.n_cells)
    gth, gy0, n_bad = c.sensitivity(w)
    assert n_bad == 0
    g_sum = np.zeros(m.n_reactions)
    for k in range(cells.n_cells):
        tape = _tape_for(oracle_lib, *c.get_tape(k))
        kt = oracle_lib.rate_constants(m, cells.T[k], cells.P[k])
        ref = oracle_lib.tangent(m, kt, cells.y[:, k], tape, dy0[:, k], dth)
        assert np.all(np.abs(dy[:, k] - ref) <= 1e-8 * np.abs(ref) + 1e-12 * np.abs(ref).max()), k
        ly0, g = oracle_lib.adjoint(m, kt, cells.y[:, k], tape, w[:, k])
        g_sum += g
        assert np.all(np.abs(gy0[:, k] - ly0) <= 1e-8 * np.abs(ly0) + 1e-12 * np.abs(ly0).max()), k
    assert np.all(np.abs(gth - g_sum) <= 1e-8 * np.abs(g_sum) + 1e-12 * np.abs(g_sum).max())
