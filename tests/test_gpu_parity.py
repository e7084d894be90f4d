"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

The tolerances and the rounding-spread rule are those of parity_util.  The
FP32-LU path must match the FP64 oracle within 20 tolerance units and be as
accurate as it against a tight reference.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_00011_gb300 import synth  # noqa: E402

from parity_util import FLOOR, compare as _compare  # noqa: E402


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
def mechs(cg):
    return {"small": cg.Mechanism(synth.mechanism_small()), "tropo": cg.Mechanism(synth.mechanism_tropo()),
            "pressure": cg.Mechanism(synth.mechanism_tropo_pressure())}


# ---------------------------------------------------------------- kernel level

@pytest.mark.parametrize("name", ["small", "tropo", "pressure"])
def test_deriv_matches_oracle(oracle_lib, cg, mechs, name):
    # pressures from 1e3 to 1.05e5 Pa: the fall-off reactions from near one limit to near the other
    m = mechs[name]
    cells = synth.random_cells(m.n_species, 70, T_range=(200, 310), P_range=(1e3, 1.05e5), seed=5)
    c = cg.Cells(m, cells.n_cells)
    c.set_state(cells.T, cells.P, cells.y)
    ytest = synth.random_cells(m.n_species, 70, seed=6).y
    f = c.eval_deriv(ytest)
    om = oracle_lib.OracleMechanism(m.synth)
    for k in range(cells.n_cells):
        kt = oracle_lib.rate_constants(om, cells.T[k], cells.P[k])
        fo = oracle_lib.deriv(om, kt, ytest[:, k])
        J = oracle_lib.jacobian(om, kt, ytest[:, k])
        scale = np.abs(J) @ np.abs(ytest[:, k]) + 1e-300       # size of the terms summed into f_i
        assert np.all(np.abs(f[:, k] - fo) <= 1e-13 * scale)


@pytest.mark.parametrize("name", ["small", "tropo", "pressure"])
@pytest.mark.parametrize("design", [0, 1, 2])
def test_deriv_designs_match_oracle(oracle_lib, cg, mechs, name, design):
    # the gather design and the paper's reaction-parallel atomic design (both
    # reaction-data layouts) on 333 cells (a ragged last block), per-cell photolysis
    m = mechs[name]
    cells = synth.random_cells(m.n_species, 333, T_range=(200, 320), P_range=(2e4, 1e5), seed=12)
    c = cg.Cells(m, cells.n_cells)
    c.set_state(cells.T, cells.P, cells.y)
    n_phot = int(np.sum(m.synth.kind == 1))
    jp = np.abs(np.random.default_rng(13).standard_normal((n_phot, cells.n_cells))) * 1e-3
    c.set_photolysis(jp)
    ytest = synth.random_cells(m.n_species, cells.n_cells, seed=14).y
    f = c.eval_deriv_design(design, ytest)
    om = oracle_lib.OracleMechanism(m.synth)
    for k in range(cells.n_cells):
        kt = oracle_lib.rate_constants(om, cells.T[k], cells.P[k], jphot=jp[:, k])
        fo = oracle_lib.deriv(om, kt, ytest[:, k])
        scale = np.abs(oracle_lib.jacobian(om, kt, ytest[:, k])) @ np.abs(ytest[:, k]) + 1e-300
        assert np.all(np.abs(f[:, k] - fo) <= 1e-13 * scale), k
    # the cached rate constants follow set_theta
    th = np.linspace(-0.5, 0.5, m.n_reactions)
    c.set_theta(th)
    f2 = c.eval_deriv_design(design, ytest)
    kt = oracle_lib.rate_constants(om, cells.T[0], cells.P[0], jphot=jp[:, 0], theta=th)
    fo = oracle_lib.deriv(om, kt, ytest[:, 0])
    assert np.allclose(f2[:, 0], fo, rtol=1e-12, atol=1e-12 * np.abs(fo).max())


@pytest.mark.parametrize("name", ["small", "tropo"])
@pytest.mark.parametrize("prec", [64, 32])
def test_newton_solve_matches_dense(oracle_lib, cg, mechs, name, prec):
    m = mechs[name]
    C = 40
    cells = synth.random_cells(m.n_species, C, T_range=(220, 310), P_range=(2e4, 1e5), seed=8)
    c = cg.Cells(m, C, lu_precision=prec)
    c.set_state(cells.T, cells.P, cells.y)
    rng = np.random.default_rng(9)
    b = rng.standard_normal((m.n_species, C))
    om = oracle_lib.OracleMechanism(m.synth)
    tol = 1e-9 if prec == 64 else 2e-4
    for cc in (1e-3, 1.0, 30.0):
        x = c.eval_newton_solve(cc, cells.y, b)
        for k in range(C):
            kt = oracle_lib.rate_constants(om, cells.T[k], cells.P[k])
            Mk = np.eye(m.n_species) - cc * oracle_lib.jacobian(om, kt, cells.y[:, k])
            xr = np.linalg.solve(Mk, b[:, k])
            # backward error of the GPU solution in the matrix norm
            res = np.linalg.norm(Mk @ x[:, k] - b[:, k], np.inf)
            assert res <= tol * (np.linalg.norm(Mk, np.inf) * np.linalg.norm(xr, np.inf) + np.linalg.norm(b[:, k], np.inf))


# ---------------------------------------------------------------- full solve

def test_solve_small_workload(oracle_lib, cg, mechs):
    wl = synth.workload_small()
    y, st = cg.solve(mechs["small"], wl.cells, wl.dt, wl.rtol, wl.atol)
    yo, so = oracle_lib.solve_cells(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol)
    _compare(y, st, yo, so, oracle_lib, wl, wl.cells)


@pytest.mark.parametrize("driver", ["plain", "persistent"])
def test_solve_tropo_subset(oracle_lib, cg, mechs, driver):
    # 301 cells: several blocks and waves with a ragged tail
    wl = synth.workload_tropo(301)
    y, st = cg.solve(mechs["tropo"], wl.cells, wl.dt, wl.rtol, wl.atol, driver=driver)
    yo, so = oracle_lib.solve_cells(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol)
    err, flips, odd = _compare(y, st, yo, so, oracle_lib, wl, wl.cells)
    print(f"tropo 301 cells ({driver}): max rel err {err:.2e} on well-determined cells, "
          f"decision flips {flips}, rounding-limited cells {odd}")


@pytest.mark.parametrize("driver", ["plain", "persistent"])
def test_solve_pressure_dependent(oracle_lib, cg, mechs, driver):
    # Troe fall-off, k_a + k_b [M] and k_a + k_c [M] / (1 + k_c [M] / k_b) reactions,
    # 1e3..1.05e5 Pa; 301 cells
    wl = synth.workload_pressure(301)
    y, st = cg.solve(mechs["pressure"], wl.cells, wl.dt, wl.rtol, wl.atol, driver=driver)
    yo, so = oracle_lib.solve_cells(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol)
    err, flips, odd = _compare(y, st, yo, so, oracle_lib, wl, wl.cells)
    print(f"pressure-dependent 301 cells ({driver}): max rel err {err:.2e}, flips {flips}, rounding-limited {odd}")


@pytest.mark.parametrize("S,R,U,Ph", [(50, 130, 40, 13), (128, 330, 100, 34)])
def test_solve_other_species_counts(oracle_lib, cg, S, R, U, Ph):
    # 33-64 and 97-128 species (128 is the maximum) take the kernels' 2- and 4-slot
    # register paths, which the named workloads do not reach; both drivers, 61 cells.
    # The 128-species cells take 200-560 steps, and 3 of 61 flip a borderline decision
    # (up to 18 tolerance units from the oracle, each closer to a tight reference than
    # the oracle's own result): flips are checked against the tight reference.
    m = synth.random_mechanism(S, R, U, Ph, name=f"synthetic_{S}sp_{R}rx")
    cells = synth.random_cells(S, 61, T_range=(220.0, 310.0), P_range=(2e4, 1e5))
    wl = synth.Workload(m.name, m, cells, 600.0, 1, 1e-4, 1e-10)
    mech = cg.Mechanism(m)
    yo, so = oracle_lib.solve_cells(m, cells, wl.dt, wl.rtol, wl.atol)
    for driver in ("plain", "persistent"):
        y, st = cg.solve(mech, cells, wl.dt, wl.rtol, wl.atol, driver=driver)
        _compare(y, st, yo, so, oracle_lib, wl, cells, max_odd_frac=0.1, tight_flips=True)


@pytest.mark.parametrize("name", ["small", "tropo", "s128"])
def test_persistent_shapes_every_mechanism(cg, mechs, name):
    """The persistent driver's default launch shape exists for every mechanism
    size, and so does a shape with fewer resident blocks per SM than fit (one
    block of two cells per SM: the blocks' shared memory is padded so that no
    second block joins an SM); for a small batch and one of more than two
    cells per warp, both give the plain driver's results bitwise."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    if name == "s128":
        m = synth.random_mechanism(128, 330, 100, 34, name="synthetic_128sp_330rx")
        mech = cg.Mechanism(m)
    else:
        mech = mechs[name]
        m = mech.synth
    for n in (9, 2 * 8 * n_sm + 5):
        cells = synth.random_cells(m.n_species, n, T_range=(220.0, 310.0), P_range=(2e4, 1e5), seed=n)
        ya, sa = cg.solve(mech, cells, 600.0, 1e-4, 1e-10, driver="plain")
        for shape in ({}, {"cells_per_block": 2, "blocks_per_sm": 1}):
            yb, sb = cg.solve(mech, cells, 600.0, 1e-4, 1e-10, driver="persistent", **shape)
            assert np.array_equal(ya, yb) and np.array_equal(sa, sb), (name, n, shape)


def test_device_mode_refuses_host_buffers(cg, mechs):
    """With CHEM_MEM_DEVICE the library hands the caller's buffers to its
    kernels and device-side copies as they are, so a host pointer is refused
    before anything is launched or copied."""
    import ctypes as ct
    L = cg.load()
    wl = synth.workload_tropo(16)
    c = cg.Cells(mechs["tropo"], 16, rtol=wl.rtol, atol=wl.atol)
    c.set_state(wl.cells.T, wl.cells.P, wl.cells.y)
    y_before = c.get_state()
    host = np.ones(16 * 72)
    dev_buf = torch.ones(16 * 72, dtype=torch.float64, device="cuda")
    hp, dp = ct.c_void_p(host.ctypes.data), ct.c_void_p(dev_buf.data_ptr())
    for rc in (L.chem_cells_set_state(c.handle, dp, dp, hp, cg.MEM_DEVICE, None),
               L.chem_get_state(c.handle, hp, cg.MEM_DEVICE, None),
               L.chem_eval_deriv(c.handle, dp, hp, cg.MEM_DEVICE, None),
               L.chem_eval_reciprocal(hp, dp, 16, cg.MEM_DEVICE, None),
               L.chem_eval_warp_sum(dp, hp, 1, cg.MEM_DEVICE, None)):
        assert rc == -1 and "host memory" in L.chem_last_error().decode()
    torch.cuda.synchronize()
    assert np.array_equal(c.get_state(), y_before)
    assert torch.equal(dev_buf, torch.ones_like(dev_buf))
    # device buffers of the current device pass
    out = torch.empty(16, dtype=torch.float64, device="cuda")
    assert L.chem_eval_reciprocal(dp, ct.c_void_p(out.data_ptr()), 16, cg.MEM_DEVICE, None) == 0
    torch.cuda.synchronize()
    assert torch.all(out == 1.0)
    c.close()


def test_drivers_agree_bitwise(cg, mechs):
    wl = synth.workload_tropo(97)
    ya, sa = cg.solve(mechs["tropo"], wl.cells, wl.dt, wl.rtol, wl.atol, driver="plain")
    yb, sb = cg.solve(mechs["tropo"], wl.cells, wl.dt, wl.rtol, wl.atol, driver="persistent", cells_per_block=3)
    assert np.array_equal(ya, yb) and np.array_equal(sa, sb)


def test_fp32_lu_within_bound(oracle_lib, cg, mechs):
    # The FP32 factor/solve changes the corrector's iterates, so borderline
    # decisions flip and the step sequence differs from the FP64 oracle's.  The
    # bound is therefore on accuracy: against a tight FP64 reference (oracle at
    # rtol 1e-10) the FP32-LU result must be as accurate as the FP64 oracle
    # (max over cells within 1.25x, median within 1.1x of the oracle's error);
    # its distance from the oracle is printed beside it (the FP64 oracle's own
    # global error reaches 100 tolerance units on some cells).
    wl = synth.workload_tropo(200)
    y, st = cg.solve(mechs["tropo"], wl.cells, wl.dt, wl.rtol, wl.atol, lu_precision=32)
    yo, so = oracle_lib.solve_cells(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol)
    yt, stt = oracle_lib.solve_cells(wl.mech, wl.cells, wl.dt, 1e-10, 1e-18)
    assert np.all(st["status"] == 0) and np.all(stt["status"] == 0)
    tol = wl.rtol * np.abs(yo) + wl.atol
    units = (np.abs(y - yo) / tol).max()
    acc32 = (np.abs(y - yt) / (wl.rtol * np.abs(yt) + wl.atol)).max(axis=0)
    acc64 = (np.abs(yo - yt) / (wl.rtol * np.abs(yt) + wl.atol)).max(axis=0)
    assert acc32.max() <= 1.25 * acc64.max() and np.median(acc32) <= 1.1 * np.median(acc64)
    rel = np.where(np.abs(yo) > FLOOR, np.abs(y - yo) / np.maximum(np.abs(yo), 1e-300), 0.0).max(axis=1)
    print(f"fp32 LU: per-species max rel err vs FP64 oracle (above 1e-10): median {np.median(rel):.2e}, "
          f"max {rel.max():.2e}; accuracy vs tight reference (tolerance units, max/median) "
          f"{acc32.max():.1f}/{np.median(acc32):.2f} vs FP64 {acc64.max():.1f}/{np.median(acc64):.2f}; "
          f"max distance from the FP64 oracle {units:.1f} tolerance units; "
          f"Newton iterations {st['newton_iters'].sum() / so['newton_iters'].sum():.3f}x the FP64 oracle's")


def test_per_cell_photolysis(oracle_lib, cg, mechs):
    wl = synth.workload_batching(150)
    y, st = cg.solve(mechs["tropo"], wl.cells, wl.dt, wl.rtol, wl.atol)
    yo, so = oracle_lib.solve_cells(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol)
    _compare(y, st, yo, so, oracle_lib, wl, wl.cells)


# ---------------------------------------------------------------- edge cases

def test_empty_and_single_cell(oracle_lib, cg, mechs):
    wl = synth.workload_tropo(1)
    c0 = cg.Cells(mechs["tropo"], 0)
    c0.set_state(np.zeros(0), np.zeros(0), np.zeros((72, 0)))
    c0.solve_step(600.0)
    assert c0.get_state().shape == (72, 0)
    y, st = cg.solve(mechs["tropo"], wl.cells, wl.dt, wl.rtol, wl.atol)
    yo, so = oracle_lib.solve_cells(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol)
    _compare(y, st, yo, so, oracle_lib, wl, wl.cells)


def test_bad_inputs_and_step_cap(oracle_lib, cg, mechs):
    wl = synth.workload_tropo(6)
    cells = synth.subset(wl.cells, np.arange(6))
    cells.T[1] = np.nan
    cells.P[2] = -1.0
    cells.y[5, 3] = np.inf
    y, st = cg.solve(mechs["tropo"], cells, wl.dt, wl.rtol, wl.atol, max_steps=3)
    yo, so = oracle_lib.solve_cells(wl.mech, cells, wl.dt, wl.rtol, wl.atol, max_steps=3)
    assert st["status"].tolist() == so["status"].tolist() == [1, 6, 6, 6, 1, 1]
    np.testing.assert_array_equal(y[:, [0, 4, 5]], cells.y[:, [0, 4, 5]])


def test_api_errors(cg, mechs):
    with pytest.raises(cg.ChemError):
        cg.Cells(mechs["tropo"], 4, rtol=-1.0)
    c = cg.Cells(mechs["tropo"], 4)
    with pytest.raises(cg.ChemError):
        c.solve_step(600.0)          # before set_state
    bad = synth.mechanism_from_list(2, [dict(reac=[0], prod=[5], A=1.0)])
    with pytest.raises(cg.ChemError):
        cg.Mechanism(bad)
    # pressure-dependent kinds: a high-pressure limit must be positive, Troe needs Fc in (0, 1] and N > 0
    for rx in (dict(reac=[0, 1], prod=[0, 1], A=1e-30, kind=synth.TROE, A2=0.0),
               dict(reac=[0, 1], prod=[0, 1], A=1e-30, kind=synth.TROE, A2=1e-11, Fc=1.5),
               dict(reac=[0, 1], prod=[0, 1], A=1e-30, kind=synth.TROE, A2=1e-11, N=0.0),
               dict(reac=[0, 1], prod=[0, 1], A=1e-13, kind=synth.FALLOFF_SUM, A2=-1.0, A3=1e-33),
               dict(reac=[0, 1], prod=[0, 1], A=1e-13, kind=synth.PRESSURE_SUM, A2=float("nan")),
               dict(reac=[0, 1], prod=[0, 1], A=1e-13, kind=7)):
        with pytest.raises(cg.ChemError):
            cg.Mechanism(synth.mechanism_from_list(2, [rx]))


def test_reciprocal_within_one_ulp(cg):
    # The solve kernels' FP64 reciprocal (hardware estimate, two Newton-Raphson
    # steps) against the correctly rounded 1/x over its stated domain, normal x with
    # 2^-1022 <= |x| <= 2^1022: every result within 1 ulp, most correctly rounded.
    # Magnitudes are drawn uniformly in the exponent over the whole domain, plus
    # the domain's ends, powers of two and values just beside them.
    rng = np.random.default_rng(9)
    e = rng.integers(-1022, 1022, 400_000)
    x = np.ldexp(rng.uniform(1.0, 2.0, e.size), e) * rng.choice([-1.0, 1.0], e.size)
    edges = np.array([2.0 ** -1022, 2.0 ** 1022, 1.0, 2.0, 0.5, 3.0, 1e-300, 1e300, 1e-10, 1e10])
    x = np.concatenate([x, edges, -edges, np.nextafter(edges, 0), np.nextafter(edges, np.inf)])
    x = x[(np.abs(x) >= 2.0 ** -1022) & (np.abs(x) <= 2.0 ** 1022)]
    r = cg.eval_reciprocal(x)
    ref = 1.0 / x
    ulps = np.abs(r - ref) / np.spacing(np.abs(ref))
    assert np.all(np.isfinite(r)) and ulps.max() <= 1.0, (x[np.argmax(ulps)], ulps.max())
    print(f"recip_nr: {x.size} values, max {ulps.max():.2f} ulp, correctly rounded {np.mean(r == ref):.4%}")


def test_warp_sum_within_ulps(cg):
    # The solve kernels sum each norm's 32 per-lane terms (squared weighted
    # values, >= 0) on the integer pipe: fixed point relative to the largest
    # term, an exact integer sum, one rounding.  Each truncated term loses less
    # than 1/32 ulp of the largest, so the result is within 1.5 ulp of the exact
    # sum (math.fsum, correctly rounded).  Groups span wide and narrow dynamic
    # ranges, zeros, ties and carries at powers of two; the fallback groups
    # (infinite, NaN, every term below 2^-959) take an FP64 butterfly.
    import math
    rng = np.random.default_rng(17)
    groups = []
    for span in (0, 1, 4, 16, 60, 200):
        c = rng.uniform(-150, 150, (400, 1))
        groups.append(10.0 ** (c + rng.uniform(-span / 2, span / 2 + 1e-12, (400, 32))))
    g = rng.uniform(0.5, 2.0, (200, 32))
    g[rng.random((200, 32)) < 0.5] = 0.0                           # zeros
    groups.append(g)
    groups.append(np.full((8, 32), 1.0))                           # carries into the next binade
    groups.append(np.full((8, 32), 1.0 + 2.0 ** -52))              # ties at the last bit
    t = np.full((8, 32), 2.0 ** -53)
    t[:, 0] = 1.0                                                  # exact ties below one ulp
    groups.append(t)
    groups.append(np.ldexp(rng.uniform(1.0, 2.0, (50, 32)), rng.integers(900, 1000, (50, 32))))   # near overflow
    x = np.concatenate(groups)
    x[-1, 0] = 1.0e308
    r = cg.eval_warp_sum(x)
    exact = np.array([math.fsum(row) for row in x])
    fin = np.isfinite(exact)
    ulps = np.abs(r[fin] - exact[fin]) / np.spacing(exact[fin])
    assert ulps.max() <= 1.5, (x[fin][np.argmax(ulps)], ulps.max())
    assert np.all(np.isinf(r[~fin]))
    # fallback groups
    fb = np.array([[np.inf] + [1.0] * 31, [np.nan] + [1.0] * 31, [2.0 ** -1000] * 32, [0.0] * 32])
    rf = cg.eval_warp_sum(fb)
    assert np.isinf(rf[0]) and np.isnan(rf[1]) and rf[3] == 0.0
    assert abs(rf[2] - 32 * 2.0 ** -1000) <= 4 * np.spacing(32 * 2.0 ** -1000)
    print(f"warp sum: {x.shape[0]} groups, max {ulps.max():.2f} ulp, correctly rounded {np.mean(ulps == 0):.2%}")
