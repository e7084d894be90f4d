"""chem_solve_step_noalloc through the C ABI, against chem_solve_step and the oracle.

The allocation-free entry point serves callers that may not allocate device
memory while they run (a host model under its own memory manager or a fixed
device budget).  They own every buffer; the library keeps the persistent
driver's work-queue counter and its staging counters in a static device array
and clears them on each call.  The cells are independent, so the result does
not depend on the order the queue hands them out in: two calls in a row must
both reproduce the regular entry point bit for bit, which also shows the
counter is reset between calls.  This file is collected last.
"""
import ctypes as ct

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_00011_gb300 import synth  # noqa: E402

from parity_util import compare  # noqa: E402


@pytest.fixture(scope="module")
def cg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_00011_gb300 import build, chemgpu
    build.build()
    torch.cuda.init()
    chemgpu.load()
    return chemgpu


def _dev():
    return torch.device("cuda", torch.cuda.current_device())


def _p(t):
    return ct.c_void_p(t.data_ptr())


def _opts(cg, wl, **kw):
    L = cg.load()
    o = cg.Opts()
    L.chem_opts_default(ct.byref(o))
    o.rtol, o.atol = wl.rtol, wl.atol
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _regular(cg, mech, wl, theta=None, **kw):
    """chem_solve_step on a persistent batch (the entry point the caller would otherwise use)."""
    c = cg.Cells(mech, wl.cells.n_cells, rtol=wl.rtol, atol=wl.atol, driver="persistent", **kw)
    c.set_state(wl.cells.T, wl.cells.P, wl.cells.y)
    if wl.cells.J is not None:
        c.set_photolysis(wl.cells.J)
    if theta is not None:
        c.set_theta(theta)
    c.solve_step(wl.dt)
    y, st = c.get_state(), c.get_stats()
    c.close()
    return y, st


def _noalloc(cg, mech, wl, opts, theta=None):
    """One call of the allocation-free entry point on caller-owned device buffers."""
    L = cg.load()
    dev = _dev()
    C = wl.cells.n_cells
    T = torch.from_numpy(wl.cells.T).to(dev)
    P = torch.from_numpy(wl.cells.P).to(dev)
    y = torch.from_numpy(wl.cells.y).to(dev)
    J = None if wl.cells.J is None else torch.from_numpy(wl.cells.J).to(dev)
    th = None if theta is None else torch.from_numpy(theta).to(dev)
    stats = torch.zeros((C, cg.STATS_DTYPE.itemsize // 8), dtype=torch.int64, device=dev)
    stream = ct.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    rc = L.chem_solve_step_noalloc(mech.handle, C, _p(T), _p(P), None if J is None else _p(J),
                                   None if th is None else _p(th), _p(y), _p(stats), wl.dt, ct.byref(opts), stream)
    assert rc == 0, L.chem_last_error().decode()
    torch.cuda.synchronize(dev)
    return y.cpu().numpy(), stats.cpu().numpy().view(cg.STATS_DTYPE).reshape(C)


def test_noalloc_matches_solve_step_on_two_calls(oracle_lib, cg):
    wl = synth.workload_tropo(333)
    mech = cg.Mechanism(wl.mech)
    y_ref, st_ref = _regular(cg, mech, wl)
    opts = _opts(cg, wl)
    for call in range(2):
        y, st = _noalloc(cg, mech, wl, opts)
        assert np.array_equal(y, y_ref) and np.array_equal(st, st_ref), call
        assert cg.staging_fallbacks() == (0, 0)
    # and the oracle, by the parity rules of the other GPU tests
    yo, so = oracle_lib.solve_cells(wl.mech, wl.cells, wl.dt, wl.rtol, wl.atol)
    rep = compare(y, st, yo, so, oracle_lib, wl, wl.cells, label="noalloc 333 cells")
    print("noalloc:", rep.summary())


def test_noalloc_photolysis_theta_fp32_lu(cg):
    # per-cell photolysis J[n_phot][C], a nonzero theta and the FP32 LU, on two calls
    wl = synth.workload_batching(257)
    mech = cg.Mechanism(wl.mech)
    theta = np.linspace(-0.3, 0.3, wl.mech.n_reactions)
    y_ref, st_ref = _regular(cg, mech, wl, theta=theta, lu_precision=32)
    opts = _opts(cg, wl, lu_precision=32)
    for call in range(2):
        y, st = _noalloc(cg, mech, wl, opts, theta=theta)
        assert np.array_equal(y, y_ref) and np.array_equal(st, st_ref), call


def test_noalloc_staging_fallback_counter(cg):
    # stage_wait = -1 makes every block skip its wait for the staged tables and read
    # them from global memory: the same bytes, so the same results, and one fallback
    # per block (4 cells per block, one block per SM: min(SMs, ceil(C / 4)) blocks)
    wl = synth.workload_tropo(333)
    mech = cg.Mechanism(wl.mech)
    y0, st0 = _noalloc(cg, mech, wl, _opts(cg, wl, cells_per_block=4, blocks_per_sm=1))
    assert cg.staging_fallbacks() == (0, 0)
    y1, st1 = _noalloc(cg, mech, wl, _opts(cg, wl, cells_per_block=4, blocks_per_sm=1, stage_wait=-1))
    n_sm = torch.cuda.get_device_properties(_dev()).multi_processor_count
    assert cg.staging_fallbacks() == (min(n_sm, -(-333 // 4)), 0)
    assert np.array_equal(y0, y1) and np.array_equal(st0, st1)


def test_noalloc_refuses_bad_arguments(cg):
    L = cg.load()
    wl = synth.workload_tropo(64)
    mech = cg.Mechanism(wl.mech)
    dev = _dev()
    C = wl.cells.n_cells
    T = torch.from_numpy(wl.cells.T).to(dev)
    P = torch.from_numpy(wl.cells.P).to(dev)
    y = torch.from_numpy(wl.cells.y).to(dev)
    stats = torch.zeros((C, cg.STATS_DTYPE.itemsize // 8), dtype=torch.int64, device=dev)
    stream = ct.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    opts = _opts(cg, wl)
    host_T = np.array(wl.cells.T)

    def call(n, Tp, opts_=opts):
        return L.chem_solve_step_noalloc(mech.handle, n, Tp, _p(P), None, None, _p(y), _p(stats), wl.dt,
                                         ct.byref(opts_), stream)

    # a host pointer is refused before any launch: y keeps its input
    rc = call(C, ct.c_void_p(host_T.ctypes.data))
    assert rc == -1 and "host memory" in L.chem_last_error().decode()
    torch.cuda.synchronize(dev)
    assert np.array_equal(y.cpu().numpy(), wl.cells.y)
    # so is the adjoint tape, which only a batch can hold
    rc = call(C, _p(T), _opts(cg, wl, record_adjoint=1))
    assert rc == -1 and "record_adjoint" in L.chem_last_error().decode()
    # sizes beyond the stated maximum are refused with a clear error
    rc = call(1 << 31, _p(T))
    assert rc == -1 and "CHEM_NOALLOC_MAX_CELLS" in L.chem_last_error().decode()
    torch.cuda.synchronize(dev)
    assert np.array_equal(y.cpu().numpy(), wl.cells.y)
