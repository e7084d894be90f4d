"""chem_solve_step_noalloc through the C ABI, against chem_solve_step.

The allocation-free entry point serves callers that may not allocate device
memory while they run (a host model under its own memory manager or a fixed
device budget).  They own every buffer; the library keeps the persistent
driver's work-queue counter in a static device array and clears it on each
call.  Two calls in a row must both reproduce the regular entry point, which
shows the counter is reset between calls.  This file is collected last.
"""
import ctypes as ct

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_00011_gb300 import synth  # noqa: E402

FLOOR, REL = 1e-10, 1e-6     # the FP64 parity tolerance of the other GPU tests


def test_noalloc_matches_solve_step_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_00011_gb300 import build, chemgpu
    build.build()
    torch.cuda.init()
    L = chemgpu.load()
    wl = synth.workload_tropo(333)
    C, S = wl.cells.n_cells, wl.mech.n_species
    mech = chemgpu.Mechanism(wl.mech)
    y_ref, st_ref = chemgpu.solve(mech, wl.cells, wl.dt, wl.rtol, wl.atol, driver="persistent")

    dev = torch.device("cuda", torch.cuda.current_device())
    T = torch.from_numpy(wl.cells.T).to(dev)
    P = torch.from_numpy(wl.cells.P).to(dev)
    stats = torch.zeros((C, chemgpu.STATS_DTYPE.itemsize // 8), dtype=torch.int64, device=dev)
    opts = chemgpu.Opts()
    L.chem_opts_default(ct.byref(opts))
    opts.rtol, opts.atol = wl.rtol, wl.atol
    stream = ct.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    for call in range(2):
        y = torch.from_numpy(wl.cells.y).to(dev)
        stats.zero_()
        rc = L.chem_solve_step_noalloc(mech.handle, C, ct.c_void_p(T.data_ptr()), ct.c_void_p(P.data_ptr()),
                                       None, None, ct.c_void_p(y.data_ptr()), ct.c_void_p(stats.data_ptr()),
                                       wl.dt, ct.byref(opts), stream)
        assert rc == 0, L.chem_last_error().decode()
        torch.cuda.synchronize(dev)
        yn = y.cpu().numpy()
        st = stats.cpu().numpy().view(chemgpu.STATS_DTYPE).reshape(C)
        assert np.array_equal(st["status"], st_ref["status"]), call
        assert np.array_equal(st["steps"], st_ref["steps"]), call
        mask = np.abs(y_ref) > FLOOR
        rel = np.abs(yn - y_ref)[mask] / np.abs(y_ref)[mask]
        assert rel.max() <= REL, (call, rel.max())

    # sizes beyond the stated maximum are refused with a clear error
    rc = L.chem_solve_step_noalloc(mech.handle, (1 << 31), ct.c_void_p(T.data_ptr()), ct.c_void_p(P.data_ptr()),
                                   None, None, ct.c_void_p(T.data_ptr()), ct.c_void_p(stats.data_ptr()),
                                   wl.dt, ct.byref(opts), stream)
    assert rc == -1 and "CHEM_NOALLOC_MAX_CELLS" in L.chem_last_error().decode()
