"""The sharded differentiation path: two ranks (gloo on the host, each with its
own CUDA context on the one GPU; their kernels never wait on each other) each
run their contiguous cell range of a batch forward and through
chem_sensitivity, then sum dL/dtheta over ranks in rank order.  The result
must equal one batch's dL/dtheta to rounding (the per-cell gradients are the
same; only the order of the sum over cells differs), and the ranks' dL/dy0
shards must concatenate to the single batch's bit for bit (a cell's forward
and backward do not depend on the other cells)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_CELLS, N_STEPS = 41, 2


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _solve_and_differentiate(cells, wl, w, chemgpu):
    m = chemgpu.Mechanism(wl.mech)
    c = chemgpu.Cells(m, cells.n_cells, rtol=wl.rtol, atol=wl.atol, driver="persistent", record_adjoint=True)
    c.set_state(cells.T, cells.P, cells.y)
    for _ in range(N_STEPS):
        c.solve_step(wl.dt)
    gth, gy0, n_bad = c.sensitivity(w)
    assert n_bad == 0
    return gth, gy0


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2501_00011_gb300 import chemgpu, shard, synth
        torch.cuda.set_device(0)
        wl = synth.workload_adjoint(N_CELLS)
        b, e = shard.cell_range(N_CELLS, rank, world)
        cells = synth.subset(wl.cells, np.arange(b, e))
        w = synth.loss_weights(wl.mech.n_species, N_CELLS)[:, b:e].copy()
        gth, gy0 = _solve_and_differentiate(cells, wl, w, chemgpu)
        total = shard.reduce_theta_grad(gth)
        q.put((rank, b, e, total, gy0, None))
    except BaseException as exc:          # reported to the parent, which fails the test
        q.put((rank, 0, 0, None, None, repr(exc)))
    finally:
        dist.destroy_process_group()


def test_sharded_adjoint_equals_single_batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import multiprocessing as mp
    from paper_2501_00011_gb300 import build, chemgpu, synth
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=600) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(o[5] is None for o in out), [o[5] for o in out]
    torch.cuda.init()
    chemgpu.load()
    wl = synth.workload_adjoint(N_CELLS)
    w = synth.loss_weights(wl.mech.n_species, N_CELLS)
    gth, gy0 = _solve_and_differentiate(wl.cells, wl, w, chemgpu)
    for rank, b, e, total, gy0_shard, _ in out:
        np.testing.assert_allclose(total, gth, rtol=1e-12, atol=1e-14 * np.abs(gth).max())
        assert np.array_equal(gy0_shard, gy0[:, b:e]), rank
    assert np.array_equal(out[0][3], out[1][3])      # every rank holds the same sum
