"""The oracle over cell shards in worker processes, one per host core.

TEST INFRASTRUCTURE ONLY, like the rest of this package: tests and the
benchmark's CPU-baseline leg use it to run the plain single-threaded oracle on
every cell of a full-size batch.  Each worker runs the unchanged oracle
(``oracle.solve_cells``, ``oracle.adjoint``) on a contiguous shard of cells;
cells are independent, so the shards' results are exactly those of one
sequential run.  Workers are started with the 'spawn' method: a child forked
from a process that has already used a GPU can hang.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

import numpy as np


def n_workers(workers: int | None = None) -> int:
    """Worker count: the host's cores unless given."""
    n = workers or os.cpu_count() or 1
    return max(1, int(n))


class Workers:
    """A set of spawned oracle worker processes kept for several calls (pass it
    as `executor`); a context manager."""

    def __init__(self, workers: int | None = None):
        self.n = n_workers(workers)
        self.ex = ProcessPoolExecutor(max_workers=self.n, mp_context=mp.get_context("spawn"))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.ex.shutdown()


def _run(fn, tasks, nw, executor):
    """Results of fn over tasks, in order: in this process, on the given
    Workers, or on a pool made for this call."""
    if executor is not None:
        return list(executor.ex.map(fn, tasks))
    if nw == 1:
        return [fn(t) for t in tasks]
    with ProcessPoolExecutor(max_workers=min(nw, len(tasks)), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, tasks))


def _shards(n: int, parts: int):
    parts = max(1, min(parts, n))
    bounds = np.linspace(0, n, parts + 1).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]


def _solve_shard(args):
    mech, T, P, J, y, dt, rtol, atol, n_steps, max_steps, theta, between, first_step = args
    import oracle
    from paper_2501_00011_gb300 import synth
    cells = synth.Cells(T=np.array(T), P=np.array(P), y=np.array(y), J=None if J is None else np.array(J))
    st = None
    for k in range(n_steps):
        cells.y, st = oracle.solve_cells(mech, cells, dt, rtol, atol, max_steps=max_steps, theta=theta)
        if between is not None and k + 1 < n_steps:
            between(cells.y, cells.T, first_step + k)
    return cells.y, st


def solve(mech, cells, dt, rtol, atol, n_steps: int = 1, max_steps: int = 5000, theta=None, between=None,
          first_step: int = 0, workers: int | None = None, chunks_per_worker: int = 4, executor=None):
    """n_steps consecutive oracle solves of every cell of a synth.Cells batch.

    between(y, T, step) (a picklable top-level function, may be None) runs on a
    shard's columns after every step but the last, as a host model would
    between chemistry steps; it must act on each cell alone.  Returns
    (y [S, C], stats of the last step [C])."""
    import oracle
    C = cells.n_cells
    if C == 0:
        return np.array(cells.y, np.float64), np.zeros(0, oracle.STATS_DTYPE)
    nw = executor.n if executor is not None else n_workers(workers)
    shards = _shards(C, nw * chunks_per_worker)
    tasks = []
    for a, b in shards:
        J = None if cells.J is None else cells.J[:, a:b]
        tasks.append((mech, cells.T[a:b], cells.P[a:b], J, cells.y[:, a:b], dt, rtol, atol, n_steps, max_steps,
                      theta, between, first_step))
    y = np.empty_like(np.asarray(cells.y, np.float64))
    st = np.zeros(C, oracle.STATS_DTYPE)
    for (a, b), (ys, ss) in zip(shards, _run(_solve_shard, tasks, nw, executor)):
        y[:, a:b], st[a:b] = ys, ss
    return y, st


def _adjoint_shard(args):
    mech, T, P, J, theta, y0, tapes, lam = args
    import oracle
    S, n = y0.shape
    ly0 = np.zeros((S, n))
    g = np.zeros((n, mech.n_reactions))
    for k in range(n):
        kt = oracle.rate_constants(mech, T[k], P[k], jphot=None if J is None else J[:, k], theta=theta)
        ly0[:, k], g[k] = oracle.adjoint(mech, kt, y0[:, k], tapes[k], lam[:, k])
    return ly0, g


def adjoint(mech, cells, tapes, lam, theta=None, workers: int | None = None, chunks_per_worker: int = 4,
            executor=None):
    """The oracle's discrete adjoint of every cell's tape (oracle.Tape, one per
    cell): (dL/dy0 [S, C], per-cell dL/dtheta [C, R]) for dL/dy_final = lam [S, C]."""
    C = cells.n_cells
    nw = executor.n if executor is not None else n_workers(workers)
    shards = _shards(C, nw * chunks_per_worker)
    tasks = [(mech, cells.T[a:b], cells.P[a:b], None if cells.J is None else cells.J[:, a:b], theta,
              np.ascontiguousarray(cells.y[:, a:b]), tapes[a:b], np.ascontiguousarray(lam[:, a:b]))
             for a, b in shards]
    ly0 = np.zeros((mech.n_species, C))
    g = np.zeros((C, mech.n_reactions))
    for (a, b), (l, gg) in zip(shards, _run(_adjoint_shard, tasks, nw, executor)):
        ly0[:, a:b], g[a:b] = l, gg
    return ly0, g


def _forward_adjoint_shard(args):
    mech, T, P, y0, dt, n_steps, rtol, atol, lam = args
    import oracle
    S, n = y0.shape
    ly0 = np.zeros((S, n))
    g = np.zeros(mech.n_reactions)
    for k in range(n):
        kt = oracle.rate_constants(mech, T[k], P[k])
        _, _, tape = oracle.integrate_steps(mech, kt, y0[:, k], dt, n_steps, rtol, atol)
        ly0[:, k], gk = oracle.adjoint(mech, kt, y0[:, k], tape, lam[:, k])
        g += gk
    return ly0, g


def forward_adjoint(mech, cells, dt, n_steps, rtol, atol, lam, workers: int | None = None, executor=None,
                    chunks_per_worker: int = 4):
    """The oracle's whole differentiation workload: per cell n_steps solves
    recording the tape, then the discrete adjoint of the tape for dL/dy_final =
    lam [S, C].  Returns (dL/dy0 [S, C], dL/dtheta [R] summed over cells)."""
    C = cells.n_cells
    nw = executor.n if executor is not None else n_workers(workers)
    shards = _shards(C, nw * chunks_per_worker)
    tasks = [(mech, cells.T[a:b], cells.P[a:b], np.ascontiguousarray(cells.y[:, a:b]), dt, n_steps, rtol, atol,
              np.ascontiguousarray(lam[:, a:b])) for a, b in shards]
    ly0 = np.zeros((mech.n_species, C))
    g = np.zeros(mech.n_reactions)
    for (a, b), (l, gg) in zip(shards, _run(_forward_adjoint_shard, tasks, nw, executor)):
        ly0[:, a:b] = l
        g += gg
    return ly0, g
