"""Shared parity checks of the GPU path against the oracle (test helpers).

Tolerances.  The FP64 path must match the oracle within a relative error of
1e-6 on every species above 1e-10 mol/mol.  Both sides run the same written
integrator; their arithmetic differs only in rounding order (FMA contraction,
warp reductions, exp/pow last bits, sparse static-order vs dense pivoted LU).
Where the discrete map is ill-conditioned those rounding differences are
amplified: in a few cells the oracle's own result moves by up to 4e-4
relative (and, with host work between steps, by up to 20% and 5 tolerance
units) when its inputs are perturbed at the 1e-15 level, with identical step
sequences; the spread is heavy-tailed (for one 50,000-cell batching cell, 4
perturbed runs reach 4e-5 and 64 runs 4e-4).  Such a result is not determined
beyond rounding, so for a cell above the 1e-6 bar the check measures the
oracle's rounding spread over 16 perturbed runs and requires the GPU to lie
within 10x that spread, both relative and in tolerance units, and within one
tolerance unit where the spread is smaller ("rounding-limited" cells).
Cells whose step sequence differs (a borderline accept/converge decision
flipped by rounding: "flips") must agree within 10 tolerance units, or, where
the caller allows it, be no less accurate than the oracle's result against a
tight reference.  The counts of both kinds are bounded by max_odd_frac and
reported in every assertion message.

Full-size batches run the oracle on all host cores (oracle.pool), so every
cell is compared, not a sample.
"""
from dataclasses import dataclass

import numpy as np

from oracle import pool
from paper_2501_00011_gb300 import synth

FLOOR = 1e-10
REL = 1e-6


@dataclass
class Parity:
    """Outcome of compare(): iterating gives (worst, flips, odd) for older callers."""
    n_cells: int
    worst: float            # max rel err over well-determined cells with identical step sequences
    flips: int              # cells whose step sequence differs from the oracle's
    odd: int                # rounding-limited cells (above REL, within 10x the oracle's own spread)
    flip_units: float       # largest difference of a flipped cell, tolerance units
    odd_rel: float          # largest rel err of a rounding-limited cell
    odd_units: float = 0.0  # largest difference of a rounding-limited cell, tolerance units

    def __iter__(self):
        return iter((self.worst, self.flips, self.odd))

    def summary(self) -> str:
        return (f"{self.n_cells} cells: max rel err {self.worst:.2e} on identical step sequences; "
                f"flips {self.flips} (max {self.flip_units:.2f} tolerance units); "
                f"rounding-limited {self.odd} (max rel err {self.odd_rel:.2e}, {self.odd_units:.2f} tolerance units)")


def oracle_steps(oracle_lib, wl, cells, n_steps, between=None, rtol=None, atol=None, max_steps=5000):
    """The oracle over n_steps consecutive solves of wl.dt (all host cores for
    large batches); stats of the last.  between(y, T, step) runs between steps."""
    rtol = wl.rtol if rtol is None else rtol
    atol = wl.atol if atol is None else atol
    if cells.n_cells >= 64:
        return pool.solve(wl.mech, cells, wl.dt, rtol, atol, n_steps=n_steps, between=between, max_steps=max_steps)
    cur = synth.subset(cells, np.arange(cells.n_cells))
    st = None
    for k in range(n_steps):
        cur.y, st = oracle_lib.solve_cells(wl.mech, cur, wl.dt, rtol, atol, max_steps=max_steps)
        if between is not None and k + 1 < n_steps:
            between(cur.y, cur.T, k)
    return cur.y, st


def spreads(oracle_lib, wl, cells, idx, n_steps=1, n=16, between=None, units=False):
    """For every cell in idx, the largest relative move (on species above the
    floor) of the oracle's result when its input state is perturbed by 1e-15
    relative (rounding-level noise), over n perturbed runs; with units=True
    also the largest move in tolerance units."""
    idx = np.asarray(idx, np.int64)
    if idx.size == 0:
        return (np.zeros(0), np.zeros(0)) if units else np.zeros(0)
    rep = np.repeat(idx, n)
    sub = synth.subset(cells, rep)
    rng = np.random.default_rng(int(idx[0]))
    sub.y = sub.y * (1 + 1e-15 * rng.standard_normal(sub.y.shape))
    yp, _ = oracle_steps(oracle_lib, wl, sub, n_steps, between)
    yo, _ = oracle_steps(oracle_lib, wl, synth.subset(cells, idx), n_steps, between)
    out = np.zeros(idx.size)
    out_units = np.zeros(idx.size)
    for i in range(idx.size):
        ref = yo[:, i]
        mask = np.abs(ref) > FLOOR
        diff = np.abs(yp[:, i * n:(i + 1) * n] - ref[:, None])
        d = diff[mask] / np.abs(ref[mask])[:, None]
        out[i] = float(d.max()) if d.size else 0.0
        out_units[i] = float((diff / (wl.rtol * np.abs(ref) + wl.atol)[:, None]).max())
    return (out, out_units) if units else out


def spread(oracle_lib, wl, cells, c, n_steps=1, n=16, between=None):
    return float(spreads(oracle_lib, wl, cells, [c], n_steps, n, between)[0])


def tight_errors(oracle_lib, wl, cells, idx, y, yo, n_steps=1, between=None):
    """Errors of y and yo (columns idx) against the oracle at rtol 1e-10, atol 1e-18,
    in tolerance units of the workload, max over species."""
    idx = np.asarray(idx, np.int64)
    sub = synth.subset(cells, idx)
    yt, stt = oracle_steps(oracle_lib, wl, sub, n_steps, between, rtol=1e-10, atol=1e-18, max_steps=200_000)
    assert np.all(stt["status"] == 0)
    unit = wl.rtol * np.abs(yt) + wl.atol
    return (np.abs(y[:, idx] - yt) / unit).max(axis=0), (np.abs(yo[:, idx] - yt) / unit).max(axis=0)


def compare(y, st, yo, so, oracle_lib=None, wl=None, cells=None, n_steps=1, max_odd_frac=0.03, tight_flips=False,
            between=None, label=""):
    """Parity of a batch (every column of y against the oracle's yo).

    cells is the input batch whose columns y / yo hold the results.  With
    tight_flips, a cell whose step sequence differs may lie farther than 10
    tolerance units from the oracle's result if it is no less accurate than the
    oracle's against a tight reference (both are correct results: the tolerance
    bounds each step's local error, not the global one)."""
    tag = f"[{label}] " if label else ""
    bad_status = np.nonzero(st["status"] != so["status"])[0]
    assert bad_status.size == 0, f"{tag}status differs on {bad_status.size} cells, e.g. {bad_status[:8].tolist()}"
    ok = so["status"] == 0
    same = (st["steps"] == so["steps"]) & (st["newton_iters"] == so["newton_iters"])
    tol = wl.rtol * np.abs(yo) + wl.atol
    n_ok = max(1, int(ok.sum()))
    units = np.max(np.abs(y - yo) / tol, axis=0)
    flips = np.nonzero(ok & ~same)[0]
    far = flips[units[flips] > 10.0]
    if far.size:
        assert tight_flips, f"{tag}{far.size} flipped cells beyond 10 tolerance units: " \
                            f"{[(int(c), round(float(units[c]), 2)) for c in far[:8]]}"
        eg, eo = tight_errors(oracle_lib, wl, cells, far, y, yo, n_steps, between)
        bad = eg > 1.25 * eo + 1.0
        assert not bad.any(), f"{tag}flipped cells less accurate than the oracle (cell, GPU and oracle errors " \
                              f"against the tight reference in tolerance units): " \
                              f"{[(int(c), round(float(a), 2), round(float(b), 2)) for c, a, b in zip(far[bad], eg[bad], eo[bad])][:8]}"
    # relative errors of the cells with identical step sequences
    absy = np.abs(yo)
    mask = absy > FLOOR
    rel = np.where(mask, np.abs(y - yo) / np.where(mask, absy, 1.0), 0.0).max(axis=0)
    cand = np.nonzero(ok & same)[0]
    odd = cand[rel[cand] > REL]
    worst = float(rel[cand[rel[cand] <= REL]].max()) if np.any(rel[cand] <= REL) else 0.0
    if odd.size:
        sp, sp_units = spreads(oracle_lib, wl, cells, odd, n_steps, between=between, units=True)
        beyond = [(int(c), float(rel[c]), float(s), float(units[c]), float(su))
                  for c, s, su in zip(odd, sp, sp_units) if rel[c] > 10 * s or units[c] > max(1.0, 10 * su)]
        assert not beyond, f"{tag}cells beyond 10x the oracle's rounding spread (cell, rel, spread, units, " \
                           f"spread units): {beyond[:8]}"
    rep = Parity(int(y.shape[1]), worst, int(flips.size), int(odd.size),
                 float(units[flips].max()) if flips.size else 0.0, float(rel[odd].max()) if odd.size else 0.0,
                 float(units[odd].max()) if odd.size else 0.0)
    limit = max(2, max_odd_frac * n_ok)
    assert flips.size + odd.size <= limit, f"{tag}too many flipped or rounding-limited cells " \
                                           f"(limit {limit:.0f}): {rep.summary()}"
    return rep


def sample_cells(n_cells, n_sample, seed=0):
    """First, last and evenly spread cells plus a few random ones (sorted, unique)."""
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([[0, n_cells - 1], np.linspace(0, n_cells - 1, n_sample // 2).astype(int),
                                    rng.integers(0, n_cells, n_sample - n_sample // 2)]))
    return idx
