"""Python binding of the CPU oracle (ctypes over oracle/oracle.c).

TEST INFRASTRUCTURE ONLY: tests, the smoke check and the benchmark's CPU
baseline may use it; the product path (the CUDA library and its binding) never
imports it.  It shares no code with the CUDA path; both are fed from the seeded
input generators in ``paper_2501_00011_gb300.synth``.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SOURCES = ["oracle.c", "adjoint.c"]
_lock = threading.Lock()
_lib = None

STATUS = {0: "OK", 1: "MAX_STEPS", 2: "H_TOO_SMALL", 3: "ERR_FAIL", 4: "CONV_FAIL",
          5: "NONFINITE", 6: "BAD_INPUT"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction) into oracle/_build."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    deps = srcs + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(d) for d in deps):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Mech(ct.Structure):
    _fields_ = [("n_species", ct.c_int32), ("n_reactions", ct.c_int32),
                ("kind", ct.c_void_p), ("n_reac", ct.c_void_p), ("reac", ct.c_void_p),
                ("n_prod", ct.c_void_p), ("prod", ct.c_void_p),
                ("yld", ct.c_void_p), ("A", ct.c_void_p), ("Ea", ct.c_void_p),
                ("B", ct.c_void_p), ("J", ct.c_void_p), ("ext", ct.c_void_p)]


class _Opts(ct.Structure):
    _fields_ = [("rtol", ct.c_double), ("atol", ct.c_double),
                ("max_order", ct.c_int32), ("max_steps", ct.c_int32),
                ("fixed_h", ct.c_double), ("fixed_order", ct.c_int32),
                ("newton_maxiter", ct.c_int32), ("newton_tol", ct.c_double),
                ("init_D", ct.c_void_p), ("y_hist", ct.c_void_p), ("plain_form", ct.c_int32)]


class _Stats(ct.Structure):
    _fields_ = [("status", ct.c_int32), ("steps", ct.c_int32), ("rejects", ct.c_int32),
                ("conv_fails", ct.c_int32), ("newton_iters", ct.c_int32), ("f_evals", ct.c_int32),
                ("jac_evals", ct.c_int32), ("solves", ct.c_int32), ("final_order", ct.c_int32),
                ("order_sum", ct.c_int32), ("final_h", ct.c_double)]


STATS_DTYPE = np.dtype([("status", "<i4"), ("steps", "<i4"), ("rejects", "<i4"),
                        ("conv_fails", "<i4"), ("newton_iters", "<i4"), ("f_evals", "<i4"),
                        ("jac_evals", "<i4"), ("solves", "<i4"), ("final_order", "<i4"),
                        ("order_sum", "<i4"), ("final_h", "<f8")])
assert STATS_DTYPE.itemsize == ct.sizeof(_Stats)


class _Tape(ct.Structure):
    _fields_ = [("cap", ct.c_int32), ("n", ct.c_int32), ("overflow", ct.c_int32), ("pad", ct.c_int32),
                ("kind", ct.c_void_p), ("q", ct.c_void_p), ("val", ct.c_void_p), ("y", ct.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ct.CDLL(build())
            P = ct.c_void_p
            L.orc_rate_constants.argtypes = [P, ct.c_double, ct.c_double, P, P, P]
            L.orc_deriv.argtypes = [P, P, P, P]
            L.orc_jacobian.argtypes = [P, P, P, P]
            L.orc_lu_factor.argtypes = [ct.c_int, P, P]
            L.orc_lu_factor.restype = ct.c_int
            L.orc_lu_solve.argtypes = [ct.c_int, P, P, P]
            L.orc_rescale.argtypes = [ct.c_int, ct.c_int, ct.c_double, P]
            L.orc_grid_eta.argtypes = [ct.c_double, ct.c_int, ct.c_double]
            L.orc_grid_eta.restype = ct.c_double
            L.orc_integrate.argtypes = [P, P, P, ct.c_double, P, P, P]
            L.orc_integrate.restype = ct.c_int
            L.orc_solve_cells.argtypes = [P, ct.c_int64, P, P, P, P, P, ct.c_double, P, P]
            L.orc_solve_cells.restype = ct.c_int
            if hasattr(L, "orc_adjoint"):
                L.orc_adjoint.argtypes = [P, P, P, P, P, P, P]
                L.orc_adjoint.restype = ct.c_int
                L.orc_replay.argtypes = [P, P, P, P, P, P, P]
                L.orc_replay.restype = ct.c_int
                L.orc_tangent.argtypes = [P, P, P, P, P, P, P]
                L.orc_tangent.restype = ct.c_int
            _lib = L
        return _lib


def _p(a: np.ndarray | None):
    return None if a is None else ct.c_void_p(a.ctypes.data)


class OracleMechanism:
    """Keeps the arrays of a synth.Mechanism alive behind an orc_mech struct."""

    def __init__(self, mech):
        self.mech = mech
        self.S, self.R = mech.n_species, mech.n_reactions
        self._arrs = dict(
            kind=np.ascontiguousarray(mech.kind, np.int32),
            n_reac=np.ascontiguousarray(mech.n_reac, np.int32),
            reac=np.ascontiguousarray(mech.reac, np.int32),
            n_prod=np.ascontiguousarray(mech.n_prod, np.int32),
            prod=np.ascontiguousarray(mech.prod, np.int32),
            yld=np.ascontiguousarray(mech.yld, np.float64),
            A=np.ascontiguousarray(mech.A, np.float64), Ea=np.ascontiguousarray(mech.Ea, np.float64),
            B=np.ascontiguousarray(mech.B, np.float64), J=np.ascontiguousarray(mech.J, np.float64),
            ext=np.ascontiguousarray(np.zeros((self.R, 8)) if getattr(mech, "ext", None) is None else mech.ext,
                                     np.float64))
        assert self._arrs["reac"].shape[1] == 3 and self._arrs["prod"].shape[1] == 8
        a = self._arrs
        self.c = _Mech(self.S, self.R, *(a[k].ctypes.data for k in
                                         ("kind", "n_reac", "reac", "n_prod", "prod", "yld", "A", "Ea", "B", "J",
                                          "ext")))
        self.n_phot = int(np.count_nonzero(a["kind"] == 1))

    @property
    def ref(self):
        return ct.byref(self.c)


def _mk(mech) -> OracleMechanism:
    return mech if isinstance(mech, OracleMechanism) else OracleMechanism(mech)


def rate_constants(mech, T: float, P: float, jphot=None, theta=None) -> np.ndarray:
    m = _mk(mech)
    kt = np.empty(m.R)
    jp = None if jphot is None else np.ascontiguousarray(jphot, np.float64)
    th = None if theta is None else np.ascontiguousarray(theta, np.float64)
    lib().orc_rate_constants(m.ref, float(T), float(P), _p(jp), _p(th), _p(kt))
    return kt


def deriv(mech, kt, y) -> np.ndarray:
    m = _mk(mech)
    kt = np.ascontiguousarray(kt, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    f = np.empty(m.S)
    lib().orc_deriv(m.ref, _p(kt), _p(y), _p(f))
    return f


def jacobian(mech, kt, y) -> np.ndarray:
    m = _mk(mech)
    kt = np.ascontiguousarray(kt, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    J = np.empty((m.S, m.S))
    lib().orc_jacobian(m.ref, _p(kt), _p(y), _p(J))
    return J


def lu_solve_dense(A, b) -> np.ndarray:
    A = np.array(A, np.float64, order="C")
    b = np.array(b, np.float64)
    n = A.shape[0]
    piv = np.empty(n, np.int32)
    if lib().orc_lu_factor(n, _p(A), _p(piv)) != 0:
        raise ZeroDivisionError("exactly singular matrix")
    lib().orc_lu_solve(n, _p(A), _p(piv), _p(b))
    return b


def rescale(D, q: int, eta: float) -> np.ndarray:
    D = np.array(D, np.float64, order="C")
    lib().orc_rescale(D.shape[1], int(q), float(eta), _p(D))
    return D


def grid_eta(err2: float, p: int, bias: float) -> float:
    """Step factor for the squared error estimate err2 (see orc_grid_eta)."""
    return lib().orc_grid_eta(float(err2), int(p), float(bias))


@dataclass
class Tape:
    kind: np.ndarray
    q: np.ndarray
    val: np.ndarray
    y: np.ndarray

    @property
    def n_steps(self) -> int:
        return int(np.count_nonzero(self.kind == 2))


def _opts(rtol, atol, max_order=5, max_steps=5000, fixed_h=0.0, fixed_order=0, newton_maxiter=0,
          newton_tol=0.0, init_D=None, y_hist=None, plain_form=False):
    return _Opts(rtol, atol, max_order, max_steps, fixed_h, fixed_order, newton_maxiter, newton_tol,
                 None if init_D is None else init_D.ctypes.data,
                 None if y_hist is None else y_hist.ctypes.data, int(bool(plain_form)))


def integrate(mech, kt, y0, dt, rtol, atol, max_order=5, max_steps=5000, fixed_h=0.0, fixed_order=0,
              newton_maxiter=0, newton_tol=0.0, init_D=None, n_hist=0, tape_cap=0):
    """Integrate one cell.  Returns (y, stats-dict[, y_hist][, tape])."""
    m = _mk(mech)
    y = np.array(y0, np.float64)
    kt = np.ascontiguousarray(kt, np.float64)
    D = None if init_D is None else np.ascontiguousarray(init_D, np.float64)
    hist = np.zeros((n_hist, m.S)) if n_hist else None
    o = _opts(rtol, atol, max_order, max_steps, fixed_h, fixed_order, newton_maxiter, newton_tol, D, hist)
    st = _Stats()
    tape = None
    tp = None
    if tape_cap:
        tape = Tape(np.zeros(tape_cap, np.int32), np.zeros(tape_cap, np.int32), np.zeros(tape_cap),
                    np.zeros((tape_cap, m.S)))
        tp = _Tape(tape_cap, 0, 0, 0, tape.kind.ctypes.data, tape.q.ctypes.data, tape.val.ctypes.data,
                   tape.y.ctypes.data)
    lib().orc_integrate(m.ref, _p(kt), _p(y), float(dt), ct.byref(o), ct.byref(st),
                        None if tp is None else ct.byref(tp))
    stats = {k: getattr(st, k) for k, _ in _Stats._fields_}
    out = [y, stats]
    if n_hist:
        out.append(hist)
    if tape_cap:
        if tp.overflow:
            raise RuntimeError("tape overflow")
        n = tp.n
        out.append(Tape(tape.kind[:n].copy(), tape.q[:n].copy(), tape.val[:n].copy(), tape.y[:n].copy()))
    return tuple(out)


def solve_cells(mech, cells, dt, rtol, atol, max_order=5, max_steps=5000, theta=None, jphot="cells",
                plain_form=False):
    """Solve every cell of a synth.Cells batch once over [0, dt].

    Returns (y [S, C], stats structured array [C]).  ``jphot="cells"`` uses the
    batch's per-cell photolysis rates when it has them.  plain_form: make every
    test in its plain form (square-root norms, divisions), for the pin that
    the default squared form decides the same."""
    m = _mk(mech)
    y = np.array(cells.y, np.float64, order="C")
    C = y.shape[1]
    T = np.ascontiguousarray(cells.T, np.float64)
    P = np.ascontiguousarray(cells.P, np.float64)
    jp = cells.J if (isinstance(jphot, str) and jphot == "cells") else jphot
    jp = None if jp is None else np.ascontiguousarray(jp, np.float64)
    th = None if theta is None else np.ascontiguousarray(theta, np.float64)
    st = np.zeros(C, STATS_DTYPE)
    o = _opts(rtol, atol, max_order, max_steps, plain_form=plain_form)
    lib().orc_solve_cells(m.ref, C, _p(T), _p(P), _p(jp), _p(th), _p(y), float(dt), ct.byref(o), _p(st))
    return y, st


def _tape_struct(tape: Tape):
    arrs = (np.ascontiguousarray(tape.kind, np.int32), np.ascontiguousarray(tape.q, np.int32),
            np.ascontiguousarray(tape.val, np.float64), np.ascontiguousarray(tape.y, np.float64))
    n = arrs[0].size
    return _Tape(n, n, 0, 0, *(a.ctypes.data for a in arrs)), arrs


def integrate_steps(mech, kt, y0, dt, n_steps, rtol, atol, max_order=5, max_steps=5000, tape_cap=20000):
    """n_steps consecutive solves of one cell; returns (y, [stats], concatenated Tape)."""
    y = np.array(y0, np.float64)
    stats, parts = [], []
    for _ in range(n_steps):
        y, st, tp = integrate(mech, kt, y, dt, rtol, atol, max_order=max_order, max_steps=max_steps,
                              tape_cap=tape_cap)
        stats.append(st)
        parts.append(tp)
    tape = Tape(np.concatenate([p.kind for p in parts]), np.concatenate([p.q for p in parts]),
                np.concatenate([p.val for p in parts]), np.concatenate([p.y for p in parts]))
    return y, stats, tape


def replay(mech, kt, y0, tape: Tape, keep_steps=False, kt_M=None):
    """The frozen-control map of a tape: y0 -> y_final (and y after every STEP event).

    The iteration matrices are formed with the rate constants kt_M (default kt):
    pass the recorded run's constants to perturb kt with the matrices frozen."""
    m = _mk(mech)
    ts, keep = _tape_struct(tape)
    y0 = np.ascontiguousarray(y0, np.float64)
    out = np.empty(m.S)
    ys = np.zeros((tape.kind.size, m.S)) if keep_steps else None
    ktM = None if kt_M is None else np.ascontiguousarray(kt_M, np.float64)
    kt = np.ascontiguousarray(kt, np.float64)
    rc = lib().orc_replay(m.ref, _p(kt), _p(ktM), _p(y0), ct.byref(ts), _p(out), _p(ys))
    if rc:
        raise RuntimeError("replay: singular or missing iteration matrix")
    return (out, ys) if keep_steps else out


def tangent(mech, kt, y0, tape: Tape, dy0, dtheta):
    m = _mk(mech)
    ts, keep = _tape_struct(tape)
    out = np.empty(m.S)
    # contiguous copies held in locals: they must outlive the call
    kt, y0, dy0, dtheta = (np.ascontiguousarray(a, np.float64) for a in (kt, y0, dy0, dtheta))
    rc = lib().orc_tangent(m.ref, _p(kt), _p(y0), ct.byref(ts), _p(dy0), _p(dtheta), _p(out))
    if rc:
        raise RuntimeError("tangent: singular or missing iteration matrix")
    return out


def adjoint(mech, kt, y0, tape: Tape, lam_final):
    """(dL/dy0, dL/dtheta) of the frozen-control map for dL/dy_final = lam_final."""
    m = _mk(mech)
    ts, keep = _tape_struct(tape)
    ly0 = np.empty(m.S)
    g = np.empty(m.R)
    # contiguous copies held in locals: they must outlive the call
    kt, y0, lam_final = (np.ascontiguousarray(a, np.float64) for a in (kt, y0, lam_final))
    rc = lib().orc_adjoint(m.ref, _p(kt), _p(y0), ct.byref(ts), _p(lam_final), _p(ly0), _p(g))
    if rc:
        raise RuntimeError("adjoint: singular or missing iteration matrix")
    return ly0, g


# ---------------------------------------------------------------- coupled cells
# The paper's multi-cell system (Implementations, Multi-cells): the cells of a
# group are integrated as one ODE system.  The oracle writes that system out as
# one mechanism over all the group's species, reaction j of cell g acting on
# species g*S + s with cell g's rate constant, and integrates it with the same
# integrator (one step size, order and Newton iteration, one WRMS norm over
# every species of the group; the dense LU factors the block-diagonal matrix).

def replicate(mech, G: int):
    """The mechanism of G cells as one system (species g*S + s, reactions g*R + j)."""
    from paper_2501_00011_gb300 import synth
    S, R = mech.n_species, mech.n_reactions
    big = synth.empty_mechanism(G * S, G * R, f"{mech.name}_x{G}")
    for g in range(G):
        sl = slice(g * R, (g + 1) * R)
        big.kind[sl] = mech.kind
        big.n_reac[sl] = mech.n_reac
        big.n_prod[sl] = mech.n_prod
        big.reac[sl] = np.where(mech.reac >= 0, mech.reac + g * S, -1)
        big.prod[sl] = np.where(mech.prod >= 0, mech.prod + g * S, -1)
        big.yld[sl] = mech.yld
        big.A[sl], big.Ea[sl], big.B[sl], big.J[sl] = mech.A, mech.Ea, mech.B, mech.J
        big.ext[sl] = synth.rate_ext(mech)
    return big


def solve_coupled(mech, cells, dt, rtol, atol, G: int, max_order=5, max_steps=5000):
    """Every group of G consecutive cells (the last may be shorter) integrated as one
    system over [0, dt].  Returns (y [S, C], stats [C]: each cell has its group's)."""
    S, C = mech.n_species, cells.n_cells
    y = np.array(cells.y, np.float64, order="C")
    st = np.zeros(C, STATS_DTYPE)
    for c0 in range(0, C, G):
        idx = np.arange(c0, min(C, c0 + G))
        big = replicate(mech, idx.size)
        kt = np.concatenate([rate_constants(mech, cells.T[c], cells.P[c],
                                            jphot=None if cells.J is None else cells.J[:, c]) for c in idx])
        y0 = np.concatenate([cells.y[:, c] for c in idx])
        yg, sg = integrate(big, kt, y0, dt, rtol, atol, max_order=max_order, max_steps=max_steps)
        y[:, idx] = yg.reshape(idx.size, S).T
        for c in idx:
            for k in STATS_DTYPE.names:
                if k in sg:
                    st[c][k] = sg[k]
    return y, st
