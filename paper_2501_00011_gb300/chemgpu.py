"""Thin ctypes binding of libchemgpu.so (include/chemgpu.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; CUDA
tensors are passed as device pointers, everything else as host pointers.
There is no CPU fallback: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "_lib", "libchemgpu.so")

MEM_HOST, MEM_DEVICE = 0, 1
DRIVERS = {"plain": 0, "persistent": 1}
STATUS = {0: "OK", 1: "MAX_STEPS", 2: "H_TOO_SMALL", 3: "ERR_FAIL", 4: "CONV_FAIL",
          5: "NONFINITE", 6: "BAD_INPUT"}

# every symbol include/chemgpu.h declares
EXPORTS = ["chem_opts_default", "chem_mechanism_create", "chem_mechanism_destroy",
           "chem_mechanism_info", "chem_mechanism_structure", "chem_cells_create",
           "chem_cells_destroy", "chem_cells_set_state", "chem_cells_set_photolysis",
           "chem_cells_set_theta", "chem_solve_step", "chem_solve_steps", "chem_autotune",
           "chem_get_state", "chem_get_stats", "chem_staging_fallbacks",
           "chem_eval_deriv", "chem_eval_newton_solve", "chem_eval_deriv_design", "chem_solve_step_noalloc", "chem_sensitivity",
           "chem_sensitivity_checkpointed", "chem_eval_reciprocal", "chem_eval_warp_sum", "chem_measure_fma_peak",
           "chem_tangent", "chem_get_tape", "chem_pipeline_create", "chem_pipeline_destroy", "chem_pipeline_run", "chem_last_error"]


DERIV_GATHER, DERIV_ATOMIC_AOS, DERIV_ATOMIC_SOA = 0, 1, 2


class Reaction(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("n_reac", ct.c_int32), ("reac", ct.c_int32 * 3),
                ("n_prod", ct.c_int32), ("prod", ct.c_int32 * 8), ("yld", ct.c_double * 8),
                ("A", ct.c_double), ("Ea_over_R", ct.c_double), ("B", ct.c_double), ("J", ct.c_double),
                ("A2", ct.c_double), ("Ea2_over_R", ct.c_double), ("B2", ct.c_double),
                ("A3", ct.c_double), ("Ea3_over_R", ct.c_double), ("B3", ct.c_double),
                ("Fc", ct.c_double), ("N", ct.c_double)]


class Opts(ct.Structure):
    _fields_ = [("rtol", ct.c_double), ("atol", ct.c_double), ("max_order", ct.c_int32),
                ("max_steps", ct.c_int32), ("lu_precision", ct.c_int32), ("driver", ct.c_int32),
                ("cells_per_block", ct.c_int32), ("blocks_per_sm", ct.c_int32),
                ("record_adjoint", ct.c_int32), ("tape_steps", ct.c_int32), ("couple_cells", ct.c_int32),
                ("stage_wait", ct.c_int32)]


class MechInfo(ct.Structure):
    _fields_ = [(n, ct.c_int32) for n in (
        "n_species", "n_reactions", "n_photolysis", "nnz_jac", "nnz_lu", "n_pairs",
        "passes_f", "passes_jac", "passes_lu", "passes_fwd", "passes_bwd",
        "ops_f", "ops_jac", "ops_lu", "ops_fwd", "ops_bwd")] + \
        [(n, ct.c_double) for n in ("flops_f", "flops_jac", "flops_lu", "flops_solve")] + \
        [("smem_per_cell_fp64", ct.c_int32), ("smem_per_cell_fp32", ct.c_int32),
         ("flops_adj_iter", ct.c_double), ("flops_tan_iter", ct.c_double)]


STATS_DTYPE = np.dtype([("status", "<i4"), ("steps", "<i4"), ("rejects", "<i4"),
                        ("conv_fails", "<i4"), ("newton_iters", "<i4"), ("f_evals", "<i4"),
                        ("jac_evals", "<i4"), ("solves", "<i4"), ("final_order", "<i4"),
                        ("order_sum", "<i4"), ("final_h", "<f8")])

_lib = None
_lock = threading.Lock()


class ChemError(RuntimeError):
    pass


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or SO_PATH
        if not os.path.exists(p):
            raise ChemError(f"CUDA library not built: {p} (run paper_2501_00011_gb300.build.build())")
        L = ct.CDLL(p)
        V = ct.c_void_p
        L.chem_opts_default.argtypes = [V]
        L.chem_mechanism_create.argtypes = [ct.c_int32, ct.c_int32, V, ct.POINTER(V)]
        L.chem_mechanism_destroy.argtypes = [V]
        L.chem_mechanism_info.argtypes = [V, V]
        L.chem_mechanism_structure.argtypes = [V, V, V]
        L.chem_cells_create.argtypes = [V, ct.c_int64, V, ct.POINTER(V)]
        L.chem_cells_destroy.argtypes = [V]
        L.chem_cells_set_state.argtypes = [V, V, V, V, ct.c_int32, V]
        L.chem_cells_set_photolysis.argtypes = [V, V, ct.c_int32, V]
        L.chem_cells_set_theta.argtypes = [V, V, ct.c_int32, V]
        L.chem_solve_step.argtypes = [V, ct.c_double, V]
        L.chem_get_state.argtypes = [V, V, ct.c_int32, V]
        L.chem_get_stats.argtypes = [V, V, ct.c_int32, V]
        L.chem_staging_fallbacks.argtypes = [V, V, V, V]
        L.chem_eval_deriv.argtypes = [V, V, V, ct.c_int32, V]
        L.chem_eval_newton_solve.argtypes = [V, ct.c_double, V, V, V, ct.c_int32, V]
        L.chem_eval_deriv_design.argtypes = [V, ct.c_int32, V, V, ct.c_int32, V]
        L.chem_solve_step_noalloc.argtypes = [V, ct.c_int64, V, V, V, V, V, V, ct.c_double, V, V]
        L.chem_sensitivity.argtypes = [V, V, V, V, ct.c_int32, V]
        L.chem_eval_reciprocal.argtypes = [V, V, ct.c_int64, ct.c_int32, V]
        L.chem_eval_warp_sum.argtypes = [V, V, ct.c_int64, ct.c_int32, V]
        L.chem_measure_fma_peak.argtypes = [ct.c_int32, V, V, V]
        L.chem_sensitivity_checkpointed.argtypes = [V, V, ct.c_int32, ct.c_double, ct.c_int32, V, V, V, ct.c_int32, V]
        L.chem_tangent.argtypes = [V, V, V, V, ct.c_int32, V]
        L.chem_solve_steps.argtypes = [V, ct.c_double, ct.c_int32, V]
        L.chem_autotune.argtypes = [V, ct.c_double, ct.c_int64, V, V]
        L.chem_get_tape.argtypes = [V, ct.c_int64, V, V, V, V, ct.c_int32, V, V]
        L.chem_pipeline_create.argtypes = [V, ct.c_int64, ct.c_int32, V, ct.POINTER(V)]
        L.chem_pipeline_destroy.argtypes = [V]
        L.chem_pipeline_run.argtypes = [V, V, V, V, V, ct.c_double, ct.c_int32, CHUNK_FN, V, V]
        L.chem_last_error.restype = ct.c_char_p
        for name in EXPORTS:
            if name not in ("chem_opts_default", "chem_mechanism_destroy", "chem_cells_destroy",
                            "chem_pipeline_destroy", "chem_last_error"):
                getattr(L, name).restype = ct.c_int
        _lib = L
        return L


def _check(rc: int, what: str):
    if rc < 0:
        raise ChemError(f"{what} failed ({rc}): {load().chem_last_error().decode()}")
    return rc


def _stream_ptr(stream):
    if stream is not None:
        return ct.c_void_p(getattr(stream, "cuda_stream", stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def _ptr(a, dtype=np.float64):
    """(pointer, mem, keepalive) for a torch tensor or numpy array of float64."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise ChemError("tensors must be contiguous float64")
            return ct.c_void_p(a.data_ptr()), (MEM_DEVICE if a.is_cuda else MEM_HOST), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ct.c_void_p(arr.ctypes.data), MEM_HOST, arr


def reactions_from_synth(m: synth.Mechanism):
    R = m.n_reactions
    arr = (Reaction * max(R, 1))()
    ext = synth.rate_ext(m)
    for j in range(R):
        r = arr[j]
        r.kind = int(m.kind[j])
        r.n_reac = int(m.n_reac[j])
        for s in range(3):
            r.reac[s] = int(m.reac[j, s]) if s < m.n_reac[j] else 0
        r.n_prod = int(m.n_prod[j])
        for p in range(8):
            r.prod[p] = int(m.prod[j, p]) if p < m.n_prod[j] else 0
            r.yld[p] = float(m.yld[j, p]) if p < m.n_prod[j] else 0.0
        r.A, r.Ea_over_R, r.B, r.J = float(m.A[j]), float(m.Ea[j]), float(m.B[j]), float(m.J[j])
        (r.A2, r.Ea2_over_R, r.B2, r.A3, r.Ea3_over_R, r.B3, r.Fc, r.N) = (float(v) for v in ext[j])
    return arr


class Mechanism:
    """A compiled mechanism on the current CUDA device."""

    def __init__(self, mech: synth.Mechanism):
        L = load()
        self.synth = mech
        self.n_species, self.n_reactions = mech.n_species, mech.n_reactions
        rx = reactions_from_synth(mech)
        h = ct.c_void_p()
        _check(L.chem_mechanism_create(self.n_species, self.n_reactions, ct.cast(rx, ct.c_void_p),
                                       ct.byref(h)), "chem_mechanism_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = MechInfo()
        _check(load().chem_mechanism_info(self._h, ct.byref(inf)), "chem_mechanism_info")
        return {k: getattr(inf, k) for k, _ in MechInfo._fields_}

    def structure(self):
        S = self.n_species
        pos = np.zeros(S, np.int32)
        fill = np.zeros((S, S), np.uint8)
        _check(load().chem_mechanism_structure(self._h, ct.c_void_p(pos.ctypes.data),
                                               ct.c_void_p(fill.ctypes.data)), "chem_mechanism_structure")
        return pos, fill

    def close(self):
        if getattr(self, "_h", None):
            load().chem_mechanism_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cells:
    """Device state of a batch of cells."""

    def __init__(self, mech: Mechanism, n_cells: int, rtol: float = 1e-4, atol: float = 1e-10,
                 max_order: int = 5, max_steps: int = 5000, lu_precision: int = 64,
                 driver: str = "plain", cells_per_block: int = 0, blocks_per_sm: int = 0,
                 record_adjoint: bool = False, tape_steps: int = 0, couple_cells: int = 1, stage_wait: int = 0):
        L = load()
        self.mech = mech
        self.n_cells = int(n_cells)
        o = Opts()
        L.chem_opts_default(ct.byref(o))
        o.rtol, o.atol, o.max_order, o.max_steps = rtol, atol, max_order, max_steps
        o.lu_precision, o.driver = lu_precision, DRIVERS[driver]
        o.cells_per_block, o.blocks_per_sm = cells_per_block, blocks_per_sm
        o.record_adjoint, o.tape_steps = int(record_adjoint), tape_steps
        o.couple_cells = int(couple_cells)
        o.stage_wait = int(stage_wait)
        self.opts = o
        h = ct.c_void_p()
        _check(L.chem_cells_create(mech.handle, self.n_cells, ct.byref(o), ct.byref(h)), "chem_cells_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def set_state(self, T, P, y, stream=None):
        (pt, mt, k1), (pp, mp, k2), (py, my, k3) = _ptr(T), _ptr(P), _ptr(y)
        if not (mt == mp == my):
            raise ChemError("T, P and y must all be on the host or all on the device")
        _check(load().chem_cells_set_state(self._h, pt, pp, py, mt, _stream_ptr(stream)), "chem_cells_set_state")

    def set_photolysis(self, J, stream=None):
        if J is None:
            _check(load().chem_cells_set_photolysis(self._h, None, MEM_HOST, None), "chem_cells_set_photolysis")
            return
        pj, mj, keep = _ptr(J)
        _check(load().chem_cells_set_photolysis(self._h, pj, mj, _stream_ptr(stream)), "chem_cells_set_photolysis")

    def set_theta(self, theta, stream=None):
        if theta is None:
            _check(load().chem_cells_set_theta(self._h, None, MEM_HOST, None), "chem_cells_set_theta")
            return
        pt, mt, keep = _ptr(theta)
        _check(load().chem_cells_set_theta(self._h, pt, mt, _stream_ptr(stream)), "chem_cells_set_theta")

    def solve_step(self, dt: float, stream=None):
        _check(load().chem_solve_step(self._h, float(dt), _stream_ptr(stream)), "chem_solve_step")

    def solve_steps(self, dt: float, n_steps: int, stream=None):
        """n_steps consecutive steps of dt as one captured CUDA graph launch."""
        _check(load().chem_solve_steps(self._h, float(dt), int(n_steps), _stream_ptr(stream)), "chem_solve_steps")

    def autotune(self, dt: float, n_sample: int = 0):
        """Measure launch shapes on a sample of the current state; returns (cells_per_block, blocks_per_sm)."""
        w, b = ct.c_int32(0), ct.c_int32(0)
        _check(load().chem_autotune(self._h, float(dt), int(n_sample), ct.byref(w), ct.byref(b)), "chem_autotune")
        return w.value, b.value

    def get_state(self, out=None, stream=None):
        """Returns y [S, C]; into `out` (tensor/array) if given, else a new numpy array."""
        if out is None:
            out = np.empty((self.mech.n_species, self.n_cells))
        po, mo, keep = _ptr(out)
        if isinstance(out, np.ndarray) and keep is not out:
            raise ChemError("out must be a contiguous float64 array")
        _check(load().chem_get_state(self._h, po, mo, _stream_ptr(stream)), "chem_get_state")
        return out

    def get_stats(self, stream=None) -> np.ndarray:
        st = np.zeros(self.n_cells, STATS_DTYPE)
        _check(load().chem_get_stats(self._h, ct.c_void_p(st.ctypes.data), MEM_HOST, _stream_ptr(stream)),
               "chem_get_stats")
        return st

    def staging_fallbacks(self, stream=None):
        """(fallbacks, unfinished) of the last solve call: blocks whose table staging
        fell back to global memory, and blocks that exited before a late copy landed."""
        return staging_fallbacks(self, stream)

    def eval_deriv(self, y, stream=None):
        """f(y) for every cell ([S, C] numpy in, numpy out), on the GPU."""
        yy = np.ascontiguousarray(y, np.float64)
        f = np.empty_like(yy)
        _check(load().chem_eval_deriv(self._h, ct.c_void_p(yy.ctypes.data), ct.c_void_p(f.ctypes.data), MEM_HOST,
                                      _stream_ptr(stream)), "chem_eval_deriv")
        return f

    def eval_newton_solve(self, c: float, y, b, stream=None):
        """x = (I - c J(y))^{-1} b for every cell, on the GPU."""
        yy = np.ascontiguousarray(y, np.float64)
        bb = np.ascontiguousarray(b, np.float64)
        x = np.empty_like(yy)
        _check(load().chem_eval_newton_solve(self._h, float(c), ct.c_void_p(yy.ctypes.data), ct.c_void_p(bb.ctypes.data),
                                             ct.c_void_p(x.ctypes.data), MEM_HOST, _stream_ptr(stream)),
               "chem_eval_newton_solve")
        return x

    def eval_deriv_design(self, design: int, y, out=None, stream=None):
        """f(y) [S, C] by one of the DERIV_* kernel designs (rate constants cached per state)."""
        if out is None:
            out = np.empty((self.mech.n_species, self.n_cells)) if isinstance(y, np.ndarray) else y.new_empty(y.shape)
        (py, my, k1), (po, mo, k2) = _ptr(y), _ptr(out)
        if my != mo:
            raise ChemError("y and out must both be on the host or both on the device")
        _check(load().chem_eval_deriv_design(self._h, int(design), py, po, my, _stream_ptr(stream)),
               "chem_eval_deriv_design")
        return out

    def sensitivity(self, dL_dy, dL_dtheta=None, dL_dy0=None, stream=None):
        """(dL/dtheta [R], dL/dy0 [S, C], n_bad) for L = sum dL_dy * y."""
        R = self.mech.n_reactions
        dy = dL_dy
        if dL_dtheta is None:
            dL_dtheta = np.zeros(R)
        if dL_dy0 is None:
            dL_dy0 = np.zeros((self.mech.n_species, self.n_cells))
        (pa, ma, k1), (pt, mt, k2), (p0, m0, k3) = _ptr(dy), _ptr(dL_dtheta), _ptr(dL_dy0)
        if not (ma == mt == m0):
            raise ChemError("dL_dy, dL_dtheta and dL_dy0 must all be on the host or all on the device")
        n_bad = _check(load().chem_sensitivity(self._h, pa, pt, p0, ma, _stream_ptr(stream)), "chem_sensitivity")
        return dL_dtheta, dL_dy0, n_bad

    def sensitivity_checkpointed(self, states, dt: float, dL_dy, last_recorded: bool = False, dL_dtheta=None,
                                 dL_dy0=None, stream=None):
        """(dL/dtheta [R], dL/dy0 [S, C], n_bad) through len(states) solve steps of dt by step
        checkpointing: states [n_steps, S, C] holds the state at the start of each step; the
        library re-solves each step from it (the last one too unless last_recorded) and chains
        the adjoint through them, last step first (chem_sensitivity_checkpointed)."""
        R = self.mech.n_reactions
        if dL_dtheta is None:
            dL_dtheta = np.zeros(R)
        if dL_dy0 is None:
            dL_dy0 = np.zeros((self.mech.n_species, self.n_cells))
        n_steps = int(states.shape[0])
        (ps, ms, k0), (pa, ma, k1), (pt, mt, k2), (p0, m0, k3) = _ptr(states), _ptr(dL_dy), _ptr(dL_dtheta), _ptr(dL_dy0)
        if not (ms == ma == mt == m0):
            raise ChemError("states, dL_dy, dL_dtheta and dL_dy0 must all be on the host or all on the device")
        n_bad = _check(load().chem_sensitivity_checkpointed(self._h, ps, n_steps, float(dt), int(bool(last_recorded)),
                                                            pa, pt, p0, ma, _stream_ptr(stream)),
                       "chem_sensitivity_checkpointed")
        return dL_dtheta, dL_dy0, n_bad

    def tangent(self, dy0, dtheta=None, dy=None, stream=None):
        """(dy [S, C], n_bad): the directional derivative of the current state
        along dy0 [S, C] (the state at set_state) and dtheta [R] (None: 0)."""
        if dy is None:
            dy = np.zeros((self.mech.n_species, self.n_cells))
        (p0, m0, k1), (po, mo, k2) = _ptr(dy0), _ptr(dy)
        pt, mt, k3 = _ptr(dtheta) if dtheta is not None else (None, m0, None)
        if not (m0 == mo == mt):
            raise ChemError("dy0, dtheta and dy must all be on the host or all on the device")
        n_bad = _check(load().chem_tangent(self._h, p0, pt, po, m0, _stream_ptr(stream)), "chem_tangent")
        return dy, n_bad

    def get_tape(self, cell: int, rows: bool = True):
        """(kind, q, val, rows) of one cell's recorded tape; rows [n_rows, S] belong,
        in order, to the INIT, REFACTOR and ITER events (None with rows=False)."""
        n, nr = ct.c_int32(0), ct.c_int32(0)
        _check(load().chem_get_tape(self._h, int(cell), None, None, None, None, 0, ct.byref(n), ct.byref(nr)),
               "chem_get_tape")
        kind = np.zeros(n.value, np.int32)
        q = np.zeros(n.value, np.int32)
        val = np.zeros(n.value)
        r = np.zeros((nr.value, self.mech.n_species)) if rows else None
        _check(load().chem_get_tape(self._h, int(cell), ct.c_void_p(kind.ctypes.data), ct.c_void_p(q.ctypes.data),
                                    ct.c_void_p(val.ctypes.data), None if r is None else ct.c_void_p(r.ctypes.data),
                                    n.value, ct.byref(n), ct.byref(nr)), "chem_get_tape")
        return kind, q, val, r

    def close(self):
        if getattr(self, "_h", None):
            load().chem_cells_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def eval_warp_sum(x, stream=None):
    """The solve kernels' warp sum of each row of x (numpy, host, shape (n, 32)), on the GPU."""
    xx = np.ascontiguousarray(x, np.float64)
    assert xx.ndim == 2 and xx.shape[1] == 32
    out = np.empty(xx.shape[0], np.float64)
    _check(load().chem_eval_warp_sum(ct.c_void_p(xx.ctypes.data), ct.c_void_p(out.ctypes.data), xx.shape[0], MEM_HOST,
                                     _stream_ptr(stream)), "chem_eval_warp_sum")
    return out


def eval_reciprocal(x, stream=None):
    """The solve kernels' FP64 reciprocal of every element of x (numpy, host), on the GPU."""
    xx = np.ascontiguousarray(x, np.float64)
    out = np.empty_like(xx)
    _check(load().chem_eval_reciprocal(ct.c_void_p(xx.ctypes.data), ct.c_void_p(out.ctypes.data), xx.size, MEM_HOST,
                                       _stream_ptr(stream)), "chem_eval_reciprocal")
    return out


def measure_fma_peak(precision: int = 64, stream=None):
    """(TFLOP/s, ms) of the FMA-throughput kernel on the current device."""
    tf, ms = ct.c_double(0.0), ct.c_double(0.0)
    _check(load().chem_measure_fma_peak(int(precision), ct.byref(tf), ct.byref(ms), _stream_ptr(stream)),
           "chem_measure_fma_peak")
    return tf.value, ms.value


def staging_fallbacks(cells=None, stream=None):
    """Staging counters (fallbacks, unfinished) of a batch's last solve call, or with
    cells None of chem_solve_step_noalloc's last call on the current device."""
    fb, un = ct.c_int64(0), ct.c_int64(0)
    _check(load().chem_staging_fallbacks(None if cells is None else cells.handle, ct.byref(fb), ct.byref(un),
                                         _stream_ptr(stream)), "chem_staging_fallbacks")
    return fb.value, un.value


CHUNK_FN = ct.CFUNCTYPE(ct.c_int, ct.c_int64, ct.c_int64, ct.c_int32, ct.c_void_p)


def _host_ptr(a, what):
    """Pointer to a host array the library reads and writes in place: a C-contiguous
    float64 numpy array or CPU torch tensor (no copies are made)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous():
                raise ChemError(f"{what} must be a contiguous float64 host tensor")
            return ct.c_void_p(a.data_ptr())
    except ImportError:
        pass
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.flags.writeable):
        raise ChemError(f"{what} must be a writeable C-contiguous float64 numpy array")
    return ct.c_void_p(a.ctypes.data)


def pinned_empty(shape):
    """A page-locked float64 host array (numpy view of a pinned torch tensor), so the
    pipeline's copies run asynchronously."""
    import torch
    return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()


class Pipeline:
    """Host-resident state with the chemistry on the GPU, overlapped chunk by chunk
    (chem_pipeline_*): per chunk its own device batch and stream; the host's work on
    a chunk whose result is back runs while the GPU solves the others."""

    def __init__(self, mech: Mechanism, n_cells: int, n_chunks: int, rtol: float = 1e-4, atol: float = 1e-10,
                 max_order: int = 5, max_steps: int = 5000, lu_precision: int = 64, driver: str = "persistent",
                 cells_per_block: int = 0, blocks_per_sm: int = 0):
        L = load()
        self.mech = mech
        self.n_cells, self.n_chunks = int(n_cells), int(n_chunks)
        o = Opts()
        L.chem_opts_default(ct.byref(o))
        o.rtol, o.atol, o.max_order, o.max_steps = rtol, atol, max_order, max_steps
        o.lu_precision, o.driver = lu_precision, DRIVERS[driver]
        o.cells_per_block, o.blocks_per_sm = cells_per_block, blocks_per_sm
        h = ct.c_void_p()
        _check(L.chem_pipeline_create(mech.handle, self.n_cells, self.n_chunks, ct.byref(o), ct.byref(h)),
               "chem_pipeline_create")
        self._h = h

    def run(self, T, P, y, dt: float, n_steps: int = 1, fn=None, J=None, stats: bool = False):
        """Integrate host y [S, C] in place over n_steps steps of dt; fn(c0, c1, step) runs on
        this thread once cells [c0, c1) of a step are back (it may update those columns of
        y, T, P, J; a true return value stops the run).  Returns the last step's stats
        (stats=True) or None."""
        err = []

        def cb(c0, c1, step, user):
            try:
                return 1 if fn(int(c0), int(c1), int(step)) else 0
            except BaseException as e:          # re-raised after the library has drained its streams
                err.append(e)
                return 1

        cfn = CHUNK_FN(cb) if fn is not None else CHUNK_FN()
        st = np.zeros(self.n_cells, STATS_DTYPE) if stats else None
        rc = load().chem_pipeline_run(self._h, _host_ptr(T, "T"), _host_ptr(P, "P"),
                                      None if J is None else _host_ptr(J, "J"), _host_ptr(y, "y"), float(dt),
                                      int(n_steps), cfn, None, None if st is None else ct.c_void_p(st.ctypes.data))
        if err:
            raise err[0]
        _check(rc, "chem_pipeline_run")
        return st

    def close(self):
        if getattr(self, "_h", None):
            load().chem_pipeline_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(mech: Mechanism, cells: synth.Cells, dt: float, rtol: float, atol: float, n_steps: int = 1,
          **opts):
    """Convenience: host arrays in, (y [S, C], stats) out, through the C ABI."""
    c = Cells(mech, cells.n_cells, rtol=rtol, atol=atol, **opts)
    try:
        c.set_state(cells.T, cells.P, cells.y)
        if cells.J is not None:
            c.set_photolysis(cells.J)
        for _ in range(n_steps):
            c.solve_step(dt)
        y = c.get_state()
        return y, c.get_stats()
    finally:
        c.close()


def _autograd_function():
    import torch

    class ChemSolveFn(torch.autograd.Function):
        """y_final = solve(theta, y0) over n_steps solve_step calls; backward runs the
        discrete adjoint (chem_sensitivity).  theta [R] and y0 [S, C] are float64
        tensors on the batch's device; T, P [C] likewise.

        Step checkpointing: the forward keeps the state at the start of every
        step and the final one (S x C doubles each).  The backward differentiates
        the whole recorded tape when it fits; when it does not (a cell's tape
        overflowed) or when checkpoint=True, it hands the kept states to
        chem_sensitivity_checkpointed, which re-runs the steps one at a time
        from them, last first, each with a fresh tape, and chains the adjoint
        through them: the tape then only has to hold one step.  The batch must
        not be used otherwise between the forward and the backward."""

        @staticmethod
        def forward(ctx, theta, y0, cells, T, P, dt, n_steps, checkpoint):
            n_steps = int(n_steps)
            th = theta.detach().contiguous()
            cells.set_theta(th)
            states = torch.empty((n_steps + 1,) + tuple(y0.shape), dtype=y0.dtype, device=y0.device)
            states[0].copy_(y0.detach())
            if checkpoint:
                # one tape per step: start every step afresh from the kept state
                for k in range(n_steps):
                    cells.set_state(T, P, states[k])
                    cells.solve_step(dt)
                    cells.get_state(out=states[k + 1])
            else:
                cells.set_state(T, P, states[0])
                for k in range(n_steps):
                    cells.solve_step(dt)
                    cells.get_state(out=states[k + 1])
            ctx.cells, ctx.T, ctx.P, ctx.dt, ctx.theta = cells, T, P, dt, th
            ctx.states, ctx.per_step = states, bool(checkpoint)
            ctx.R = theta.numel()
            return states[-1].clone()

        @staticmethod
        def backward(ctx, gy):
            import torch as _t
            c = ctx.cells
            c.set_theta(ctx.theta)          # the backward evaluates rates with the forward's theta
            gth = _t.zeros(ctx.R, dtype=_t.float64, device=gy.device)
            gy0 = _t.zeros_like(gy)
            lam = gy.contiguous()
            if not ctx.per_step:
                _, _, n_bad = c.sensitivity(lam, gth, gy0)
                if n_bad == 0:
                    return gth, gy0, None, None, None, None, None, None
            # the tape is current for the last step in per-step mode
            _, _, n_bad = c.sensitivity_checkpointed(ctx.states[:-1], ctx.dt, lam, last_recorded=ctx.per_step,
                                                     dL_dtheta=gth, dL_dy0=gy0)
            if n_bad:
                raise ChemError(f"{n_bad} (cell, step) pairs have no sensitivity (tape overflow or failed solve)")
            return gth, gy0, None, None, None, None, None, None

    return ChemSolveFn


_FN = None


def solve_with_grad(cells: Cells, theta, y0, T, P, dt: float, n_steps: int = 1, checkpoint: bool = False):
    """Differentiable multi-cell solve (cells must be created with record_adjoint=True).

    checkpoint=True records one step at a time (the tape holds one step; the
    backward re-runs steps from kept states); otherwise the backward falls back
    to that only when the whole tape overflowed."""
    global _FN
    if _FN is None:
        _FN = _autograd_function()
    return _FN.apply(theta, y0, cells, T, P, dt, n_steps, checkpoint)
