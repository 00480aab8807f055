"""Thin ctypes binding of libpm_gb300 (include/pm.h). Argument marshalling only.

Every numerical step runs in the library's CUDA kernels. PyTorch supplies device memory and the
current CUDA stream; this module passes raw pointers. If the shared library has not been built
the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

from . import build as _build

# ---- C structures -----------------------------------------------------------------------------

PM_OK, PM_EINVAL, PM_ENOMEM, PM_ECUDA, PM_NOT_CONVERGED, PM_BREAKDOWN, PM_TIMEOUT, PM_DISCONNECTED, PM_EBUSY, \
    PM_EBOUNDS = range(10)
PM_BUILD_CHECKED = 1
PM_WALL_WEST, PM_WALL_EAST, PM_WALL_SOUTH, PM_WALL_NORTH = 1, 2, 4, 8
OP_VEL_U1, OP_VEL_U2, OP_VEL_U3, OP_PRESSURE, OP_MASS = 0, 1, 2, 3, 4
OP_VEL1_U1, OP_VEL1_U2, OP_VEL1_U3, OP_GRAD_X, OP_GRAD_Y, OP_GRAD_Z = 5, 6, 7, 8, 9, 10
PREC_JACOBI, PREC_IC0, PREC_NONE, PREC_LINE = 0, 1, 2, 3
PREC_DEFAULT = -1
FP64, FP32_REFINE, BF16_REFINE = 0, 1, 2
STEP_LUMPED, STEP_CONSISTENT = 0, 1
KERNEL_AUTO, KERNEL_STREAM, KERNEL_RESIDENT = 0, 1, 2
(FIELD_U1, FIELD_U2, FIELD_U3, FIELD_U1_PREV, FIELD_U2_PREV, FIELD_U3_PREV, FIELD_P, FIELD_Q,
 FIELD_UT1, FIELD_UT2, FIELD_UT3, FIELD_BP) = range(12)
DIAG_KINETIC_ENERGY, DIAG_DIV_U, DIAG_DIV_UT, DIAG_P_MEAN, DIAG_COUNT = range(5)
DIAG_NAMES = ("kinetic_energy", "div_u", "div_u_tilde", "p_mean")

# Slot offsets (di, dj, dk) of the 15-slot layout, in slot order (documented in pm.h's layout).
SLOT_OFFSETS = [(0, 0, -1), (0, 0, 0), (0, 0, 1), (1, 0, 0), (1, 0, 1), (-1, 0, -1), (-1, 0, 0),
                (0, 1, 0), (0, 1, 1), (0, -1, -1), (0, -1, 0), (1, 1, 0), (1, 1, 1), (-1, -1, -1),
                (-1, -1, 0)]
NBR_OFFSETS = [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1)]


class MeshDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("slip_walls", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("ocean_mask", ctypes.c_void_p), ("depth", ctypes.c_void_p)]


class Physics(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double * 3), ("dt", ctypes.c_double), ("coriolis", ctypes.c_void_p)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("x0_is_guess", ctypes.c_int32),
                ("max_restarts", ctypes.c_int32), ("inner_rtol", ctypes.c_double),
                ("kernel", ctypes.c_int32), ("pad", ctypes.c_int32)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer_iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("first_pass_iters", ctypes.c_int32), ("rel_residual_true", ctypes.c_double),
                ("rel_residual_rec", ctypes.c_double), ("seconds", ctypes.c_double),
                ("bytes_moved", ctypes.c_double), ("rel_residual_floor", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class OperatorInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_pad", ctypes.c_int64), ("ncols", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64)]


# Every exported symbol of include/pm.h with its ctypes signature.
_P = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "pm_assemble_operator": (_I, [ctypes.POINTER(MeshDesc), ctypes.POINTER(Physics), ctypes.POINTER(_P), _P]),
    "pm_operator_bytes": (ctypes.c_int64, [ctypes.POINTER(MeshDesc)]),
    "pm_operator_info_get": (_I, [_P, ctypes.POINTER(OperatorInfo)]),
    "pm_operator_columns": (_I, [_P, _P, _P]),
    "pm_operator_export": (_I, [_P, _I, _P, _P, _P]),
    "pm_spmv": (_I, [_P, _I, _P, _P, _P]),
    "pm_residual": (_I, [_P, _I, _P, _P, _P, _P, _P]),
    "pm_pcg_solve": (_I, [_P, _I, _P, _P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), _P]),
    "pm_pcg_solve_noalloc": (_I, [_P, _I, _P, _P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats), _P]),
    "pm_state_create": (_I, [_P, ctypes.POINTER(_P)]),
    "pm_state_get": (_I, [_P, _P, _P, _P, _P, _P]),
    "pm_state_set": (_I, [_P, _P, _P, _P, _P, ctypes.c_int32, _P]),
    "pm_state_step_index": (ctypes.c_int32, [_P]),
    "pm_state_field": (_I, [_P, ctypes.c_int32, _P, _P]),
    "pm_state_set_field": (_I, [_P, ctypes.c_int32, _P, _P]),
    "pm_state_set_step_index": (_I, [_P, ctypes.c_int32]),
    "pm_state_save": (_I, [_P, ctypes.c_char_p, _P]),
    "pm_state_load": (_I, [_P, ctypes.c_char_p, _P]),
    "pm_state_diagnostics": (_I, [_P, _P, _P, _P]),
    "pm_project_step": (_I, [_P, _P, _P, _P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveOpts),
                             ctypes.c_int32, _P, _P]),
    "pm_operator_destroy": (None, [_P]),
    "pm_state_destroy": (None, [_P]),
    "pm_status_string": (ctypes.c_char_p, [_I]),
    "pm_last_error": (_I, [ctypes.c_char_p, ctypes.c_int32]),
    "pm_kernel_launch_count": (ctypes.c_int64, []),
    "pm_batch_create": (_I, [_P, _P, _P, ctypes.c_int32, ctypes.POINTER(SolveOpts), ctypes.c_int32,
                             ctypes.POINTER(_P), _P]),
    "pm_batch_solve": (_I, [_P, _P, _P, _P, _P]),
    "pm_batch_info": (_I, [_P, _P, _P, _P, _P]),
    "pm_batch_destroy": (None, [_P]),
    "pm_pcg_solve_batched": (_I, [_P, _P, _P, _P, ctypes.c_int32, ctypes.POINTER(SolveOpts), _P, _P]),
    "pm_debug_barrier_timeout": (_I, [_P]),
    "pm_server_create": (_I, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(SolveOpts), ctypes.c_int32,
                              ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_P), _P]),
    "pm_server_workspace_bytes": (ctypes.c_size_t, [_P, ctypes.c_int32]),
    "pm_server_admit": (_I, [_P, _P, _I, ctypes.c_int32, _P, _P, _P, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int32),
                             _P]),
    "pm_server_run": (_I, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), _P]),
    "pm_server_poll": (_I, [_P, _P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "pm_server_info": (_I, [_P, _P, _P, _P, _P, _P]),
    "pm_server_destroy": (None, [_P]),
    "pm_kernel_timing": (_I, [ctypes.c_int32]),
    "pm_kernel_timing_get": (_I, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]),
    "pm_set_log": (_I, [ctypes.c_char_p, ctypes.c_double]),
    "pm_build_flags": (ctypes.c_int32, []),
}

KT_SPMV, KT_UPDATE, KT_PUPDATE, KT_IC0, KT_LINE = 0, 1, 2, 3, 4


def kernel_timing(enable: bool):
    _check(load().pm_kernel_timing(1 if enable else 0), "kernel_timing")


def kernel_timing_get(kind: int):
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    _check(load().pm_kernel_timing_get(kind, ctypes.byref(ms), ctypes.byref(cnt)), "kernel_timing_get")
    return ms.value, cnt.value

_lib = None
_lib_path = _build.LIB


def library_path() -> str:
    return _build.LIB


def select_library(path: Optional[str] = None) -> str:
    """Make every wrapper of this module call the library at `path` (None: the default build),
    e.g. the checked build (build(checked=True)); returns the path selected before, to restore it.
    Handles created through one library must not be passed to another."""
    global _lib, _lib_path
    prev = _lib_path
    lib = load(path or _build.LIB)
    _lib, _lib_path = lib, path or _build.LIB
    return prev


def set_log(path: Optional[str] = None, hbm_peak_gbs: float = 0.0):
    """pm_set_log: append one JSON line per solved system to `path` (None closes the log)."""
    _check(load().pm_set_log(os.fsencode(path) if path is not None else None, float(hbm_peak_gbs)), "set_log")


def build_flags() -> int:
    return int(load().pm_build_flags())


def load(path: Optional[str] = None):
    """Load the shared library (no build, no GPU needed) and bind every signature."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        raise RuntimeError(f"libpm_gb300.so is not built ({p}); run __graft_entry__.build() "
                           "or python -m paper_1207_0486_gb300.build")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class PMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(status: int, what: str, allow=()):
    if status != PM_OK and status not in allow:
        buf = ctypes.create_string_buffer(512)
        load().pm_last_error(buf, 512)
        raise PMError(status, f"{what}: {load().pm_status_string(status).decode()}: {buf.value.decode()}")
    return status


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, n=None, name="tensor"):
    """Device pointer of a contiguous CUDA float64 tensor (checked)."""
    if t is None:
        return None
    torch = _torch()
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA float64 tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} has {t.numel()} elements, expected {n}")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Options:
    rtol: float = 1e-8
    max_iter: int = 100000
    prec: int = PREC_JACOBI
    precision: int = FP64
    x0_is_guess: bool = False
    max_restarts: int = 3
    inner_rtol: float = 1e-4
    kernel: int = 0            # KERNEL_AUTO, KERNEL_STREAM, KERNEL_RESIDENT

    def c(self) -> SolveOpts:
        return SolveOpts(self.rtol, self.max_iter, self.prec, self.precision, int(self.x0_is_guess),
                         self.max_restarts, self.inner_rtol, self.kernel, 0)


class Operator:
    """Device-resident operators of one basin (pm_operator)."""

    def __init__(self, handle, basin=None):
        self.handle = handle
        self.basin = basin
        info = OperatorInfo()
        _check(load().pm_operator_info_get(handle, ctypes.byref(info)), "info")
        self.n, self.n_pad, self.ncols, self.nz = info.n, info.n_pad, info.ncols, info.nz
        self.nx, self.ny = info.nx, info.ny

    @property
    def device_bytes(self) -> int:
        info = OperatorInfo()
        _check(load().pm_operator_info_get(self.handle, ctypes.byref(info)), "info")
        return info.device_bytes

    def columns(self):
        ci = np.empty(self.ncols, dtype=np.int32)
        cj = np.empty(self.ncols, dtype=np.int32)
        _check(load().pm_operator_columns(self.handle, ci.ctypes.data, cj.ctypes.data), "columns")
        return ci, cj

    def export(self, which: int):
        vals = np.empty(15 * self.n, dtype=np.float64)
        nbr = np.empty(7 * self.ncols, dtype=np.int32)
        st = np.empty(self.n, dtype=np.uint16)
        _check(load().pm_operator_export(self.handle, which, vals.ctypes.data, nbr.ctypes.data,
                                         st.ctypes.data), "export")
        return vals.reshape(15, self.n), nbr.reshape(self.ncols, 7), st

    def column_field(self, grid: np.ndarray) -> np.ndarray:
        """(ny, nx) grid field -> per-column array in library column order."""
        ci, cj = self.columns()
        return np.ascontiguousarray(grid[cj, ci], dtype=np.float64)

    def spmv(self, which: int, x, y, stream=None):
        _check(load().pm_spmv(self.handle, which, _dptr(x, self.n, "x"), _dptr(y, self.n, "y"),
                              _stream(stream)), "spmv")

    def residual(self, which: int, b, x, r, stream=None, norms: bool = True):
        """pm_residual: r = b - A x in compensated arithmetic. Returns (||r||^2, || |A||x| + |b| ||^2,
        ||b||^2) when norms is true (synchronising), else None."""
        nb = (ctypes.c_double * 3)() if norms else None
        _check(load().pm_residual(self.handle, which, _dptr(b, self.n, "b"), _dptr(x, self.n, "x"),
                                  _dptr(r, self.n, "r"), nb, _stream(stream)), "residual")
        return (nb[0], nb[1], nb[2]) if norms else None

    def solve(self, which: int, b, x, opts: Options = Options(), stream=None, allow_not_converged=False):
        st = SolveStats()
        o = opts.c()
        r = load().pm_pcg_solve(self.handle, which, _dptr(b, self.n, "b"), _dptr(x, self.n, "x"),
                                ctypes.byref(o), ctypes.byref(st), _stream(stream))
        _check(r, "pcg_solve", allow=(PM_NOT_CONVERGED,) if allow_not_converged else ())
        return st

    def solve_noalloc(self, which: int, b, x, opts: Options = Options(), stream=None, allow_not_converged=False):
        """pm_pcg_solve_noalloc: Jacobi / plain PCG whose scratch is the library's static array."""
        st = SolveStats()
        o = opts.c()
        r = load().pm_pcg_solve_noalloc(self.handle, which, _dptr(b, self.n, "b"), _dptr(x, self.n, "x"),
                                        ctypes.byref(o), ctypes.byref(st), _stream(stream))
        _check(r, "pcg_solve_noalloc", allow=(PM_NOT_CONVERGED,) if allow_not_converged else ())
        return st

    def close(self):
        if self.handle:
            load().pm_operator_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mesh_desc(basin):
    """Build the C mesh descriptor; the returned tuple keeps the host arrays alive."""
    mask = np.ascontiguousarray(basin.mask, dtype=np.uint8)
    depth = np.ascontiguousarray(basin.depth, dtype=np.float64)
    d = MeshDesc(basin.nx, basin.ny, basin.nz, basin.slip_walls, basin.dx, basin.dy,
                 mask.ctypes.data, depth.ctypes.data)
    return d, (mask, depth)


def operator_bytes(basin) -> int:
    d, keep = mesh_desc(basin)
    return int(load().pm_operator_bytes(ctypes.byref(d)))


def assemble_operator(basin, stream=None) -> Operator:
    """pm_assemble_operator on a workloads.Basin."""
    d, keep = mesh_desc(basin)
    cor = None if basin.coriolis is None else np.ascontiguousarray(basin.coriolis, dtype=np.float64)
    ph = Physics((ctypes.c_double * 3)(*basin.nu), basin.dt, None if cor is None else cor.ctypes.data)
    h = ctypes.c_void_p()
    _check(load().pm_assemble_operator(ctypes.byref(d), ctypes.byref(ph), ctypes.byref(h), _stream(stream)),
           "assemble_operator")
    return Operator(h, basin)


def pcg_solve(op: Operator, which: int, b, x, opts: Options = Options(), stream=None, **kw):
    return op.solve(which, b, x, opts, stream, **kw)


class State:
    """Time-step state u^k, u^{k-1}, p^k of one basin (pm_state)."""

    def __init__(self, op: Operator):
        self.op = op
        h = ctypes.c_void_p()
        _check(load().pm_state_create(op.handle, ctypes.byref(h)), "state_create")
        self.handle = h

    @property
    def step_index(self) -> int:
        return int(load().pm_state_step_index(self.handle))

    def get(self, stream=None):
        torch = _torch()
        n = self.op.n
        out = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(4)]
        _check(load().pm_state_get(self.handle, *[_dptr(t) for t in out], _stream(stream)), "state_get")
        return out

    def field(self, which: int, out=None, stream=None):
        """pm_state_field: one state field (FIELD_*) as a CUDA float64 tensor."""
        torch = _torch()
        out = torch.empty(self.op.n, dtype=torch.float64, device="cuda") if out is None else out
        _check(load().pm_state_field(self.handle, which, _dptr(out, self.op.n, "out"), _stream(stream)), "state_field")
        return out

    def set_field(self, which: int, src, stream=None):
        """pm_state_set_field: u^k, u^{k-1}, p or q (FIELD_U1 .. FIELD_Q) from a CUDA float64 tensor."""
        _check(load().pm_state_set_field(self.handle, which, _dptr(src, self.op.n, "src"), _stream(stream)),
               "state_set_field")

    def set_step_index(self, k: int):
        _check(load().pm_state_set_step_index(self.handle, k), "state_set_step_index")

    def snapshot(self, stream=None):
        """Device copies of the fields that define the time loop (u^k, u^{k-1}, p, q) and the step
        index; restore() puts them back (the in-memory counterpart of save / load)."""
        return [self.field(f, stream=stream) for f in range(FIELD_Q + 1)], self.step_index

    def restore(self, snap, stream=None):
        fields, k = snap
        for f, t in enumerate(fields):
            self.set_field(f, t, stream)
        self.set_step_index(k)

    def save(self, path: str, stream=None):
        """pm_state_save: checkpoint file (header + little-endian float64 fields)."""
        _check(load().pm_state_save(self.handle, os.fsencode(path), _stream(stream)), "state_save")

    def load_checkpoint(self, path: str, stream=None):
        """pm_state_load: resume from a checkpoint written by save() for the same basin."""
        _check(load().pm_state_load(self.handle, os.fsencode(path), _stream(stream)), "state_load")

    def diagnostics(self, stream=None) -> dict:
        """pm_state_diagnostics: kinetic energy, discrete divergences of u^k and of the last
        prediction, mean pressure."""
        out = (ctypes.c_double * DIAG_COUNT)()
        _check(load().pm_state_diagnostics(self.op.handle, self.handle, out, _stream(stream)), "state_diagnostics")
        return {name: out[i] for i, name in enumerate(DIAG_NAMES)}

    def set(self, u1=None, u2=None, u3=None, p=None, step_index=0, stream=None):
        _check(load().pm_state_set(self.handle, _dptr(u1), _dptr(u2), _dptr(u3), _dptr(p),
                                   step_index, _stream(stream)), "state_set")

    def close(self):
        if self.handle:
            load().pm_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def project_step(op: Operator, state: State, theta1=None, theta2=None, vel: Options = None,
                 pres: Options = None, correction: int = STEP_LUMPED, stream=None,
                 allow_not_converged=False):
    """pm_project_step. theta1/theta2: CUDA float64 tensors of length ncols (or None)."""
    vel = vel or Options(prec=PREC_IC0)
    pres = pres or Options(prec=PREC_JACOBI)
    stats = (SolveStats * 7)()
    vo, po = vel.c(), pres.c()
    r = load().pm_project_step(op.handle, state.handle, _dptr(theta1, op.ncols, "theta1"),
                               _dptr(theta2, op.ncols, "theta2"), ctypes.byref(vo), ctypes.byref(po),
                               correction, stats, _stream(stream))
    _check(r, "project_step", allow=(PM_NOT_CONVERGED,) if allow_not_converged else ())
    return [stats[i] for i in range(7)]


def kernel_launch_count() -> int:
    return int(load().pm_kernel_launch_count())


class Batch:
    """A batch of independent systems solved by one persistent, graph-captured kernel (pm_batch)."""

    def __init__(self, ops: Sequence[Operator], which: Sequence[int], opts: Options = None,
                 autotune: bool = False, stream=None, prec: Sequence[int] = None):
        """prec: None (opts.prec for every entry) or one preconditioner per entry (PREC_DEFAULT
        takes opts.prec)."""
        opts = opts or Options(prec=PREC_LINE)
        self.ops = list(ops)
        self.which = list(which)
        n = len(self.ops)
        hops = (ctypes.c_void_p * n)(*[o.handle.value if isinstance(o.handle, ctypes.c_void_p) else o.handle
                                       for o in self.ops])
        hw = (ctypes.c_int * n)(*self.which)
        if prec is not None and len(prec) != n:
            raise ValueError("prec needs one entry per system")
        hp = (ctypes.c_int32 * n)(*prec) if prec is not None else None
        o = opts.c()
        h = ctypes.c_void_p()
        _check(load().pm_batch_create(hops, hw, hp, n, ctypes.byref(o), 1 if autotune else 0, ctypes.byref(h),
                                      _stream(stream)), "batch_create")
        self.handle = h
        self._keep = (hops, hw, hp)

    def info(self):
        tc, blk, grid = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        nt = ctypes.c_int64()
        _check(load().pm_batch_info(self.handle, ctypes.byref(tc), ctypes.byref(blk), ctypes.byref(grid),
                                    ctypes.byref(nt)), "batch_info")
        return {"tile_cols": tc.value, "block": blk.value, "grid": grid.value, "tiles": nt.value}

    def solve(self, bs, xs, stream=None, allow_not_converged=False):
        n = len(self.ops)
        pb = (ctypes.c_void_p * n)(*[_dptr(b, o.n, "b").value for b, o in zip(bs, self.ops)])
        px = (ctypes.c_void_p * n)(*[_dptr(x, o.n, "x").value for x, o in zip(xs, self.ops)])
        stats = (SolveStats * n)()
        r = load().pm_batch_solve(self.handle, pb, px, stats, _stream(stream))
        _check(r, "batch_solve", allow=(PM_NOT_CONVERGED,) if allow_not_converged else ())
        return [stats[i] for i in range(n)]

    def close(self):
        if getattr(self, "handle", None):
            load().pm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _handle(h):
    return h.value if isinstance(h, ctypes.c_void_p) else h


class Server:
    """Continuous batching solve server (pm_server): a slot table advanced by the persistent kernel,
    systems admitted and retired between launches."""

    def __init__(self, slots: int = 64, nz_cap: int = 64, opts: Options = None, tile_cols: int = 64,
                 block: int = 128, blocks_per_sm: int = 0, stream=None):
        opts = opts or Options(prec=PREC_LINE, precision=FP32_REFINE, rtol=1e-8, inner_rtol=1e-2)
        self.opts = opts
        self.slots = slots
        o = opts.c()
        h = ctypes.c_void_p()
        _check(load().pm_server_create(slots, nz_cap, ctypes.byref(o), tile_cols, block, blocks_per_sm,
                                       ctypes.byref(h), _stream(stream)), "server_create")
        self.handle = h
        self._out_slots = (ctypes.c_int32 * slots)()
        self._out_stats = (SolveStats * slots)()

    def workspace_bytes(self, op: Operator) -> int:
        return int(load().pm_server_workspace_bytes(_handle(op.handle), self.opts.precision))

    def admit(self, op: Operator, which: int, b, x, work, stream=None, prec: int = None):
        """Admit one system (prec: its preconditioner, None for the server's); returns its slot, or
        None when every slot is taken (PM_EBUSY)."""
        torch = _torch()
        if not (work.is_cuda and work.dtype == torch.uint8 and work.is_contiguous()):
            raise ValueError("work must be a contiguous CUDA uint8 tensor")
        slot = ctypes.c_int32(-1)
        r = load().pm_server_admit(self.handle, _handle(op.handle), which, PREC_DEFAULT if prec is None else prec,
                                   _dptr(b, op.n, "b"), _dptr(x, op.n, "x"),
                                   ctypes.c_void_p(work.data_ptr()), work.numel(), ctypes.byref(slot),
                                   _stream(stream))
        if r == PM_EBUSY:
            return None
        _check(r, "server_admit")
        return slot.value

    def run(self, quantum: int = 16, stream=None) -> int:
        act = ctypes.c_int32(0)
        _check(load().pm_server_run(self.handle, quantum, ctypes.byref(act), _stream(stream)), "server_run")
        return act.value

    def poll(self):
        """Finished systems since the last poll: list of (slot, SolveStats)."""
        n = ctypes.c_int32(0)
        _check(load().pm_server_poll(self.handle, self._out_slots, self._out_stats, self.slots, ctypes.byref(n)),
               "server_poll")
        out = []
        for i in range(n.value):
            out.append((self._out_slots[i], SolveStats.from_buffer_copy(self._out_stats[i])))
        return out

    def info(self):
        tc, blk, grid = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        cap, la = ctypes.c_int64(), ctypes.c_int64()
        _check(load().pm_server_info(self.handle, ctypes.byref(tc), ctypes.byref(blk), ctypes.byref(grid),
                                     ctypes.byref(cap), ctypes.byref(la)), "server_info")
        return {"tile_cols": tc.value, "block": blk.value, "grid": grid.value, "tile_capacity": cap.value,
                "launches": la.value}

    def close(self):
        if getattr(self, "handle", None):
            load().pm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_barrier_timeout(stream=None) -> int:
    """Status of a deliberately expired bounded grid wait (PM_TIMEOUT expected)."""
    return int(load().pm_debug_barrier_timeout(_stream(stream)))
