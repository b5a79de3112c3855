"""Thin Python binding of libmtssph.so (include/mtssph.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Device memory comes from PyTorch's caching allocator through the library's
allocator hook, and the library's work is ordered on a PyTorch CUDA stream.
The names follow the C calls (mts_body_create -> Body(...),
mts_advance_slow_step -> Body.advance_slow_step, ...).  There is no CPU
fallback: without the built library or without a CUDA device every call
raises.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import re
import sys
import weakref
from typing import Optional

import numpy as np

from . import _build

OK = 0
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_SINGULAR_B, ERR_NONFINITE, ERR_TIMEOUT, \
    ERR_UNSTABLE_DT, ERR_STATE = range(1, 9)
FP64, MIXED = 0, 1
DAMP_AUTO, DAMP_BLOCKS, DAMP_WIDE = 0, 1, 2
WHOLE_AXIS = 62
ELASTIC_SVK, NEOHOOKE_J2 = 0, 1
F_U, F_X, F_V, F_DEFGRAD, F_PB, F_C, F_ALPHA, F_CPINV, F_ACC = range(9)

_lib = None
_live_contexts: "weakref.WeakSet" = weakref.WeakSet()


def _shutdown():
    """Release every body and context while PyTorch (whose allocator frees the
    device memory) is still alive; interpreter teardown order is arbitrary."""
    for ctx in list(_live_contexts):
        try:
            ctx.close()
        except Exception:
            pass


atexit.register(_shutdown)


class MtsError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where} failed (status {status}): {msg}")
        self.status = status


class Allocator(C.Structure):
    ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
    RELEASE = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)
    _fields_ = [("alloc", ALLOC), ("release", RELEASE), ("user", C.c_void_p)]


class BodyDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("precision", C.c_int32), ("n", C.c_int64),
                ("X", C.c_void_p), ("dx", C.c_double), ("h_over_dx", C.c_double),
                ("damp_layout", C.c_int32), ("tile", C.c_int32),
                ("dx_axis", C.c_double * 3)]


class StepParams(C.Structure):
    _fields_ = [("dt_slow", C.c_double), ("ramp_value", C.c_double),
                ("dt_sub_override", C.c_double), ("ke_tol", C.c_double),
                ("ke_ref", C.c_double), ("max_substeps", C.c_int64),
                ("ke_mode", C.c_int32), ("check_every", C.c_int32),
                ("force_dt", C.c_int32), ("reserved", C.c_int32)]


class StepReport(C.Structure):
    _fields_ = [("substeps", C.c_int64), ("converged", C.c_int32), ("status", C.c_int32),
                ("ke_final", C.c_double), ("max_v", C.c_double), ("max_a", C.c_double),
                ("dt_last", C.c_double), ("end_force", C.c_double * 3),
                ("tip_deflection", C.c_double * 3), ("kernel_launches", C.c_int64),
                ("prof_count", C.c_int64), ("prof_ms", C.c_double)]


def header_functions() -> list:
    """Names of every function declared in include/mtssph.h."""
    text = open(_build.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mts_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Load (building first if stale) libmtssph.so and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = C.CDLL(path)
    vp, d, i32, i64 = C.c_void_p, C.c_double, C.c_int32, C.c_int64
    sig = {
        "mts_ctx_create": [C.c_int, vp, C.POINTER(Allocator), C.POINTER(vp)],
        "mts_ctx_destroy": [vp],
        "mts_last_error": [],
        "mts_version": [],
        "mts_body_create": [vp, C.POINTER(BodyDesc), C.POINTER(vp)],
        "mts_body_destroy": [vp],
        "mts_body_permutation": [vp, vp],
        "mts_body_damping_layout": [vp, vp, C.POINTER(i32)],
        "mts_save_state": [vp, vp, C.POINTER(C.c_size_t)],
        "mts_release_bc_concentration": [vp, i64, vp],
        "mts_set_diffusion_mode": [vp, i32],
        "mts_batch_create": [vp, i32, vp, C.POINTER(vp)],
        "mts_adjoint_enable": [vp, i64],
        "mts_adjoint_reset": [vp],
        "mts_adjoint_seed": [vp, vp, vp, vp],
        "mts_adjoint_slow_step": [vp, C.POINTER(StepParams), i64, vp],
        "mts_read_adjoint": [vp, i32, vp, i64],
        "mts_adjoint_equilibrium": [vp, i64, d, vp, C.POINTER(i64)],
        "mts_batch_advance": [vp, vp, vp],
        "mts_batch_destroy": [vp],
        "mts_load_state": [vp, vp, C.c_size_t],
        "mts_body_neighbors": [vp, C.POINTER(i64), vp, vp],
        "mts_body_colouring": [vp, C.POINTER(i64), vp, vp, vp, vp, vp],
        "mts_set_material": [vp, C.c_int, d, d, d, d, d, d, d],
        "mts_set_damping": [vp, d],
        "mts_set_diffusion": [vp, d, d, d],
        "mts_set_bc_displacement": [vp, i64, vp, C.c_uint32, vp, i32],
        "mts_set_bc_concentration": [vp, i64, vp, d],
        "mts_set_tip": [vp, i64, vp],
        "mts_diffusion_dt": [vp, C.POINTER(d), C.POINTER(d)],
        "mts_advance_slow_step": [vp, C.POINTER(StepParams), C.POINTER(StepReport)],
        "mts_substep_partial": [vp, d, d, i32],
        "mts_set_profiling": [vp, i32],
        "mts_read_field": [vp, i32, vp, i64],
        "mts_write_field": [vp, i32, vp, i64],
        "mts_kinetic_energy_noalloc": [vp, i32, i32, i64, d, vp, vp],
        "mts_selftest_conversions": [vp, i64, C.c_uint64, vp],
        "mts_body_set_shapes": [vp, i32, i32],
        "mts_body_shapes": [vp, C.POINTER(i32), C.POINTER(i32)],
        "mts_body_autotune": [vp, i32, d, C.POINTER(i32), C.POINTER(i32), C.POINTER(d)],
        "mts_batch_autotune": [vp, i32, d],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.mts_ctx_destroy.restype = None
    L.mts_body_destroy.restype = None
    L.mts_batch_destroy.restype = None
    L.mts_last_error.restype = C.c_char_p
    _lib = L
    return L


def _check(st: int, where: str):
    if st != OK:
        raise MtsError(st, where, lib().mts_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Context:
    """mts_ctx on one CUDA device with a PyTorch stream and allocator."""

    def __init__(self, device: int = 0, torch_allocator: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("mtssph needs a CUDA device; there is no CPU fallback")
        self.device = device
        self._torch = torch
        self.stream = torch.cuda.Stream(device=device)
        alloc_p = None
        if torch_allocator:
            stream = self.stream

            def _alloc(nbytes, user):
                try:
                    with torch.cuda.device(device):
                        return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream)
                except Exception:
                    return None

            def _release(ptr, nbytes, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._cb = (Allocator.ALLOC(_alloc), Allocator.RELEASE(_release))
            self._alloc = Allocator(self._cb[0], self._cb[1], None)
            alloc_p = C.byref(self._alloc)
        h = C.c_void_p()
        _check(lib().mts_ctx_create(device, C.c_void_p(self.stream.cuda_stream), alloc_p,
                                    C.byref(h)), "mts_ctx_create")
        self._h = h
        self._bodies: "weakref.WeakSet" = weakref.WeakSet()
        _live_contexts.add(self)

    @property
    def handle(self):
        if not getattr(self, "_h", None):
            raise RuntimeError("context is closed")
        return self._h

    def close(self):
        """Destroy the context after every body created on it."""
        if getattr(self, "_h", None):
            for b in list(self._bodies):
                b.close()
            self.stream.synchronize()
            lib().mts_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Body:
    """mts_body: a particle body with its fixed neighbourhood on the GPU."""

    def __init__(self, ctx: Context, X: np.ndarray, dx: float, h_over_dx: float = 1.3,
                 precision: int = FP64, damp_layout: int = DAMP_AUTO, dx_axis=None,
                 tile: int = 0):
        """dx_axis: lattice spacing per axis (anisotropic kernel); None = dx.
        tile: particles per Morton tile of the gather kernels (0 = default)."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        self.n, self.dim = X.shape
        self.ctx = ctx
        self.precision = precision
        da = (C.c_double * 3)(*([0.0] * 3 if dx_axis is None else
                                list(dx_axis) + [0.0] * (3 - len(dx_axis))))
        desc = BodyDesc(self.dim, precision, self.n, X.ctypes.data, dx, h_over_dx, damp_layout,
                        int(tile), da)
        h = C.c_void_p()
        _check(lib().mts_body_create(ctx.handle, C.byref(desc), C.byref(h)), "mts_body_create")
        self._h = h
        self._batches: "weakref.WeakSet" = weakref.WeakSet()
        ctx._bodies.add(self)

    def close(self):
        if getattr(self, "_h", None):
            for bt in list(self._batches):     # a batch borrows its bodies
                bt.close()
            lib().mts_body_destroy(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    # -- setup products
    def permutation(self) -> np.ndarray:
        p = np.zeros(self.n, np.int64)
        _check(lib().mts_body_permutation(self._h, _ptr(p)), "mts_body_permutation")
        return p

    def damping_layout(self):
        """(per-axis block shifts, level cap) of the damping order in use."""
        sh = np.zeros(3, np.int32)
        cap = C.c_int32()
        _check(lib().mts_body_damping_layout(self._h, _ptr(sh), C.byref(cap)),
               "mts_body_damping_layout")
        return tuple(int(x) for x in sh[:self.dim]), int(cap.value)

    def neighbors(self):
        nnz = C.c_int64()
        _check(lib().mts_body_neighbors(self._h, C.byref(nnz), None, None), "mts_body_neighbors")
        off = np.zeros(self.n + 1, np.int64)
        idx = np.zeros(max(nnz.value, 1), np.int32)
        _check(lib().mts_body_neighbors(self._h, C.byref(nnz), _ptr(off), _ptr(idx)),
               "mts_body_neighbors")
        return off, idx[:nnz.value]

    def colouring(self):
        m = C.c_int64()
        _check(lib().mts_body_colouring(self._h, C.byref(m), None, None, None, None, None),
               "mts_body_colouring")
        k = max(m.value, 1)
        pa, pb, col, sub = (np.zeros(k, np.int32) for _ in range(4))
        key = np.zeros(k, np.int64)
        _check(lib().mts_body_colouring(self._h, C.byref(m), _ptr(pa), _ptr(pb), _ptr(col),
                                        _ptr(key), _ptr(sub)), "mts_body_colouring")
        mm = m.value
        return pa[:mm], pb[:mm], col[:mm], key[:mm], sub[:mm]

    # -- configuration
    def set_material(self, model: int, rho0: float, E: float, nu: float, sigma0: float = 0.0,
                     sigma_inf: float = 0.0, delta: float = 0.0, H: float = 0.0):
        _check(lib().mts_set_material(self._h, model, rho0, E, nu, sigma0, sigma_inf, delta, H),
               "mts_set_material")
        self._material = (model, rho0, E, nu, sigma0, sigma_inf, delta, H)

    def set_damping(self, eta: float):
        _check(lib().mts_set_damping(self._h, eta), "mts_set_damping")

    def set_diffusion(self, D: float, beta: float, c0: float):
        _check(lib().mts_set_diffusion(self._h, D, beta, c0), "mts_set_diffusion")
        self._diffusion = (D, beta, c0)

    # -- parameters of the reverse mode
    def parameters(self) -> np.ndarray:
        """theta = (E, sigma0, sigma_inf, delta, H, D, beta) as currently set."""
        m = getattr(self, "_material", None)
        if m is None:
            raise RuntimeError("no material set")
        D, beta, _ = getattr(self, "_diffusion", (0.0, 0.0, 0.0))
        return np.array([m[2], m[4], m[5], m[6], m[7], D, beta])

    def set_parameters(self, theta):
        """Set theta (see parameters()); the concentration field is kept."""
        th = [float(x) for x in theta]
        m = self._material
        self.set_material(m[0], m[1], th[0], m[3], th[1], th[2], th[3], th[4])
        if getattr(self, "_diffusion", None) is not None:
            c = self.read(F_C)
            self.set_diffusion(th[5], th[6], self._diffusion[2])
            self.write(F_C, c)

    # -- reverse mode (FP64 arithmetic; a mixed-precision body is reversed on its FP64 twin)
    def adjoint_enable(self, max_substeps: int):
        _check(lib().mts_adjoint_enable(self._h, int(max_substeps)), "mts_adjoint_enable")
        self._adj_cap = int(max_substeps)

    def adjoint_reset(self):
        _check(lib().mts_adjoint_reset(self._h), "mts_adjoint_reset")

    def adjoint_seed(self, u_bar=None, tip_bar=None, force_bar=None):
        ub = None if u_bar is None else np.ascontiguousarray(u_bar, np.float64).reshape(self.n * self.dim)
        tb = None if tip_bar is None else np.ascontiguousarray(
            list(tip_bar) + [0.0] * (3 - len(tip_bar)), np.float64)
        fb = None if force_bar is None else np.ascontiguousarray(
            list(force_bar) + [0.0] * (3 - len(force_bar)), np.float64)
        _check(lib().mts_adjoint_seed(self._h, None if ub is None else _ptr(ub),
                                      None if tb is None else _ptr(tb),
                                      None if fb is None else _ptr(fb)), "mts_adjoint_seed")

    def adjoint_slow_step(self, substeps: int, dt_slow: float = 0.0, ramp: float = 0.0,
                          ke_ref: float = 1.0, ke_mode: int = 0, dt_sub: float = 0.0,
                          force_dt: bool = False, **_ignored) -> np.ndarray:
        """Reverse one slow step (the body must hold the state at its start);
        returns d objective / d theta contributed by the step."""
        p = StepParams(dt_slow, ramp, dt_sub, -1.0, ke_ref, int(substeps), ke_mode, 0,
                       int(force_dt), 0)
        th = np.zeros(7)
        _check(lib().mts_adjoint_slow_step(self._h, C.byref(p), int(substeps), _ptr(th)),
               "mts_adjoint_slow_step")
        return th

    def adjoint_equilibrium(self, max_iters: int = 100000, tol: float = 1e-10):
        """Equilibrium adjoint of the held (converged) state; returns
        (d objective / d theta, transposed substeps run)."""
        th = np.zeros(7)
        it = C.c_int64()
        _check(lib().mts_adjoint_equilibrium(self._h, int(max_iters), float(tol), _ptr(th),
                                             C.byref(it)), "mts_adjoint_equilibrium")
        return th, int(it.value)

    def read_adjoint(self, field: int) -> np.ndarray:
        w = self._width(field)
        out = np.zeros(self.n * w)
        _check(lib().mts_read_adjoint(self._h, field, _ptr(out), out.size), "mts_read_adjoint")
        return out.reshape(self.n, w) if w > 1 else out

    def set_bc_displacement(self, ids, axis_mask: int, u_unit=None, report_force: bool = False):
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        uu = None if u_unit is None else np.ascontiguousarray(u_unit, dtype=np.float64)
        _check(lib().mts_set_bc_displacement(self._h, ids.size, _ptr(ids), axis_mask,
                                             None if uu is None else _ptr(uu), int(report_force)),
               "mts_set_bc_displacement")

    def set_bc_concentration(self, ids, value: float):
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        _check(lib().mts_set_bc_concentration(self._h, ids.size, _ptr(ids), value),
               "mts_set_bc_concentration")

    def set_diffusion_mode(self, mode: int):
        """0: one-pass pairwise Laplacian; 1: two-stage flux in the deformed
        configuration (Sec. 3.2)."""
        _check(lib().mts_set_diffusion_mode(self._h, int(mode)), "mts_set_diffusion_mode")

    def release_bc_concentration(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        _check(lib().mts_release_bc_concentration(self._h, ids.size, _ptr(ids)),
               "mts_release_bc_concentration")

    def set_tip(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        _check(lib().mts_set_tip(self._h, ids.size, _ptr(ids)), "mts_set_tip")

    def diffusion_dt(self):
        a, b = C.c_double(), C.c_double()
        _check(lib().mts_diffusion_dt(self._h, C.byref(a), C.byref(b)), "mts_diffusion_dt")
        return a.value, b.value

    # -- stepping
    def advance_slow_step(self, dt_slow: float = 0.0, ramp: float = 0.0, ke_tol: float = -1.0,
                          ke_ref: float = 1.0, ke_mode: int = 0, max_substeps: int = 1,
                          dt_sub: float = 0.0, check_every: int = 0,
                          force_dt: bool = False) -> StepReport:
        p = StepParams(dt_slow, ramp, dt_sub, ke_tol, ke_ref, max_substeps, ke_mode,
                       check_every, int(force_dt), 0)
        r = StepReport()
        _check(lib().mts_advance_slow_step(self._h, C.byref(p), C.byref(r)),
               "mts_advance_slow_step")
        return r

    def set_profiling(self, stage: int):
        _check(lib().mts_set_profiling(self._h, stage), "mts_set_profiling")

    def substep_partial(self, dt: float, upto: int, ramp: float = 0.0):
        _check(lib().mts_substep_partial(self._h, dt, ramp, upto), "mts_substep_partial")

    # -- fields
    def _width(self, field: int) -> int:
        return {F_U: self.dim, F_X: self.dim, F_V: self.dim, F_ACC: self.dim, F_DEFGRAD: 9,
                F_PB: self.dim * self.dim, F_C: 1, F_ALPHA: 1, F_CPINV: 6}[field]

    def read(self, field: int, out: Optional[np.ndarray] = None) -> np.ndarray:
        """Field in the original particle order (float64); `out`, when given, is
        a C-contiguous float64 array of n * width values that receives it (for
        example pinned host memory)."""
        w = self._width(field)
        if out is None:
            out = np.zeros(self.n * w)
        elif (out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"] or out.size != self.n * w):
            raise ValueError("read: out must be a C-contiguous float64 array of n * width values")
        _check(lib().mts_read_field(self._h, field, _ptr(out), out.size), "mts_read_field")
        return out.reshape(self.n, w) if w > 1 else out.reshape(self.n)

    def write(self, field: int, values):
        w = self._width(field)
        a = np.ascontiguousarray(values, dtype=np.float64).reshape(self.n * w)
        _check(lib().mts_write_field(self._h, field, _ptr(a), a.size), "mts_write_field")

    def set_shapes(self, tile: int = 0, damp_warps: int = 0):
        """Launch shapes: particles per tile of the gather kernels (0 keeps the
        tiles) and damping warps per CTA (0 = as many as fit)."""
        _check(lib().mts_body_set_shapes(self._h, int(tile), int(damp_warps)),
               "mts_body_set_shapes")

    def shapes(self):
        t, w = C.c_int32(), C.c_int32()
        _check(lib().mts_body_shapes(self._h, C.byref(t), C.byref(w)), "mts_body_shapes")
        return {"tile": t.value, "damp_warps": w.value}

    def autotune(self, substeps: int = 8, ramp: float = 0.0):
        """Time every candidate launch shape on `substeps` substeps from the
        current state, apply the fastest and restore the state."""
        t, w, ms = C.c_int32(), C.c_int32(), C.c_double()
        _check(lib().mts_body_autotune(self._h, int(substeps), float(ramp), C.byref(t),
                                       C.byref(w), C.byref(ms)), "mts_body_autotune")
        return {"tile": t.value, "damp_warps": w.value, "ms": ms.value}

    def save_state(self) -> bytes:
        """Snapshot of the evolving state (bit-exact resume with load_state)."""
        nb = C.c_size_t()
        _check(lib().mts_save_state(self._h, None, C.byref(nb)), "mts_save_state")
        buf = C.create_string_buffer(nb.value)
        _check(lib().mts_save_state(self._h, buf, C.byref(nb)), "mts_save_state")
        return buf.raw[:nb.value]

    def load_state(self, state: bytes):
        buf = C.create_string_buffer(bytes(state), len(state))
        _check(lib().mts_load_state(self._h, buf, len(state)), "mts_load_state")


class Batch:
    """mts_batch: bodies of one context advanced by one graph launch per slow step."""

    def __init__(self, ctx: Context, bodies):
        self.ctx = ctx
        self.bodies = list(bodies)
        arr = (C.c_void_p * len(self.bodies))(*[b._h.value if b._h else None for b in self.bodies])
        h = C.c_void_p()
        _check(lib().mts_batch_create(ctx.handle, len(self.bodies), arr, C.byref(h)),
               "mts_batch_create")
        self._h = h
        for b in self.bodies:
            b._batches.add(self)

    def close(self):
        if getattr(self, "_h", None):
            lib().mts_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, substeps: int = 8, ramp: float = 0.0):
        """mts_batch_autotune: tune every body's launch shapes in turn."""
        _check(lib().mts_batch_autotune(self._h, int(substeps), float(ramp)), "mts_batch_autotune")
        return [b.shapes() for b in self.bodies]

    def advance(self, params) -> list:
        """One slow step of every body; params: one dict of advance_slow_step
        keyword arguments per body (check_every is ignored)."""
        if len(params) != len(self.bodies):
            raise ValueError("one parameter set per body")
        P = (StepParams * len(params))()
        for i, kw in enumerate(params):
            P[i] = StepParams(kw.get("dt_slow", 0.0), kw.get("ramp", 0.0), kw.get("dt_sub", 0.0),
                              kw.get("ke_tol", -1.0), kw.get("ke_ref", 1.0),
                              kw.get("max_substeps", 1), kw.get("ke_mode", 0), 0,
                              int(kw.get("force_dt", False)), 0)
        R = (StepReport * len(params))()
        _check(lib().mts_batch_advance(self._h, P, R), "mts_batch_advance")
        return list(R)


def slow_steps(body: Body, theta, steps):
    """Run the slow steps `steps` (one dict of advance_slow_step arguments
    each) with parameters theta = (E, sigma0, sigma_inf, delta, H, D, beta)
    and return the tip deflection and end force of the last one as a torch
    tensor [tip (dim), force (dim)], differentiable with respect to theta
    through the library's reverse mode (FP64 adjoint arithmetic for FP64 and
    mixed-precision bodies; substep sizes and counts held at the forward
    run's values)."""
    import torch

    class _SlowSteps(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            body.set_parameters(th.detach().cpu().numpy())
            ckpts, counts = [], []
            r = None
            for p in steps:
                ckpts.append(body.save_state())
                r = body.advance_slow_step(**p)
                counts.append(int(r.substeps))
            ctx.ckpts, ctx.counts, ctx.final = ckpts, counts, body.save_state()
            d = body.dim
            return torch.tensor(list(r.tip_deflection[:d]) + list(r.end_force[:d]),
                                dtype=torch.float64)

        @staticmethod
        def backward(ctx, gout):
            d = body.dim
            g = gout.detach().cpu().numpy()
            need = max(ctx.counts)
            if getattr(body, "_adj_cap", 0) < need:
                body.adjoint_enable(need)
            else:
                body.adjoint_reset()
            body.adjoint_seed(tip_bar=g[:d], force_bar=g[d:])
            th = np.zeros(7)
            for p, ck, k in zip(reversed(steps), reversed(ctx.ckpts), reversed(ctx.counts)):
                body.load_state(ck)
                th += body.adjoint_slow_step(k, **p)
            body.load_state(ctx.final)
            return torch.from_numpy(th).to(gout.dtype)

    return _SlowSteps.apply(theta)


def body_from_case(ctx: Context, case, precision: int = FP64, damp_layout: int = DAMP_AUTO,
                   tile: int = 0) -> Body:
    """Body with the material, damping, diffusion and BCs of a synth Case."""
    b = Body(ctx, case.X, case.dx, case.h_over_dx, precision, damp_layout,
             getattr(case, "dx_axis", None), tile)
    m = case.material
    b.set_material(ELASTIC_SVK if m.model == "svk" else NEOHOOKE_J2, m.rho0, m.E, m.nu,
                   m.sigma0, m.sigma_inf, m.delta, m.H)
    b.set_damping(case.eta)
    for bc in case.disp_bcs:
        b.set_bc_displacement(bc.ids, bc.axis_mask, bc.u_unit, bc.report_force)
    if case.diffusion is not None:
        b.set_diffusion(*case.diffusion)
    for cb in case.conc_bcs:
        b.set_bc_concentration(cb.ids, cb.value)
    if case.tip_ids is not None and len(case.tip_ids):
        b.set_tip(case.tip_ids)
    return b


def selftest_conversions(ctx: Context, n: int, seed: int = 1) -> tuple:
    """mts_selftest_conversions: (FP32 -> FP64, FP64 -> FP32) mismatches of the
    library's integer-pipe conversions against the hardware on n bit patterns."""
    out = np.zeros(2, np.int64)
    _check(lib().mts_selftest_conversions(ctx.handle, int(n), int(seed), _ptr(out)),
           "mts_selftest_conversions")
    return int(out[0]), int(out[1])


def kinetic_energy_noalloc(v_dev_ptr: int, precision: int, dim: int, n: int, mass: float,
                           out_dev_ptr: int, stream: int = 0) -> None:
    """mts_kinetic_energy_noalloc on caller-owned device buffers (no allocation):
    out[0] = sum 1/2 mass |v|^2, out[1] = max |v|, ordered on `stream`."""
    _check(lib().mts_kinetic_energy_noalloc(C.c_void_p(v_dev_ptr), precision, dim, n, mass,
                                            C.c_void_p(out_dev_ptr), C.c_void_p(stream)),
           "mts_kinetic_energy_noalloc")
