"""FP64 CPU oracle for the multi-time-step SPH solid relaxation (arXiv 2309.04010).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only users.  The CUDA library never
imports, links or calls anything here, and this package imports nothing from
the CUDA library's package.  The arithmetic lives in ``mts_oracle.c`` (plain
serial C, FP64, no FMA contraction); this module only compiles it and
marshals arguments through ctypes.

Every function of the C file cites the paper's section, equation or algorithm
it follows.  Pins against closed forms and invariants are in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mts_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libmts_oracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_ARG = 1
ERR_OOM = 2
ERR_SINGULAR = 4
ERR_NONFINITE = 5
ERR_UNSTABLE_DT = 7
ERR_STATE = 8

SVK = 0
J2 = 1

F_U, F_X, F_V, F_DEFGRAD, F_PB, F_C, F_ALPHA, F_CPINV, F_ACC = range(9)
WHOLE_AXIS = 62


class StepParams(C.Structure):
    _fields_ = [("dt_slow", C.c_double), ("ramp_value", C.c_double),
                ("dt_sub_override", C.c_double), ("ke_tol", C.c_double),
                ("ke_ref", C.c_double), ("max_substeps", C.c_int64),
                ("ke_mode", C.c_int32), ("check_every", C.c_int32),
                ("force_dt", C.c_int32), ("reserved", C.c_int32)]


class Report(C.Structure):
    _fields_ = [("substeps", C.c_int64), ("converged", C.c_int32), ("status", C.c_int32),
                ("ke_final", C.c_double), ("max_v", C.c_double), ("max_a", C.c_double),
                ("dt_last", C.c_double), ("end_force", C.c_double * 3),
                ("tip_deflection", C.c_double * 3)]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, -ffp-contract=off, no fast-math)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
               "-D_GNU_SOURCE", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        d, i64, i32, vp = C.c_double, C.c_int64, C.c_int32, C.c_void_p
        L.ob_kernel_w.restype = d
        L.ob_kernel_w.argtypes = [C.c_int, d, d]
        L.ob_kernel_dwdr.restype = d
        L.ob_kernel_dwdr.argtypes = [C.c_int, d, d]
        L.ob_create.argtypes = [C.c_int, i64, vp, d, d, C.c_int, C.POINTER(vp)]
        L.ob_create_layout.argtypes = [C.c_int, i64, vp, d, d, C.c_int, vp, C.c_int32,
                                       C.POINTER(vp)]
        L.ob_create_aniso.argtypes = [C.c_int, i64, vp, vp, d, C.c_int, vp, C.c_int32,
                                      C.POINTER(vp)]
        L.ob_destroy.argtypes = [vp]
        L.ob_destroy.restype = None
        for name in ("ob_nnz", "ob_npairs", "ob_n"):
            getattr(L, name).restype = i64
            getattr(L, name).argtypes = [vp]
        L.ob_blk_shift.argtypes = [vp]
        L.ob_dim.argtypes = [vp]
        L.ob_h.restype = d
        L.ob_h.argtypes = [vp]
        L.ob_neighbors.argtypes = [vp, vp, vp]
        L.ob_perm.argtypes = [vp, vp]
        L.ob_colouring.argtypes = [vp, vp, vp, vp, vp, vp]
        L.ob_set_material.argtypes = [vp, C.c_int, d, d, d, d, d, d, d]
        L.ob_set_damping.argtypes = [vp, d]
        L.ob_set_diffusion.argtypes = [vp, d, d, d]
        L.ob_set_bc_displacement.argtypes = [vp, i64, vp, C.c_uint, vp, C.c_int]
        L.ob_set_bc_concentration.argtypes = [vp, i64, vp, d]
        L.ob_set_tip.argtypes = [vp, i64, vp]
        L.ob_release_bc_concentration.argtypes = [vp, i64, vp]
        L.ob_set_diffusion_mode.argtypes = [vp, C.c_int]
        L.ob_stress_point.argtypes = [C.c_int, d, d, d, d, d, d, d, vp, vp, vp, vp, vp]
        L.ob_substep.argtypes = [vp, d, d, vp, vp, vp]
        L.ob_substep_partial.argtypes = [vp, d, d, C.c_int, vp]
        L.ob_diffusion_dt.argtypes = [vp, vp, vp]
        L.ob_diffusion_step.argtypes = [vp, d]
        L.ob_advance_slow_step.argtypes = [vp, C.POINTER(StepParams), C.POINTER(Report)]
        L.ob_read_field.argtypes = [vp, C.c_int, vp]
        L.ob_write_field.argtypes = [vp, C.c_int, vp]
        L.ob_b0.argtypes = [vp, vp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"oracle {where} failed with status {status}")
        self.status = status


def _check(st: int, where: str):
    if st != OK:
        raise OracleError(st, where)


def kernel_w(dim: int, h: float, r: float) -> float:
    return lib().ob_kernel_w(dim, h, r)


def kernel_dwdr(dim: int, h: float, r: float) -> float:
    return lib().ob_kernel_dwdr(dim, h, r)


def stress_point(model: int, rho0: float, E: float, nu: float, F: np.ndarray,
                 cpinv: Optional[np.ndarray] = None, alpha: float = 0.0, sigma0: float = 0.0,
                 sigma_inf: float = 0.0, delta: float = 0.0, H: float = 0.0):
    """Material point: returns (P, cpinv_new, alpha_new, plastic, newton_residual)."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(9)
    cp = (np.array([1, 1, 1, 0, 0, 0], dtype=np.float64) if cpinv is None
          else np.ascontiguousarray(cpinv, dtype=np.float64).copy())
    al = np.array([alpha], dtype=np.float64)
    P = np.zeros(9)
    res = np.zeros(1)
    plastic = lib().ob_stress_point(model, rho0, E, nu, sigma0, sigma_inf, delta, H,
                                    _ptr(F), _ptr(cp), _ptr(al), _ptr(P), _ptr(res))
    if plastic < 0:
        raise OracleError(ERR_ARG, "stress_point")
    return P.reshape(3, 3), cp, float(al[0]), bool(plastic), float(res[0])


class OracleBody:
    """A particle body advanced by the FP64 oracle (same calls as the library)."""

    def __init__(self, X: np.ndarray, dx: float, h_over_dx: float = 1.3, brute: bool = False,
                 damp_layout=None, dx_axis=None):
        """damp_layout = (shifts per axis, level cap) of the damping order; shifts
        are log2 of the block width in cells, WHOLE_AXIS for an unblocked axis,
        -1 for the smallest admissible width.  Default: smallest blocks, cap 32.
        dx_axis: lattice spacing per axis (the anisotropic kernel); None = dx on
        every axis."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        self.n, self.dim = X.shape
        h = C.c_void_p()
        if damp_layout is None:
            damp_layout = ((-1, -1, -1), 32)
        shifts = np.ascontiguousarray(list(damp_layout[0]) + [-1] * (3 - len(damp_layout[0])),
                                      dtype=np.int32)
        if dx_axis is None:
            _check(lib().ob_create_layout(self.dim, self.n, _ptr(X), dx, h_over_dx, int(brute),
                                          _ptr(shifts), int(damp_layout[1]), C.byref(h)), "create")
        else:
            dk = np.ascontiguousarray(list(dx_axis) + [dx_axis[0]] * (3 - len(dx_axis)),
                                      dtype=np.float64)
            _check(lib().ob_create_aniso(self.dim, self.n, _ptr(X), _ptr(dk), h_over_dx,
                                         int(brute), _ptr(shifts), int(damp_layout[1]),
                                         C.byref(h)), "create")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ob_destroy(self._h)
            self._h = None

    @property
    def h(self) -> float:
        return lib().ob_h(self._h)

    def neighbors(self):
        nnz = lib().ob_nnz(self._h)
        off = np.zeros(self.n + 1, dtype=np.int64)
        idx = np.zeros(max(nnz, 1), dtype=np.int32)
        _check(lib().ob_neighbors(self._h, _ptr(off), _ptr(idx)), "neighbors")
        return off, idx[:nnz]

    def perm(self):
        p = np.zeros(self.n, dtype=np.int64)
        _check(lib().ob_perm(self._h, _ptr(p)), "perm")
        return p

    def colouring(self):
        m = lib().ob_npairs(self._h)
        pa = np.zeros(max(m, 1), np.int32)
        pb = np.zeros(max(m, 1), np.int32)
        col = np.zeros(max(m, 1), np.int32)
        key = np.zeros(max(m, 1), np.int64)
        sub = np.zeros(max(m, 1), np.int32)
        _check(lib().ob_colouring(self._h, _ptr(pa), _ptr(pb), _ptr(col), _ptr(key), _ptr(sub)),
               "colouring")
        return pa[:m], pb[:m], col[:m], key[:m], sub[:m]

    @property
    def blk_shift(self) -> int:
        return lib().ob_blk_shift(self._h)

    def set_material(self, model: int, rho0: float, E: float, nu: float, sigma0: float = 0.0,
                     sigma_inf: float = 0.0, delta: float = 0.0, H: float = 0.0):
        _check(lib().ob_set_material(self._h, model, rho0, E, nu, sigma0, sigma_inf, delta, H),
               "set_material")

    def set_damping(self, eta: float):
        _check(lib().ob_set_damping(self._h, eta), "set_damping")

    def set_diffusion(self, D: float, beta: float, c0: float):
        _check(lib().ob_set_diffusion(self._h, D, beta, c0), "set_diffusion")

    def set_bc_displacement(self, ids, axis_mask: int, u_unit=None, report_force: bool = False):
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        uu = (np.zeros((ids.size, self.dim)) if u_unit is None
              else np.ascontiguousarray(u_unit, dtype=np.float64).reshape(ids.size, self.dim))
        _check(lib().ob_set_bc_displacement(self._h, ids.size, _ptr(ids), axis_mask, _ptr(uu),
                                            int(report_force)), "set_bc_displacement")

    def set_bc_concentration(self, ids, value: float):
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        _check(lib().ob_set_bc_concentration(self._h, ids.size, _ptr(ids), value),
               "set_bc_concentration")

    def set_diffusion_mode(self, mode: int):
        """0: one-pass pairwise Laplacian; 1: two-stage flux in the deformed
        configuration (Sec. 3.2)."""
        _check(lib().ob_set_diffusion_mode(self._h, int(mode)), "set_diffusion_mode")

    def release_bc_concentration(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        _check(lib().ob_release_bc_concentration(self._h, ids.size, _ptr(ids)),
               "release_bc_concentration")

    def set_tip(self, ids):
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        _check(lib().ob_set_tip(self._h, ids.size, _ptr(ids)), "set_tip")

    def diffusion_dt(self):
        a, b = C.c_double(), C.c_double()
        _check(lib().ob_diffusion_dt(self._h, C.byref(a), C.byref(b)), "diffusion_dt")
        return a.value, b.value

    def diffusion_step(self, dt: float):
        _check(lib().ob_diffusion_step(self._h, dt), "diffusion_step")

    def substep(self, dt: float, ramp: float = 0.0):
        ke, vm, am = C.c_double(), C.c_double(), C.c_double()
        _check(lib().ob_substep(self._h, dt, ramp, C.byref(ke), C.byref(vm), C.byref(am)),
               "substep")
        return ke.value, vm.value, am.value

    def substep_partial(self, dt: float, upto: int, ramp: float = 0.0):
        out = np.zeros(3)
        _check(lib().ob_substep_partial(self._h, dt, ramp, upto, _ptr(out)), "substep_partial")
        return out

    def advance(self, dt_slow: float = 0.0, ramp: float = 0.0, ke_tol: float = -1.0,
                ke_ref: float = 1.0, ke_mode: int = 0, max_substeps: int = 1,
                dt_sub: float = 0.0, force_dt: bool = False) -> Report:
        p = StepParams(dt_slow, ramp, dt_sub, ke_tol, ke_ref, max_substeps, ke_mode, 1,
                       int(force_dt), 0)
        r = Report()
        _check(lib().ob_advance_slow_step(self._h, C.byref(p), C.byref(r)), "advance")
        return r

    _WIDTH = {F_U: "d", F_X: "d", F_V: "d", F_ACC: "d", F_DEFGRAD: 9, F_PB: "dd", F_C: 1,
              F_ALPHA: 1, F_CPINV: 6}

    def _width(self, field: int) -> int:
        w = self._WIDTH[field]
        return {"d": self.dim, "dd": self.dim * self.dim}.get(w, w)

    def read(self, field: int) -> np.ndarray:
        w = self._width(field)
        out = np.zeros(self.n * w)
        _check(lib().ob_read_field(self._h, field, _ptr(out)), "read_field")
        return out.reshape(self.n, w) if w > 1 else out

    def write(self, field: int, values: np.ndarray):
        w = self._width(field)
        a = np.ascontiguousarray(values, dtype=np.float64).reshape(self.n * w)
        _check(lib().ob_write_field(self._h, field, _ptr(a)), "write_field")

    def b0(self) -> np.ndarray:
        out = np.zeros(self.n * self.dim * self.dim)
        _check(lib().ob_b0(self._h, _ptr(out)), "b0")
        return out.reshape(self.n, self.dim, self.dim)


def body_from_case(case, brute: bool = False, damp_layout=None) -> OracleBody:
    """Oracle body with the material, damping, diffusion and BCs of a synth Case."""
    b = OracleBody(case.X, case.dx, case.h_over_dx, brute=brute, damp_layout=damp_layout,
                   dx_axis=getattr(case, "dx_axis", None))
    m = case.material
    b.set_material(SVK if m.model == "svk" else J2, m.rho0, m.E, m.nu, m.sigma0, m.sigma_inf,
                   m.delta, m.H)
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
