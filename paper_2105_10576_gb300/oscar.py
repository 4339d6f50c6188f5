"""Thin ctypes binding of the OSCAR C ABI (include/oscar.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library liboscar_gb300.so built in-tree by build.py. If the library is
missing or cannot be loaded, every call raises; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "liboscar_gb300.so")

OSCAR_FP64, OSCAR_MIXED = 0, 1
CONV_PRES_RESID, CONV_DU_MAX, CONV_AREA = 0, 1, 2
FIELD_ALPHA, FIELD_P, FIELD_U, FIELD_U_VD, FIELD_U_CR = 0, 1, 2, 5, 8
FIELD_P_VD, FIELD_P_CR, FIELD_KAPPA, FIELD_PHI_VD, FIELD_PHI_CR, FIELD_NF = 11, 12, 13, 14, 17, 20

ERRORS = {0: "ok", -1: "invalid argument", -2: "out of device memory", -3: "pressure solve not converged",
          -4: "non-finite value", -5: "timeout", -6: "CUDA error"}


class OscarError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {ERRORS.get(code, 'error')} ({code})")
        self.code = code


class oscar_params(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
        ("rho1", C.c_double), ("rho2", C.c_double), ("mu1", C.c_double), ("mu2", C.c_double),
        ("sigma", C.c_double), ("theta_deg", C.c_double),
        ("U_inlet", C.c_double), ("alpha_inlet", C.c_double),
        ("n_piso", C.c_int), ("n_smooth", C.c_int), ("c_alpha", C.c_double),
        ("conv_mode", C.c_int), ("conv_tol", C.c_double),
        ("cg_rtol", C.c_double), ("cg_maxit", C.c_int), ("precision", C.c_int),
    ]


class oscar_schedule(C.Structure):
    _fields_ = [("mg_nu", C.c_int), ("mg_nu_mid", C.c_int), ("mg_nu_cta", C.c_int), ("cta_cells", C.c_int),
                ("coarse_refresh", C.c_int), ("block_x", C.c_int), ("cta_global", C.c_int)]


class oscar_stats_t(C.Structure):
    _fields_ = [
        ("k_f", C.c_int), ("N", C.c_int), ("E_last", C.c_double), ("dU_last", C.c_double),
        ("cg_iters_total", C.c_longlong), ("cg_iters_last", C.c_int), ("mg_levels", C.c_int),
        ("phase_volume", C.c_double), ("n_fluid", C.c_longlong), ("cell_updates", C.c_longlong),
        ("device_bytes", C.c_size_t), ("kernel_launches", C.c_longlong),
        ("mg_first_cta_level", C.c_int), ("mg_cta_global_level", C.c_int),
    ]


EXPORTS = ["oscar_timesteps", "oscar_create", "oscar_drag_step", "oscar_relax", "oscar_standard_step",
           "oscar_drag_step_async", "oscar_relax_async", "oscar_standard_step_async", "oscar_wait",
           "oscar_footprint", "oscar_query",
           "oscar_fields", "oscar_fields_device", "oscar_set_field", "oscar_stats", "oscar_destroy",
           "oscar_strerror", "oscar_profile", "oscar_profile_read", "oscar_profile_repeat", "oscar_get_schedule",
           "oscar_set_schedule", "oscar_phase_volume_noalloc"]

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if absent: the CUDA path is the only path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"OSCAR CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    dp = C.POINTER(C.c_double)
    H = C.c_void_p
    lib.oscar_timesteps.argtypes = [C.POINTER(oscar_params), C.POINTER(C.c_uint8), C.c_double, dp]
    lib.oscar_create.argtypes = [C.POINTER(oscar_params), C.POINTER(C.c_uint8), dp, C.c_void_p, C.POINTER(H)]
    lib.oscar_drag_step.argtypes = [H, C.c_double]
    lib.oscar_relax.argtypes = [H, C.c_double, C.c_int, C.POINTER(C.c_int), dp]
    lib.oscar_standard_step.argtypes = [H, C.c_double]
    lib.oscar_drag_step_async.argtypes = [H, C.c_double]
    lib.oscar_relax_async.argtypes = [H, C.c_double, C.c_int]
    lib.oscar_standard_step_async.argtypes = [H, C.c_double]
    lib.oscar_wait.argtypes = [H, C.POINTER(C.c_int), dp]
    lib.oscar_footprint.argtypes = [C.POINTER(oscar_params), C.POINTER(C.c_size_t)]
    lib.oscar_query.argtypes = [H]
    lib.oscar_fields.argtypes = [H, C.c_int, dp, C.c_size_t]
    lib.oscar_fields_device.argtypes = [H, C.c_int, C.c_void_p, C.c_size_t]
    lib.oscar_set_field.argtypes = [H, C.c_int, dp, C.c_size_t]
    lib.oscar_stats.argtypes = [H, C.POINTER(oscar_stats_t)]
    lib.oscar_get_schedule.argtypes = [H, C.POINTER(oscar_schedule)]
    lib.oscar_set_schedule.argtypes = [H, C.POINTER(oscar_schedule)]
    lib.oscar_destroy.argtypes = [H]
    lib.oscar_strerror.argtypes = [C.c_int]
    lib.oscar_strerror.restype = C.c_char_p
    lib.oscar_profile.argtypes = [H, C.c_int]
    lib.oscar_profile_repeat.argtypes = [H, C.c_int]
    lib.oscar_profile_read.argtypes = [H, C.c_int, C.POINTER(C.c_int), C.c_char_p, C.c_size_t,
                                       C.POINTER(C.c_uint), dp, C.POINTER(C.c_longlong)]
    lib.oscar_phase_volume_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_longlong, C.c_double, C.c_void_p,
                                               C.c_void_p]
    _lib = lib
    return lib


def make_params(p: dict) -> oscar_params:
    P = oscar_params()
    for name, typ in oscar_params._fields_:
        v = p[name]
        setattr(P, name, int(v) if typ is C.c_int else float(v))
    return P


def _check(rc: int, where: str, allow_not_converged: bool = False):
    if rc == 0 or (allow_not_converged and rc == -3):
        return rc
    raise OscarError(rc, where)


def oscar_footprint(params: dict) -> int:
    """Device bytes an instance with these parameters would hold (no allocation)."""
    lib = load()
    out = C.c_size_t(0)
    _check(lib.oscar_footprint(C.byref(make_params(params)), C.byref(out)), "oscar_footprint")
    return int(out.value)


def oscar_timesteps(params: dict, c_cfl: float, solid=None):
    """(dt_CFL, dt_B, dt_vd, N); with a solid mask the CFL velocity is the mean
    speed through the narrowest x cross-section."""
    lib = load()
    out = (C.c_double * 4)()
    P = make_params(params)
    sp = None
    if solid is not None:
        s = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        if s.size != params["nx"] * params["ny"] * (params["nz"] if params["dim"] == 3 else 1):
            raise ValueError("solid mask does not match the grid")
        sp = s.ctypes.data_as(C.POINTER(C.c_uint8))
    _check(lib.oscar_timesteps(C.byref(P), sp, c_cfl, out), "oscar_timesteps")
    return out[0], out[1], out[2], int(out[3])


def _grid_shape(p):
    return (p["nz"], p["ny"], p["nx"]) if p["dim"] == 3 else (p["ny"], p["nx"])


def _face_shapes(p):
    nx, ny = p["nx"], p["ny"]
    if p["dim"] == 2:
        return [(ny, nx + 1), (ny + 1, nx), (ny, nx)]
    nz = p["nz"]
    return [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]


class Oscar:
    """One simulation instance held on the GPU (wraps an oscar_handle)."""

    def __init__(self, params: dict, solid: np.ndarray, alpha0: np.ndarray, stream: int = 0):
        self.lib = load()
        self.p = dict(params)
        self.shape = _grid_shape(self.p)
        self.fshapes = _face_shapes(self.p)
        self._P = make_params(self.p)
        s = np.ascontiguousarray(solid, dtype=np.uint8).reshape(self.shape)
        a = np.ascontiguousarray(alpha0, dtype=np.float64).reshape(self.shape)
        h = C.c_void_p()
        _check(self.lib.oscar_create(C.byref(self._P), s.ctypes.data_as(C.POINTER(C.c_uint8)),
                                     a.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(stream), C.byref(h)),
               "oscar_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.oscar_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def drag_step(self, dt: float, strict: bool = True) -> int:
        return _check(self.lib.oscar_drag_step(self.h, dt), "oscar_drag_step", not strict)

    def relax(self, dt_cr: float, N: int, strict: bool = True):
        kf = C.c_int(0)
        test = C.c_double(0.0)
        rc = _check(self.lib.oscar_relax(self.h, dt_cr, N, C.byref(kf), C.byref(test)), "oscar_relax", not strict)
        return rc, kf.value, test.value

    # asynchronous steps: launch now, collect with wait() (one pending step per handle)
    def drag_step_async(self, dt: float) -> int:
        return _check(self.lib.oscar_drag_step_async(self.h, dt), "oscar_drag_step_async")

    def relax_async(self, dt_cr: float, N: int) -> int:
        return _check(self.lib.oscar_relax_async(self.h, dt_cr, N), "oscar_relax_async")

    def standard_step_async(self, dt: float) -> int:
        return _check(self.lib.oscar_standard_step_async(self.h, dt), "oscar_standard_step_async")

    def query(self) -> bool:
        """True when the launched step has finished (wait() then returns at once)."""
        rc = self.lib.oscar_query(self.h)
        if rc < 0:
            raise OscarError(rc, "oscar_query")
        return rc == 1

    def wait(self, strict: bool = True):
        kf = C.c_int(0)
        test = C.c_double(0.0)
        rc = _check(self.lib.oscar_wait(self.h, C.byref(kf), C.byref(test)), "oscar_wait", not strict)
        return rc, kf.value, test.value

    def standard_step(self, dt: float, strict: bool = True) -> int:
        return _check(self.lib.oscar_standard_step(self.h, dt), "oscar_standard_step", not strict)

    def _len_shape(self, which):
        if which >= FIELD_PHI_VD:
            sh = self.fshapes[(which - FIELD_PHI_VD) % 3]
        else:
            sh = self.shape
        return int(np.prod(sh)), sh

    def field(self, which: int, out: np.ndarray = None) -> np.ndarray:
        """The field as float64 in host memory; `out` (optional, contiguous
        float64 of the field's size, e.g. a view of pinned memory) receives it."""
        n, sh = self._len_shape(which)
        if out is None:
            out = np.zeros(sh)
        elif out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"] or out.size != n:
            raise ValueError("out must be a contiguous float64 array of the field's size")
        _check(self.lib.oscar_fields(self.h, which, out.ctypes.data_as(C.POINTER(C.c_double)), n), "oscar_fields")
        return out.reshape(sh)

    def field_device(self, which: int, dev_ptr: int, n: int):
        _check(self.lib.oscar_fields_device(self.h, which, C.c_void_p(dev_ptr), n), "oscar_fields_device")

    def set_field(self, which: int, arr: np.ndarray):
        n, sh = self._len_shape(which)
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(sh)
        _check(self.lib.oscar_set_field(self.h, which, a.ctypes.data_as(C.POINTER(C.c_double)), n), "oscar_set_field")

    def profile(self, enable: bool):
        """Start (clearing the last recording) or stop in-step kernel timing:
        while on, steps run eagerly with CUDA events around every launch."""
        _check(self.lib.oscar_profile(self.h, 1 if enable else 0), "oscar_profile")

    def profile_repeat(self, enable: bool):
        """Issue every plain finest-level half sweep twice (idempotent) in the
        following graph steps, for in-graph timing by difference."""
        _check(self.lib.oscar_profile_repeat(self.h, 1 if enable else 0), "oscar_profile_repeat")

    def profile_read(self) -> list:
        """[(kernel name, grid blocks, total ms, launches)] of the recording."""
        cnt = C.c_int(0)
        self.lib.oscar_profile_read(self.h, 0, C.byref(cnt), None, 0, None, None, None)
        out = []
        buf = C.create_string_buffer(512)
        for i in range(cnt.value):
            g = C.c_uint(0)
            ms = C.c_double(0.0)
            n = C.c_longlong(0)
            _check(self.lib.oscar_profile_read(self.h, i, None, buf, 512, C.byref(g), C.byref(ms), C.byref(n)),
                   "oscar_profile_read")
            out.append((buf.value.decode(errors="replace"), g.value, ms.value, n.value))
        return out

    def schedule(self) -> dict:
        """The multigrid schedule and launch shape of the pressure solves."""
        sc = oscar_schedule()
        _check(self.lib.oscar_get_schedule(self.h, C.byref(sc)), "oscar_get_schedule")
        return {name: getattr(sc, name) for name, _ in oscar_schedule._fields_}

    def set_schedule(self, sched: dict):
        """Replace (some of) the schedule; the step graphs are rebuilt."""
        cur = self.schedule()
        cur.update(sched)
        sc = oscar_schedule(**cur)
        _check(self.lib.oscar_set_schedule(self.h, C.byref(sc)), "oscar_set_schedule")

    def stats(self) -> dict:
        st = oscar_stats_t()
        _check(self.lib.oscar_stats(self.h, C.byref(st)), "oscar_stats")
        return {name: getattr(st, name) for name, _ in oscar_stats_t._fields_}


def oscar_phase_volume_noalloc(alpha_dev: int, solid_dev: int, ncell: int, cell_volume: float, result_dev: int,
                               stream: int = 0) -> int:
    """Phase volume of caller-owned device arrays with no device allocation
    (for callers that cannot call cudaMalloc, e.g. during stream capture)."""
    lib = load()
    return _check(lib.oscar_phase_volume_noalloc(C.c_void_p(alpha_dev), C.c_void_p(solid_dev), ncell, cell_volume,
                                                 C.c_void_p(result_dev), C.c_void_p(stream)),
                  "oscar_phase_volume_noalloc")
