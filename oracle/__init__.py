"""OSCAR oracle (FP64, CPU, single-threaded): Python side.

TEST INFRASTRUCTURE ONLY. The oracle is the plain reference the CUDA path is
checked against. Only the test suite, the smoke check and the bench's
CPU-baseline leg may import it; the product path never does. It shares no
code with the CUDA path: it is built from oracle/oscar_oracle.c alone with
gcc, and it imports nothing from the CUDA package.

Every function follows Maes & Menke, arXiv 2105.10576 (see the C source for
section and equation references).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oscar_oracle.c")
_LIB = os.path.join(_HERE, "liboscar_oracle.so")
_lock = threading.Lock()
_lib = None

# field numbering of or_field
ALPHA, P, UX, UY, UZ, UVDX, UVDY, UVDZ, UCRX, UCRY, UCRZ, P_VD, P_CR, KAPPA = range(14)
PHI_VD, PHI_CR, NF = 14, 17, 20


class OrParams(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
        ("rho1", C.c_double), ("rho2", C.c_double), ("mu1", C.c_double), ("mu2", C.c_double),
        ("sigma", C.c_double), ("theta_deg", C.c_double),
        ("U_inlet", C.c_double), ("alpha_inlet", C.c_double),
        ("n_piso", C.c_int), ("n_smooth", C.c_int),
        ("c_alpha", C.c_double),
        ("conv_mode", C.c_int),
        ("conv_tol", C.c_double),
        ("cg_rtol", C.c_double),
        ("cg_maxit", C.c_int),
        ("precision", C.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB)
    dp = C.POINTER(C.c_double)
    u8p = C.POINTER(C.c_uint8)
    pp = C.POINTER(OrParams)
    lib.or_create.restype = C.c_void_p
    lib.or_create.argtypes = [pp, u8p, dp]
    lib.or_destroy.argtypes = [C.c_void_p]
    lib.or_drag_step.argtypes = [C.c_void_p, C.c_double]
    lib.or_relax.argtypes = [C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_int), dp]
    lib.or_standard_step.argtypes = [C.c_void_p, C.c_double]
    lib.or_field.argtypes = [C.c_void_p, C.c_int, dp]
    lib.or_set_field.argtypes = [C.c_void_p, C.c_int, dp]
    lib.or_stats.argtypes = [C.c_void_p, dp]
    lib.or_timesteps.restype = C.c_int
    lib.or_timesteps.argtypes = [pp, u8p, C.c_double, dp]
    lib.or_stage_transport.argtypes = [pp, u8p, dp, dp, dp, dp, dp, dp, dp, C.c_double, dp]
    lib.or_stage_interface.argtypes = [pp, u8p, dp, dp, dp, dp, dp, dp]
    lib.or_stage_poisson_apply.argtypes = [pp, u8p, dp, dp, dp, dp, dp]
    lib.or_stage_poisson_cg.restype = C.c_int
    lib.or_stage_poisson_cg.argtypes = [pp, u8p, dp, dp, dp, dp, dp, C.c_double, C.c_int]
    lib.or_stage_poisson_dense.restype = C.c_int
    lib.or_stage_poisson_dense.argtypes = [pp, u8p, dp, dp, dp, dp, dp]
    lib.or_stage_normalised_residual.restype = C.c_double
    lib.or_stage_normalised_residual.argtypes = [pp, u8p, dp, dp, dp, dp, dp]
    lib.or_stage_piso.argtypes = [pp, u8p] + [dp] * 17 + [C.c_double, C.c_double, dp]
    lib.or_stage_interface_area.restype = C.c_double
    lib.or_stage_interface_area.argtypes = [pp, u8p, dp]
    lib.or_stage_relax_energy.restype = C.c_double
    lib.or_stage_relax_energy.argtypes = [pp, u8p, dp, dp, dp, dp]
    _lib = lib
    return lib


def make_params(p: dict) -> OrParams:
    P = OrParams()
    for name, typ in OrParams._fields_:
        v = p[name]
        setattr(P, name, int(v) if typ is C.c_int else float(v))
    return P


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u8(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def grid_shape(p: dict):
    return (p["nz"], p["ny"], p["nx"]) if p["dim"] == 3 else (p["ny"], p["nx"])


def face_shapes(p: dict):
    """Shapes of the x, y, z face arrays (the z array is a 1-element dummy in 2D)."""
    nx, ny = p["nx"], p["ny"]
    nz = p["nz"] if p["dim"] == 3 else 1
    sh = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]
    if p["dim"] == 2:
        sh = [(ny, nx + 1), (ny + 1, nx), (ny, nx)]
    return sh


def timesteps(p: dict, c_cfl: float, solid=None):
    """(dt_cfl, dt_B, dt_vd, N) from the CFL and Brackbill limits (Section 2.2).

    With a solid mask, the CFL velocity is the mean x velocity through the
    narrowest cross-section, U A_inlet / A_min (mass conservation); without
    one it is U_inlet."""
    lib = _load()
    out = np.zeros(4)
    P = make_params(p)
    sp = None
    if solid is not None:
        s = np.ascontiguousarray(solid, dtype=np.uint8)
        assert s.size == p["nx"] * p["ny"] * (p["nz"] if p["dim"] == 3 else 1)
        sp = _u8(s)
    rc = lib.or_timesteps(C.byref(P), sp, c_cfl, _dp(out))
    if rc != 0:
        raise ValueError("no fluid path from the inlet to the outlet")
    return out[0], out[1], out[2], int(out[3])


class OracleState:
    """One OSCAR (or standard-stepping) instance held by the oracle."""

    def __init__(self, params: dict, solid: np.ndarray, alpha0: np.ndarray):
        self.lib = _load()
        self.p = dict(params)
        self._P = make_params(self.p)
        self.shape = grid_shape(self.p)
        self.fshapes = face_shapes(self.p)
        self._solid = np.ascontiguousarray(solid, dtype=np.uint8).reshape(self.shape)
        a0 = np.ascontiguousarray(alpha0, dtype=np.float64).reshape(self.shape)
        self.h = self.lib.or_create(C.byref(self._P), _u8(self._solid), _dp(a0))

    def close(self):
        if self.h:
            self.lib.or_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def drag_step(self, dt: float) -> int:
        return self.lib.or_drag_step(self.h, dt)

    def relax(self, dt_cr: float, N: int):
        kf = C.c_int(0)
        hist = np.zeros(max(N, 1))
        rc = self.lib.or_relax(self.h, dt_cr, N, C.byref(kf), _dp(hist))
        return rc, kf.value, hist[: kf.value].copy()

    def standard_step(self, dt: float) -> int:
        return self.lib.or_standard_step(self.h, dt)

    def field(self, which: int) -> np.ndarray:
        if which >= PHI_VD:
            a = (which - PHI_VD) % 3
            out = np.zeros(self.fshapes[a])
        else:
            out = np.zeros(self.shape)
        self.lib.or_field(self.h, which, _dp(out))
        return out

    def set_field(self, which: int, arr: np.ndarray):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        self.lib.or_set_field(self.h, which, _dp(a))

    def stats(self) -> dict:
        out = np.zeros(7)
        self.lib.or_stats(self.h, _dp(out))
        return dict(k_f=int(out[0]), E=out[1], dU=out[2], cg_iters_total=int(out[3]),
                    cg_iters_last=int(out[4]), phase_volume=out[5], cg_fail=int(out[6]))


# ---------------------------------------------------------------------------
# stage functions on plain arrays
# ---------------------------------------------------------------------------
def _faces3(p, arrs):
    sh = face_shapes(p)
    out = []
    for a in range(3):
        if arrs is not None and a < len(arrs) and arrs[a] is not None:
            out.append(np.ascontiguousarray(arrs[a], dtype=np.float64).reshape(sh[a]))
        else:
            out.append(np.zeros(sh[a]))
    return out


def stage_transport(p, solid, alpha, phi, nf, dt):
    lib = _load()
    P = make_params(p)
    sh = grid_shape(p)
    s = np.ascontiguousarray(solid, np.uint8).reshape(sh)
    al = np.ascontiguousarray(alpha, np.float64).reshape(sh)
    ph = _faces3(p, phi)
    n = _faces3(p, nf)
    out = np.zeros(sh)
    lib.or_stage_transport(C.byref(P), _u8(s), _dp(al), *[_dp(x) for x in ph], *[_dp(x) for x in n], dt, _dp(out))
    return out


def stage_interface(p, solid, alpha):
    lib = _load()
    P = make_params(p)
    sh = grid_shape(p)
    s = np.ascontiguousarray(solid, np.uint8).reshape(sh)
    al = np.ascontiguousarray(alpha, np.float64).reshape(sh)
    als = np.zeros(sh)
    n = _faces3(p, None)
    kap = np.zeros(sh)
    lib.or_stage_interface(C.byref(P), _u8(s), _dp(al), _dp(als), *[_dp(x) for x in n], _dp(kap))
    return als, n[: p["dim"]], kap


def stage_interface_area(p, solid, alpha):
    """Interface area sum |grad alpha| V over fluid cells (Gauss gradient)."""
    lib = _load()
    P = make_params(p)
    sh = grid_shape(p)
    s = np.ascontiguousarray(solid, np.uint8).reshape(sh)
    al = np.ascontiguousarray(alpha, np.float64).reshape(sh)
    return lib.or_stage_interface_area(C.byref(P), _u8(s), _dp(al))


def stage_relax_energy(p, solid, alpha, u):
    """sigma * interface area + kinetic energy of the cell velocities u (list of arrays)."""
    lib = _load()
    P = make_params(p)
    sh = grid_shape(p)
    s = np.ascontiguousarray(solid, np.uint8).reshape(sh)
    al = np.ascontiguousarray(alpha, np.float64).reshape(sh)
    uu = [np.ascontiguousarray(x, np.float64).reshape(sh) for x in u] + [np.zeros(sh)] * (3 - len(u))
    return lib.or_stage_relax_energy(C.byref(P), _u8(s), _dp(al), *[_dp(x) for x in uu])


def stage_poisson_apply(p, solid, cf, q):
    lib = _load()
    P = make_params(p)
    sh = grid_shape(p)
    s = np.ascontiguousarray(solid, np.uint8).reshape(sh)
    c3 = _faces3(p, cf)
    qq = np.ascontiguousarray(q, np.float64).reshape(sh)
    y = np.zeros(sh)
    lib.or_stage_poisson_apply(C.byref(P), _u8(s), *[_dp(x) for x in c3], _dp(qq), _dp(y))
    return y


def stage_poisson_cg(p, solid, cf, b, q0=None, rtol=1e-13, maxit=5000):
    lib = _load()
    P = make_params(p)
    sh = grid_shape(p)
    s = np.ascontiguousarray(solid, np.uint8).reshape(sh)
    c3 = _faces3(p, cf)
    bb = np.ascontiguousarray(b, np.float64).reshape(sh)
    q = np.zeros(sh) if q0 is None else np.array(q0, np.float64).reshape(sh)
    it = lib.or_stage_poisson_cg(C.byref(P), _u8(s), *[_dp(x) for x in c3], _dp(bb), _dp(q), rtol, maxit)
    return q, it


def stage_poisson_dense(p, solid, cf, b):
    lib = _load()
    P = make_params(p)
    sh = grid_shape(p)
    s = np.ascontiguousarray(solid, np.uint8).reshape(sh)
    c3 = _faces3(p, cf)
    bb = np.ascontiguousarray(b, np.float64).reshape(sh)
    q = np.zeros(sh)
    rc = lib.or_stage_poisson_dense(C.byref(P), _u8(s), *[_dp(x) for x in c3], _dp(bb), _dp(q))
    if rc != 0:
        raise RuntimeError("dense Cholesky failed: matrix not SPD")
    return q


def stage_normalised_residual(p, solid, cf, b, q):
    lib = _load()
    P = make_params(p)
    sh = grid_shape(p)
    s = np.ascontiguousarray(solid, np.uint8).reshape(sh)
    c3 = _faces3(p, cf)
    bb = np.ascontiguousarray(b, np.float64).reshape(sh)
    qq = np.ascontiguousarray(q, np.float64).reshape(sh)
    return lib.or_stage_normalised_residual(C.byref(P), _u8(s), *[_dp(x) for x in c3], _dp(bb), _dp(qq))


def stage_piso(p, solid, v, v_old, q, phic, alpha_old, alpha_new, kappa=None, vin_x=0.0, dt=1e-7):
    """One PISO solve; returns (v, q, phi, E, cg_iters, cg_fail)."""
    lib = _load()
    P = make_params(p)
    sh = grid_shape(p)
    s = np.ascontiguousarray(solid, np.uint8).reshape(sh)
    vv = [np.array(v[a] if a < len(v) else np.zeros(sh), np.float64).reshape(sh) for a in range(3)]
    vo = [np.array(v_old[a] if a < len(v_old) else np.zeros(sh), np.float64).reshape(sh) for a in range(3)]
    qq = np.array(q, np.float64).reshape(sh)
    ph = _faces3(p, None)
    pc = _faces3(p, phic)
    ao = np.ascontiguousarray(alpha_old, np.float64).reshape(sh)
    an = np.ascontiguousarray(alpha_new, np.float64).reshape(sh)
    kp = None if kappa is None else np.ascontiguousarray(kappa, np.float64).reshape(sh)
    out3 = np.zeros(3)
    kp_ptr = _dp(kp) if kp is not None else C.cast(None, C.POINTER(C.c_double))
    lib.or_stage_piso(C.byref(P), _u8(s), *[_dp(x) for x in vv], *[_dp(x) for x in vo], _dp(qq),
                      *[_dp(x) for x in ph], *[_dp(x) for x in pc], _dp(ao), _dp(an), kp_ptr,
                      vin_x, dt, _dp(out3))
    return vv[: p["dim"]], qq, ph[: p["dim"]], out3[0], int(out3[1]), int(out3[2])


def stage_momentum(p, solid, v, v_old, phic, alpha_new, vin_x=0.0, dt=1e-7):
    """One evaluation of HbyA = H/A and rA = 1/A (the momentum terms of PISO)."""
    lib = _load()
    if not hasattr(lib, "_mom_ready"):
        dp = C.POINTER(C.c_double)
        lib.or_stage_momentum.argtypes = [C.POINTER(OrParams), C.POINTER(C.c_uint8)] + [dp] * 10 + \
            [C.c_double, C.c_double] + [dp] * 4
        lib._mom_ready = True
    P = make_params(p)
    sh = grid_shape(p)
    s = np.ascontiguousarray(solid, np.uint8).reshape(sh)
    vv = [np.array(v[a] if a < len(v) else np.zeros(sh), np.float64).reshape(sh) for a in range(3)]
    vo = [np.array(v_old[a] if a < len(v_old) else np.zeros(sh), np.float64).reshape(sh) for a in range(3)]
    pc = _faces3(p, phic)
    an = np.ascontiguousarray(alpha_new, np.float64).reshape(sh)
    hb = [np.zeros(sh) for _ in range(3)]
    rA = np.zeros(sh)
    lib.or_stage_momentum(C.byref(P), _u8(s), *[_dp(x) for x in vv], *[_dp(x) for x in vo],
                          *[_dp(x) for x in pc], _dp(an), vin_x, dt, *[_dp(x) for x in hb], _dp(rA))
    return hb[: p["dim"]], rA


def stage_poisson_banded(p, solid, cf, b):
    """Exact pressure solve by banded Cholesky (shortest axis numbered fastest)."""
    lib = _load()
    if not hasattr(lib, "_band_ready"):
        dp = C.POINTER(C.c_double)
        lib.or_stage_poisson_banded.restype = C.c_int
        lib.or_stage_poisson_banded.argtypes = [C.POINTER(OrParams), C.POINTER(C.c_uint8)] + [dp] * 5
        lib._band_ready = True
    P = make_params(p)
    sh = grid_shape(p)
    s = np.ascontiguousarray(solid, np.uint8).reshape(sh)
    c3 = _faces3(p, cf)
    bb = np.ascontiguousarray(b, np.float64).reshape(sh)
    q = np.zeros(sh)
    rc = lib.or_stage_poisson_banded(C.byref(P), _u8(s), *[_dp(x) for x in c3], _dp(bb), _dp(q))
    if rc != 0:
        raise RuntimeError(f"banded Cholesky failed ({rc})")
    return q
