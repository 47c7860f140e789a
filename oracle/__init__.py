"""FP64 CPU oracle of the reference-map-technique per-step update (arXiv 2104.00095).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg.  The product package never imports it.

The oracle is plain C (rmt_oracle.c), built here with gcc -O2 -ffp-contract=off -fopenmp into
liboracle.so and driven through ctypes.  The Python side only marshals arguments.  Its cell
loops run on all host cores (OMP_NUM_THREADS limits them); its sums use fixed chunks and its
element loops fixed colours, so a result does not depend on the thread count.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rmt_oracle.c")
_HDR = os.path.join(_HERE, "rmt_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

F_U, F_P, F_RHO, F_XI, F_PHI, F_LAYER = 1, 2, 3, 4, 5, 6
F_DIVTAU_N, F_DIVTAU_H, F_UFACE_X, F_UFACE_Y, F_UFACE_Z = 20, 21, 22, 23, 24
F_MAC_Q, F_ADV_U, F_USTAR, F_PSI, F_RHO_HALF, F_XI_HALF = 25, 26, 27, 28, 29, 30
F_UMAC_X, F_UMAC_Y, F_UMAC_Z = 31, 32, 33
F_REPULSION = 34

BC_NOSLIP, BC_PERIODIC = 0, 1
SHAPE_SPHERE, SHAPE_ELLIPSOID = 0, 1


class GridDesc(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("bc", C.c_int * 6),
        ("wall_u", (C.c_double * 3) * 6), ("rho_f", C.c_double), ("mu", C.c_double),
        ("eps_h", C.c_double), ("band_layers", C.c_int), ("dt", C.c_double),
        ("gravity", C.c_double * 3), ("solve_rtol", C.c_double), ("solve_max_iter", C.c_int),
        ("wall_dw", C.c_double),
    ]


class SolidDesc(C.Structure):
    _fields_ = [
        ("shape", C.c_int), ("center", C.c_double * 3), ("semi_axes", C.c_double * 3),
        ("rot", C.c_double * 9), ("rho_s", C.c_double), ("G", C.c_double), ("mu_a", C.c_double),
        ("gamma_t", C.c_double), ("active_A", C.c_double), ("active_omega", C.c_double),
        ("active_len", C.c_double), ("rep_A", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compiles liboracle.so (gcc, FP64, no FMA contraction, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))):
        return _LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c11", "-D_DEFAULT_SOURCE",
           "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.orc_create.argtypes = [C.POINTER(GridDesc), C.POINTER(C.c_void_p)]
        L.orc_add_solid.argtypes = [C.c_void_p, C.POINTER(SolidDesc), ip]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_init_pressure.argtypes = [C.c_void_p, C.c_int, C.c_double, ip]
        L.orc_body_stats.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_field_len.argtypes = [C.c_void_p, C.c_int]
        L.orc_field_len.restype = C.c_long
        L.orc_read.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, C.c_long]
        L.orc_write.argtypes = [C.c_void_p, C.c_int, C.c_int, dp, C.c_long]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_destroy.restype = None
        L.orc_dt.argtypes = [C.c_void_p]
        L.orc_dt.restype = C.c_double
        L.orc_last_iters.argtypes = [C.c_void_p, C.c_int]
        L.orc_last_true_residual.argtypes = [C.c_void_p, C.c_int]
        L.orc_last_true_residual.restype = C.c_double
        L.orc_error.argtypes = [C.c_void_p]
        L.orc_error.restype = C.c_char_p
        for fn in ("orc_heaviside", "orc_dheaviside"):
            getattr(L, fn).argtypes = [C.c_double, C.c_double]
            getattr(L, fn).restype = C.c_double
        L.orc_limited_slope.argtypes = [dp, ip, C.c_double]
        L.orc_limited_slope.restype = C.c_double
        L.orc_godunov_normal.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_godunov_normal.restype = C.c_double
        L.orc_upwind.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_upwind.restype = C.c_double
        L.orc_phi0.argtypes = [C.POINTER(SolidDesc), dp]
        L.orc_phi0.restype = C.c_double
        L.orc_neohookean.argtypes = [dp, C.c_double, dp]
        L.orc_mix_weights.argtypes = [C.c_int, dp, dp]
        L.orc_mix_weights.restype = C.c_double
        L.orc_mac_project.argtypes = [C.c_void_p, dp, dp, dp, dp, C.c_double, dp]
        L.orc_fe_solve.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_fe_apply.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_fe_apply.restype = None
        L.orc_fe_weak_div.argtypes = [C.c_void_p, dp, dp]
        L.orc_fe_weak_div.restype = None
        L.orc_cell_grad.argtypes = [C.c_void_p, dp, dp]
        L.orc_cell_grad.restype = None
        L.orc_rep_accel.argtypes = [C.c_double] * 8
        L.orc_rep_accel.restype = C.c_double
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_grid_desc(scene: dict) -> GridDesc:
    d = GridDesc()
    d.n[:] = list(scene["n"])
    d.lo[:] = list(scene.get("lo", (0.0, 0.0, 0.0)))
    d.hi[:] = list(scene.get("hi", (1.0, 1.0, 1.0)))
    d.bc[:] = list(scene["bc"])
    for f in range(6):
        d.wall_u[f][:] = list(scene.get("wall_u", [[0.0] * 3] * 6)[f])
    d.rho_f, d.mu = scene["rho_f"], scene["mu"]
    d.eps_h, d.band_layers = scene.get("eps_h", 1.5), scene.get("band_layers", 4)
    d.dt = scene.get("dt", 0.0)
    d.gravity[:] = list(scene.get("gravity", (0.0, 0.0, 0.0)))
    d.solve_rtol = scene.get("oracle_rtol", 1e-14)
    d.solve_max_iter = scene.get("oracle_max_iter", 20000)
    d.wall_dw = scene.get("wall_dw", 0.0)
    return d


def make_solid_desc(s: dict) -> SolidDesc:
    o = SolidDesc()
    o.shape = s["shape"]
    o.center[:] = list(s["center"])
    o.semi_axes[:] = list(s["semi_axes"])
    o.rot[:] = list(np.asarray(s.get("rot", np.eye(3)), dtype=np.float64).reshape(9))
    o.rho_s, o.G, o.mu_a, o.gamma_t = s["rho_s"], s["G"], s["mu_a"], s.get("gamma_t", 0.0)
    o.active_A = s.get("active_A", 0.0)
    o.active_omega = s.get("active_omega", 0.0)
    o.active_len = s.get("active_len", 1.0)
    o.rep_A = s.get("rep_A", 0.0)
    return o


class Oracle:
    """One simulation held by the CPU oracle."""

    def __init__(self, scene: dict):
        L = lib()
        self._L = L
        self.scene = scene
        self.n = tuple(scene["n"])
        self._g = C.c_void_p()
        rc = L.orc_create(C.byref(make_grid_desc(scene)), C.byref(self._g))
        if rc != 0:
            raise ValueError(f"orc_create failed ({rc})")
        self.nsol = 0
        for s in scene.get("solids", []):
            sid = C.c_int()
            rc = L.orc_add_solid(self._g, C.byref(make_solid_desc(s)), C.byref(sid))
            if rc != 0:
                raise ValueError(f"orc_add_solid failed ({rc})")
            self.nsol += 1

    def __del__(self):
        if getattr(self, "_g", None) and self._g.value:
            self._L.orc_destroy(self._g)
            self._g = C.c_void_p()

    def step(self, nsteps: int = 1) -> int:
        return self._L.orc_step(self._g, nsteps)

    def body_stats(self, solid: int = 0) -> np.ndarray:
        """[centroid velocity x, y, z, active power, volume, elastic energy, RMS of J - 1] of
        one body."""
        out = np.zeros(7)
        rc = self._L.orc_body_stats(self._g, solid, _dp(out))
        if rc != 0:
            raise ValueError(f"orc_body_stats failed ({rc})")
        return out

    def init_pressure(self, max_iters: int, tol: float):
        """Initial pressure iterations; returns (status, iterations)."""
        it = C.c_int()
        rc = self._L.orc_init_pressure(self._g, max_iters, tol, C.byref(it))
        return rc, it.value

    @property
    def dt(self) -> float:
        self.read(F_RHO)  # forces initialisation
        return self._L.orc_dt(self._g)

    def iters(self):
        return self._L.orc_last_iters(self._g, 0), self._L.orc_last_iters(self._g, 1)

    def true_residuals(self):
        return self._L.orc_last_true_residual(self._g, 0), self._L.orc_last_true_residual(self._g, 1)

    def read(self, field: int, solid: int = 0) -> np.ndarray:
        n = self._L.orc_field_len(self._g, field)
        out = np.empty(n, dtype=np.float64)
        rc = self._L.orc_read(self._g, field, solid, _dp(out), n)
        if rc != 0:
            raise ValueError(f"orc_read({field}) failed ({rc})")
        return out

    def write(self, field: int, data: np.ndarray, solid: int = 0) -> int:
        a = np.ascontiguousarray(data, dtype=np.float64).reshape(-1)
        return self._L.orc_write(self._g, field, solid, _dp(a), a.size)

    def error(self) -> str:
        return self._L.orc_error(self._g).decode()
