"""Thin ctypes binding of librmt.so (C ABI in include/rmt.h), same names as the C calls.

Argument marshalling only: every step of the method runs in the CUDA library.  Loading
fails loudly when the library cannot be built or loaded; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

RMT_OK, RMT_EINVAL, RMT_ENOMEM, RMT_ECUDA, RMT_ESTATE = 0, 1, 2, 3, 4
RMT_ENOCONVERGE, RMT_EDIVERGED, RMT_ETIMEOUT, RMT_EDEGENERATE, RMT_ERANGE = 5, 6, 7, 8, 9
RMT_BC_NOSLIP, RMT_BC_PERIODIC = 0, 1
RMT_PREC_FP64, RMT_PREC_FP32_REFINE = 0, 1
RMT_SHAPE_SPHERE, RMT_SHAPE_ELLIPSOID = 0, 1
RMT_F_U, RMT_F_P, RMT_F_RHO, RMT_F_XI, RMT_F_PHI, RMT_F_LAYER = 1, 2, 3, 4, 5, 6
RMT_F_DIVTAU_N, RMT_F_DIVTAU_H, RMT_F_UFACE_X, RMT_F_UFACE_Y, RMT_F_UFACE_Z = 20, 21, 22, 23, 24
RMT_F_MAC_Q, RMT_F_ADV_U, RMT_F_USTAR, RMT_F_PSI, RMT_F_RHO_HALF, RMT_F_XI_HALF = 25, 26, 27, 28, 29, 30
RMT_F_UMAC_X, RMT_F_UMAC_Y, RMT_F_UMAC_Z = 31, 32, 33
RMT_F_REPULSION = 34

RMT_JOB_QUEUED, RMT_JOB_RUNNING, RMT_JOB_DONE, RMT_JOB_FAILED = 0, 1, 2, 3

EXPORTS = ("rmt_create_grid", "rmt_add_solid", "rmt_step", "rmt_field_len", "rmt_read_fields",
           "rmt_write_fields", "rmt_read_fields_float", "rmt_write_fields_float", "rmt_last_cycles", "rmt_dt", "rmt_set_option", "rmt_kernel_launches", "rmt_profile",
           "rmt_profile_entries", "rmt_profile_name", "rmt_profile_read", "rmt_extrapolate_noalloc", "rmt_destroy_grid",
           "rmt_last_error", "rmt_grid_footprint", "rmt_grid_device_bytes", "rmt_batch_create", "rmt_batch_add",
           "rmt_batch_remove", "rmt_batch_step", "rmt_batch_sync", "rmt_batch_size", "rmt_batch_destroy",
           "rmt_batch_last_error", "rmt_server_create", "rmt_server_set_option", "rmt_server_submit",
           "rmt_server_poll", "rmt_server_job", "rmt_server_job_grid", "rmt_server_release",
           "rmt_server_resident_bytes", "rmt_server_clock", "rmt_server_cell_steps", "rmt_server_destroy",
           "rmt_autotune", "rmt_server_last_error", "rmt_server_stats", "rmt_wall_repulsion", "rmt_init_pressure",
           "rmt_body_stats")


class rmt_grid_desc(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("bc", C.c_int * 6),
        ("wall_u", (C.c_double * 3) * 6), ("rho_f", C.c_double), ("mu", C.c_double),
        ("eps_h", C.c_double), ("band_layers", C.c_int), ("dt", C.c_double),
        ("gravity", C.c_double * 3), ("precision", C.c_int), ("mg_rtol", C.c_double),
        ("mg_max_cycles", C.c_int), ("mg_fixed_cycles", C.c_int), ("mg_fixed_cycles_fe", C.c_int),
        ("cuda_stream", C.c_void_p), ("wall_dw", C.c_double),
    ]


class rmt_job_info(C.Structure):
    _fields_ = [
        ("state", C.c_int), ("status", C.c_int), ("steps_done", C.c_long), ("steps_total", C.c_long),
        ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double), ("device_bytes", C.c_size_t),
    ]


class rmt_server_stats_t(C.Structure):
    _fields_ = [
        ("batched_steps", C.c_long), ("graph_captures", C.c_long), ("capture_s", C.c_double),
        ("admit_s", C.c_double), ("retire_s", C.c_double), ("cell_steps", C.c_double),
    ]


class rmt_tune_result(C.Structure):
    _fields_ = [
        ("mac_pre", C.c_int), ("mac_post", C.c_int), ("mac_inner", C.c_int), ("mac_block", C.c_int),
        ("mac_cycles", C.c_int), ("fe_pre", C.c_int), ("fe_post", C.c_int), ("fe_inner", C.c_int),
        ("fe_block", C.c_int), ("fe_cycles", C.c_int), ("fe_omega", C.c_double), ("mac_ms", C.c_double),
        ("fe_ms", C.c_double), ("trials", C.c_int), ("mac_zchunk", C.c_int), ("fe_zchunk", C.c_int),
        ("mac_omega", C.c_double),
    ]


class rmt_solid_desc(C.Structure):
    _fields_ = [
        ("shape", C.c_int), ("center", C.c_double * 3), ("semi_axes", C.c_double * 3),
        ("rot", C.c_double * 9), ("rho_s", C.c_double), ("G", C.c_double), ("mu_a", C.c_double),
        ("gamma_t", C.c_double), ("active_A", C.c_double), ("active_omega", C.c_double),
        ("active_len", C.c_double), ("rep_A", C.c_double),
    ]


_lib = None


def load(build: bool = True):
    """Loads librmt.so (building it in-tree with nvcc first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"librmt.so not found at {path}; build it with paper_2104_00095_gb300.build")
    L = C.CDLL(path)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    L.rmt_create_grid.argtypes = [C.POINTER(rmt_grid_desc), C.POINTER(C.c_void_p)]
    L.rmt_add_solid.argtypes = [vp, C.POINTER(rmt_solid_desc), C.POINTER(C.c_int)]
    L.rmt_step.argtypes = [vp, C.c_int]
    L.rmt_field_len.argtypes = [vp, C.c_int]
    L.rmt_field_len.restype = C.c_long
    L.rmt_read_fields.argtypes = [vp, C.c_int, C.c_int, vp, C.c_size_t, C.c_int]
    L.rmt_write_fields.argtypes = [vp, C.c_int, C.c_int, vp, C.c_size_t, C.c_int]
    L.rmt_read_fields_float.argtypes = [vp, C.c_int, C.c_int, vp, C.c_size_t, C.c_int]
    L.rmt_write_fields_float.argtypes = [vp, C.c_int, C.c_int, vp, C.c_size_t, C.c_int]
    L.rmt_last_cycles.argtypes = [vp, C.c_int]
    L.rmt_dt.argtypes = [vp]
    L.rmt_dt.restype = C.c_double
    L.rmt_set_option.argtypes = [vp, C.c_char_p, C.c_double]
    L.rmt_set_option.restype = C.c_int
    L.rmt_kernel_launches.argtypes = []
    L.rmt_kernel_launches.restype = C.c_long
    L.rmt_profile.argtypes = [vp, C.c_int]
    L.rmt_profile.restype = C.c_int
    L.rmt_profile_entries.argtypes = []
    L.rmt_profile_entries.restype = C.c_int
    L.rmt_profile_name.argtypes = [C.c_int]
    L.rmt_profile_name.restype = C.c_char_p
    L.rmt_profile_read.argtypes = [vp, C.c_int, dp, C.POINTER(C.c_long), dp]
    L.rmt_profile_read.restype = C.c_int
    L.rmt_extrapolate_noalloc.argtypes = [C.POINTER(rmt_grid_desc), C.POINTER(rmt_solid_desc), vp, vp, vp, vp, vp]
    L.rmt_extrapolate_noalloc.restype = C.c_int
    L.rmt_destroy_grid.argtypes = [vp]
    L.rmt_last_error.argtypes = [vp]
    L.rmt_last_error.restype = C.c_char_p
    L.rmt_grid_footprint.argtypes = [C.POINTER(rmt_grid_desc), C.c_int]
    L.rmt_grid_footprint.restype = C.c_size_t
    L.rmt_grid_device_bytes.argtypes = [vp]
    L.rmt_grid_device_bytes.restype = C.c_size_t
    L.rmt_batch_create.argtypes = [vp, C.POINTER(C.c_void_p)]
    for f in ("rmt_batch_add", "rmt_batch_remove"):
        getattr(L, f).argtypes = [vp, vp]
    L.rmt_batch_step.argtypes = [vp, C.c_int]
    for f in ("rmt_batch_sync", "rmt_batch_size", "rmt_batch_destroy"):
        getattr(L, f).argtypes = [vp]
    L.rmt_batch_last_error.argtypes = [vp]
    L.rmt_batch_last_error.restype = C.c_char_p
    L.rmt_server_create.argtypes = [C.c_size_t, vp, C.POINTER(C.c_void_p)]
    L.rmt_server_set_option.argtypes = [vp, C.c_char_p, C.c_double]
    L.rmt_server_submit.argtypes = [vp, C.POINTER(rmt_grid_desc), C.POINTER(rmt_solid_desc), C.c_int, C.c_long,
                                    C.POINTER(C.c_int)]
    L.rmt_server_poll.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.rmt_server_job.argtypes = [vp, C.c_int, C.POINTER(rmt_job_info)]
    L.rmt_server_job_grid.argtypes = [vp, C.c_int]
    L.rmt_server_job_grid.restype = C.c_void_p
    L.rmt_server_release.argtypes = [vp, C.c_int]
    L.rmt_server_resident_bytes.argtypes = [vp]
    L.rmt_server_resident_bytes.restype = C.c_size_t
    for f in ("rmt_server_clock", "rmt_server_cell_steps"):
        getattr(L, f).argtypes = [vp]
        getattr(L, f).restype = C.c_double
    L.rmt_server_destroy.argtypes = [vp]
    L.rmt_server_last_error.argtypes = [vp]
    L.rmt_server_last_error.restype = C.c_char_p
    L.rmt_server_stats.argtypes = [vp, C.POINTER(rmt_server_stats_t)]
    L.rmt_server_stats.restype = C.c_int
    L.rmt_autotune.argtypes = [vp, C.c_double, C.POINTER(rmt_tune_result)]
    L.rmt_init_pressure.argtypes = [vp, C.c_int, C.c_double, C.POINTER(C.c_int)]
    L.rmt_init_pressure.restype = C.c_int
    L.rmt_body_stats.argtypes = [vp, C.c_int, C.POINTER(C.c_double)]
    L.rmt_body_stats.restype = C.c_int
    L.rmt_wall_repulsion.argtypes = [C.c_double] * 8
    L.rmt_wall_repulsion.restype = C.c_double
    for f in ("rmt_create_grid", "rmt_add_solid", "rmt_step", "rmt_read_fields", "rmt_write_fields",
              "rmt_read_fields_float", "rmt_write_fields_float", "rmt_destroy_grid", "rmt_batch_create", "rmt_batch_add", "rmt_batch_remove", "rmt_batch_step",
              "rmt_batch_sync", "rmt_batch_size", "rmt_batch_destroy", "rmt_server_create", "rmt_server_set_option",
              "rmt_server_submit", "rmt_server_poll", "rmt_server_job", "rmt_server_release", "rmt_server_destroy",
              "rmt_autotune"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def kernel_launches() -> int:
    """Kernels launched by librmt.so so far in this process."""
    return load().rmt_kernel_launches()


def make_grid_desc(scene: dict, stream: int = 0) -> rmt_grid_desc:
    d = rmt_grid_desc()
    d.n[:] = list(scene["n"])
    d.lo[:] = list(scene.get("lo", (0.0, 0.0, 0.0)))
    d.hi[:] = list(scene.get("hi", (1.0, 1.0, 1.0)))
    d.bc[:] = list(scene["bc"])
    wu = scene.get("wall_u", [[0.0] * 3] * 6)
    for f in range(6):
        d.wall_u[f][:] = list(wu[f])
    d.rho_f, d.mu = scene["rho_f"], scene["mu"]
    d.eps_h, d.band_layers = scene.get("eps_h", 1.5), scene.get("band_layers", 4)
    d.dt = scene.get("dt", 0.0)
    d.gravity[:] = list(scene.get("gravity", (0.0, 0.0, 0.0)))
    d.precision = RMT_PREC_FP32_REFINE if scene.get("precision", "fp64") == "fp32" else RMT_PREC_FP64
    d.mg_rtol = scene.get("mg_rtol", 0.0)
    d.mg_max_cycles = scene.get("mg_max_cycles", 0)
    d.mg_fixed_cycles = scene.get("mg_fixed_cycles", 0)
    d.mg_fixed_cycles_fe = scene.get("mg_fixed_cycles_fe", 0)
    d.cuda_stream = stream or None
    d.wall_dw = scene.get("wall_dw", 0.0)
    return d


def make_solid_desc(s: dict) -> rmt_solid_desc:
    o = rmt_solid_desc()
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


def footprint(scene: dict) -> int:
    """Device bytes a grid of this scene requests (rmt_grid_footprint); 0 if invalid."""
    return load().rmt_grid_footprint(C.byref(make_grid_desc(scene)), len(scene.get("solids", [])))


class RMTError(RuntimeError):
    def __init__(self, call: str, status: int, msg: str):
        super().__init__(f"{call} failed with status {status}: {msg}")
        self.status = status


class Grid:
    """One simulation on the GPU; wraps the opaque rmt_grid handle."""

    def __init__(self, scene: dict, stream: int = 0):
        self._L = load()
        self.scene = scene
        self.n = tuple(scene["n"])
        self._g = C.c_void_p()
        self._check("rmt_create_grid", self._L.rmt_create_grid(C.byref(make_grid_desc(scene, stream)),
                                                              C.byref(self._g)))
        self.nsolids = 0
        for k, v in scene.get("options", {}).items():
            self.set_option(k, v)
        for s in scene.get("solids", []):
            sid = C.c_int()
            self._check("rmt_add_solid", self._L.rmt_add_solid(self._g, C.byref(make_solid_desc(s)),
                                                              C.byref(sid)))
            self.nsolids += 1

    def _check(self, call: str, rc: int):
        if rc != RMT_OK:
            msg = self._L.rmt_last_error(self._g).decode() if self._g else ""
            raise RMTError(call, rc, msg)

    def close(self):
        if getattr(self, "_g", None) and self._g.value and getattr(self, "_owned", True):
            self._L.rmt_destroy_grid(self._g)
        self._g = C.c_void_p()

    def __del__(self):
        self.close()

    def step(self, nsteps: int = 1):
        self._check("rmt_step", self._L.rmt_step(self._g, nsteps))

    def init_pressure(self, max_iters: int, tol: float) -> int:
        """Initial pressure iterations before the first step; returns the iteration count."""
        it = C.c_int()
        self._check("rmt_init_pressure", self._L.rmt_init_pressure(self._g, int(max_iters), float(tol), C.byref(it)))
        return it.value

    def body_stats(self, solid: int = 0) -> np.ndarray:
        """Diagnostics of one body at the current time: centroid velocity (3), active power,
        volume, elastic energy, RMS of J - 1."""
        out = (C.c_double * 7)()
        self._check("rmt_body_stats", self._L.rmt_body_stats(self._g, int(solid), out))
        return np.array(out[:], dtype=np.float64)

    def field_len(self, field: int) -> int:
        return self._L.rmt_field_len(self._g, field)

    def read(self, field: int, solid: int = 0, out: np.ndarray | None = None) -> np.ndarray:
        n = self.field_len(field)
        if out is None:
            out = np.empty(n, dtype=np.float64)
        self._check("rmt_read_fields", self._L.rmt_read_fields(self._g, field, solid, out.ctypes.data, out.nbytes, 0))
        return out

    def read_device(self, field: int, ptr: int, nbytes: int, solid: int = 0):
        self._check("rmt_read_fields", self._L.rmt_read_fields(self._g, field, solid, C.c_void_p(ptr), nbytes, 1))

    def read_float(self, field: int, solid: int = 0, out: np.ndarray | None = None) -> np.ndarray:
        n = self.field_len(field)
        if out is None:
            out = np.empty(n, dtype=np.float32)
        self._check("rmt_read_fields_float",
                    self._L.rmt_read_fields_float(self._g, field, solid, out.ctypes.data, out.nbytes, 0))
        return out

    def read_float_ptr(self, field: int, ptr: int, nbytes: int, is_device: int, solid: int = 0):
        self._check("rmt_read_fields_float",
                    self._L.rmt_read_fields_float(self._g, field, solid, C.c_void_p(ptr), nbytes, is_device))

    def write_float(self, field: int, data: np.ndarray, solid: int = 0):
        a = np.ascontiguousarray(data, dtype=np.float32).reshape(-1)
        self._check("rmt_write_fields_float",
                    self._L.rmt_write_fields_float(self._g, field, solid, a.ctypes.data, a.nbytes, 0))

    def write_float_ptr(self, field: int, ptr: int, nbytes: int, is_device: int, solid: int = 0):
        self._check("rmt_write_fields_float",
                    self._L.rmt_write_fields_float(self._g, field, solid, C.c_void_p(ptr), nbytes, is_device))

    def write(self, field: int, data: np.ndarray, solid: int = 0):
        a = np.ascontiguousarray(data, dtype=np.float64).reshape(-1)
        self._check("rmt_write_fields", self._L.rmt_write_fields(self._g, field, solid, a.ctypes.data, a.nbytes, 0))

    def write_ptr(self, field: int, ptr: int, nbytes: int, is_device: int, solid: int = 0):
        self._check("rmt_write_fields",
                    self._L.rmt_write_fields(self._g, field, solid, C.c_void_p(ptr), nbytes, is_device))

    @property
    def dt(self) -> float:
        self.read(RMT_F_RHO)
        return self._L.rmt_dt(self._g)

    def set_option(self, name: str, value: float):
        self._check("rmt_set_option", self._L.rmt_set_option(self._g, name.encode(), float(value)))

    def profile(self, enable: bool):
        self._check("rmt_profile", self._L.rmt_profile(self._g, 1 if enable else 0))

    def profile_read(self) -> list:
        """[(name, total_ms, launches, bytes_per_launch)] for every profile entry."""
        out = []
        for e in range(self._L.rmt_profile_entries()):
            ms, n, b = C.c_double(), C.c_long(), C.c_double()
            self._check("rmt_profile_read", self._L.rmt_profile_read(self._g, e, C.byref(ms), C.byref(n), C.byref(b)))
            out.append((self._L.rmt_profile_name(e).decode(), ms.value, n.value, b.value))
        return out

    def cycles(self):
        return self._L.rmt_last_cycles(self._g, 0), self._L.rmt_last_cycles(self._g, 1)

    def autotune(self, rtol: float = 1e-6) -> dict:
        """Picks and applies the multigrid schedule, cycle counts and block shapes (rmt_autotune)."""
        r = rmt_tune_result()
        self._check("rmt_autotune", self._L.rmt_autotune(self._g, float(rtol), C.byref(r)))
        return {k: getattr(r, k) for k, _ in rmt_tune_result._fields_}

    def device_bytes(self) -> int:
        return self._L.rmt_grid_device_bytes(self._g)

    @classmethod
    def _wrap(cls, handle: int, scene: dict | None = None):
        """A non-owning Grid view of a handle owned elsewhere (a server job)."""
        g = cls.__new__(cls)
        g._L = load()
        g.scene = scene or {}
        g._g = C.c_void_p(handle)
        g._owned = False
        g.nsolids = len(g.scene.get("solids", []))
        return g


class Batch:
    """Grids advanced together, one CUDA-graph launch per step (rmt_batch_*)."""

    def __init__(self, stream: int = 0):
        self._L = load()
        self._b = C.c_void_p()
        self._check("rmt_batch_create", self._L.rmt_batch_create(stream or None, C.byref(self._b)))
        self.members = []

    def _check(self, call: str, rc: int):
        if rc != RMT_OK:
            msg = self._L.rmt_batch_last_error(self._b).decode() if self._b else ""
            raise RMTError(call, rc, msg)

    def add(self, g: Grid):
        self._check("rmt_batch_add", self._L.rmt_batch_add(self._b, g._g))
        self.members.append(g)

    def remove(self, g: Grid):
        self._check("rmt_batch_remove", self._L.rmt_batch_remove(self._b, g._g))
        self.members.remove(g)

    def step(self, nsteps: int = 1):
        self._check("rmt_batch_step", self._L.rmt_batch_step(self._b, nsteps))

    def sync(self):
        self._check("rmt_batch_sync", self._L.rmt_batch_sync(self._b))

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            self._L.rmt_batch_destroy(self._b)
            self._b = C.c_void_p()
            self.members = []

    def __del__(self):
        self.close()


class Server:
    """Continuous-batching simulation server under a device-memory budget (rmt_server_*)."""

    def __init__(self, budget_bytes: int, stream: int = 0, options: dict | None = None):
        self._L = load()
        self._s = C.c_void_p()
        rc = self._L.rmt_server_create(int(budget_bytes), stream or None, C.byref(self._s))
        if rc != RMT_OK:
            raise RMTError("rmt_server_create", rc, "")
        for k, v in (options or {}).items():
            self._L.rmt_server_set_option(self._s, k.encode(), float(v))
        self.scenes = {}

    def set_option(self, name: str, value: float):
        """rmt_set_option(name, value) for every job admitted from now on."""
        rc = self._L.rmt_server_set_option(self._s, name.encode(), float(value))
        if rc != RMT_OK:
            raise RMTError("rmt_server_set_option", rc, "")

    def submit(self, scene: dict, nsteps: int) -> int:
        sol = scene.get("solids", [])
        arr = (rmt_solid_desc * max(len(sol), 1))(*[make_solid_desc(s) for s in sol])
        jid = C.c_int()
        rc = self._L.rmt_server_submit(self._s, C.byref(make_grid_desc(scene)), arr, len(sol), int(nsteps),
                                       C.byref(jid))
        if rc != RMT_OK:
            raise RMTError("rmt_server_submit", rc, "job rejected")
        self.scenes[jid.value] = scene
        return jid.value

    def poll(self):
        """One scheduling round; returns (running, queued)."""
        r, q = C.c_int(), C.c_int()
        rc = self._L.rmt_server_poll(self._s, C.byref(r), C.byref(q))
        if rc != RMT_OK:
            raise RMTError("rmt_server_poll", rc, self._L.rmt_server_last_error(self._s).decode())
        return r.value, q.value

    def job(self, jid: int) -> dict:
        info = rmt_job_info()
        rc = self._L.rmt_server_job(self._s, jid, C.byref(info))
        if rc != RMT_OK:
            raise RMTError("rmt_server_job", rc, "unknown job")
        return {k: getattr(info, k) for k, _ in rmt_job_info._fields_}

    def grid(self, jid: int) -> Grid:
        h = self._L.rmt_server_job_grid(self._s, jid)
        if not h:
            raise RMTError("rmt_server_job_grid", RMT_EINVAL, "no grid for this job")
        return Grid._wrap(h, self.scenes.get(jid))

    def release(self, jid: int):
        rc = self._L.rmt_server_release(self._s, jid)
        if rc != RMT_OK:
            raise RMTError("rmt_server_release", rc, "")
        self.scenes.pop(jid, None)

    def resident_bytes(self) -> int:
        return self._L.rmt_server_resident_bytes(self._s)

    def clock(self) -> float:
        return self._L.rmt_server_clock(self._s)

    def cell_steps(self) -> float:
        return self._L.rmt_server_cell_steps(self._s)

    def stats(self) -> dict:
        st = rmt_server_stats_t()
        self._L.rmt_server_stats(self._s, C.byref(st))
        return {k: getattr(st, k) for k, _ in rmt_server_stats_t._fields_}

    def close(self):
        if getattr(self, "_s", None) and self._s.value:
            self._L.rmt_server_destroy(self._s)
            self._s = C.c_void_p()

    def __del__(self):
        self.close()
