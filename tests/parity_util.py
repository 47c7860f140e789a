"""Helpers shared by the GPU parity tests: run a scene on the CUDA path and on the oracle."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2104_00095_gb300 import rmt


def gpu_available() -> bool:
    try:
        lib = C.CDLL("libcudart.so")
        n = C.c_int(0)
        return lib.cudaGetDeviceCount(C.byref(n)) == 0 and n.value > 0
    except OSError:
        return False


needs_gpu = pytest.mark.skipif(not gpu_available(), reason="no CUDA device")

# field ids are shared by the two libraries
FIELDS_CELL = [rmt.RMT_F_U, rmt.RMT_F_P, rmt.RMT_F_RHO]
FIELDS_BODY = [rmt.RMT_F_XI, rmt.RMT_F_PHI]


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """Relative L2 difference over the entries finite in both; the NaN masks must agree."""
    fa, fb = np.isfinite(a), np.isfinite(b)
    assert np.array_equal(fa, fb), f"presence masks differ in {np.count_nonzero(fa != fb)} entries"
    if not fa.any():
        return 0.0
    nb = np.linalg.norm(b[fb])
    d = np.linalg.norm(a[fa] - b[fb])
    return d / nb if nb > 0 else d


def compare_state(g, o, nsol, tol, check_layers=True, tag=""):
    """Compares the state of a CUDA grid g with the oracle o; returns the worst rel-L2."""
    worst = 0.0
    for f in FIELDS_CELL:
        e = rel_l2(g.read(f), o.read(f))
        assert e <= tol, f"{tag} field {f}: rel-L2 {e:.3e} > {tol:.1e}"
        worst = max(worst, e)
    for m in range(nsol):
        if check_layers:
            lg, lo = g.read(rmt.RMT_F_LAYER, m), o.read(O.F_LAYER, m)
            bad = np.flatnonzero(lg != lo)
            if bad.size:
                # a label may flip only where the level set is within rounding of zero
                phi = o.read(O.F_PHI, m)
                raise AssertionError(f"{tag} body {m}: {bad.size} layer labels differ; |phi| there "
                                     f"{np.nanmax(np.abs(phi[bad])) if np.isfinite(phi[bad]).any() else 'nan'}")
        for f in FIELDS_BODY:
            e = rel_l2(g.read(f, m), o.read(f, m))
            assert e <= tol, f"{tag} body {m} field {f}: rel-L2 {e:.3e} > {tol:.1e}"
            worst = max(worst, e)
    return worst


def pair(scene):
    """The same scene on both paths (the GPU solves to 1e-13 so that both reach the same
    discrete solution; the oracle's CG runs to 1e-14)."""
    sc = dict(scene)
    sc.setdefault("mg_rtol", 1e-13)
    sc.setdefault("mg_max_cycles", 200)
    g = rmt.Grid(sc)
    o = O.Oracle(sc)
    return g, o
