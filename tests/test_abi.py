"""The C-ABI library builds for sm_103a, loads, and exports every call include/rmt.h declares.

Runs without a GPU: only host-side argument validation is exercised (no device work)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2104_00095_gb300 import rmt, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "rmt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rmt_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_call():
    L = rmt.load()
    names = _declared()
    assert set(names) == set(rmt.EXPORTS)
    for n in names:
        assert hasattr(L, n), n


def _desc(**kw):
    sc = scenes.cavity_sphere(16)
    sc.update(kw)
    return rmt.make_grid_desc(sc)


@pytest.mark.parametrize("bad", [
    dict(n=(3, 16, 16)),                                   # too small
    dict(hi=(1.0, 2.0, 1.0)),                              # anisotropic spacing
    dict(bc=[1, 0, 0, 0, 0, 0]),                           # periodic on one face only
    dict(eps_h=0.0),
    dict(band_layers=0),
    dict(n=(1290, 1290, 1290)),                            # 2^31 nodes or more: 32-bit indices
])
def test_create_grid_rejects_bad_descriptors(bad):
    L = rmt.load()
    g = C.c_void_p()
    assert L.rmt_create_grid(C.byref(_desc(**bad)), C.byref(g)) == rmt.RMT_EINVAL
    assert not g.value


def test_create_grid_rejects_odd_period_and_normal_wall_velocity():
    L = rmt.load()
    g = C.c_void_p()
    sc = scenes._box(15, periodic=True)
    assert L.rmt_create_grid(C.byref(rmt.make_grid_desc(sc)), C.byref(g)) == rmt.RMT_EINVAL
    sc = scenes.cavity_sphere(16)
    sc["wall_u"][5] = [1.0, 0.0, 0.3]  # normal component on the lid
    assert L.rmt_create_grid(C.byref(rmt.make_grid_desc(sc)), C.byref(g)) == rmt.RMT_EINVAL


def test_add_solid_validation_is_host_side():
    L = rmt.load()
    g = C.c_void_p()
    assert L.rmt_create_grid(C.byref(_desc()), C.byref(g)) == rmt.RMT_OK
    bad = rmt.make_solid_desc(scenes.solid(semi_axes=(0.0, 0.1, 0.1)))
    assert L.rmt_add_solid(g, C.byref(bad), None) == rmt.RMT_EINVAL
    good = rmt.make_solid_desc(scenes.solid())
    sid = C.c_int(-1)
    assert L.rmt_add_solid(g, C.byref(good), C.byref(sid)) == rmt.RMT_OK and sid.value == 0
    assert L.rmt_field_len(g, rmt.RMT_F_U) == 3 * 16**3
    assert L.rmt_field_len(g, rmt.RMT_F_P) == 17**3
    assert L.rmt_field_len(g, rmt.RMT_F_UFACE_X) == 3 * 17 * 16 * 16
    assert L.rmt_field_len(g, 999) == -1


def test_wall_repulsion_helper_matches_the_oracle():
    """rmt_wall_repulsion (host arithmetic, no GPU) and the oracle's A_rep agree."""
    import oracle as O
    from paper_2104_00095_gb300 import rmt

    L = rmt.load()
    rng = np.random.default_rng(7)
    for _ in range(50):
        args = [rng.uniform(1e-4, 1e-1), rng.uniform(0, 5), rng.uniform(1e-3, 0.1), rng.uniform(0.01, 0.3),
                rng.uniform(0.2, 3), rng.uniform(0.5, 1.5), rng.uniform(0, 2), rng.uniform(0, 6)]
        assert L.rmt_wall_repulsion(*args) == O.lib().orc_rep_accel(*args)
