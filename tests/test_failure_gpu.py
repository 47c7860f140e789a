"""Failure detection on the GPU path, with every failure made on the host (no device fault).

* A NaN written into the velocity from the host (the inject_nan_step option) is caught by the
  non-finite check that every pressure solve applies to the means of its right-hand side and
  solution: RMT_EDIVERGED, reported by a later call in fixed-cycle graph mode (no step waits),
  at once in adaptive mode, by rmt_batch_sync for a batch member, and by the server, which
  evicts the job, returns its memory to the budget and lets the other jobs finish.
* A multigrid cycle cap below what the tolerance needs gives RMT_ENOCONVERGE.
* An allocation made to fail (the inject_alloc option) gives RMT_ENOMEM.
* FP32 storage keeps reference maps relative to one periodic image around each body; a band that
  reaches the seam of that image window gives RMT_ERANGE (the FP64 form has no such limit).
"""
import numpy as np
import pytest

from paper_2104_00095_gb300 import rmt, scenes as S
from parity_util import needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]


def _fixed(sc, graph=1):
    return dict(sc, mg_fixed_cycles=4, mg_fixed_cycles_fe=4, options={"graph": graph})


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_nan_in_the_velocity_is_reported_as_diverged_in_graph_mode(precision):
    g = rmt.Grid(_fixed(S.cavity_sphere(24, precision=precision)))
    g.set_option("inject_nan_step", 2)
    g.step(4)  # no synchronisation inside: the failure is in flight
    u = g.read(rmt.RMT_F_U)  # waits for the stream (the read itself is allowed)
    assert not np.all(np.isfinite(u))
    with pytest.raises(rmt.RMTError) as ei:
        g.step(1)
    assert ei.value.status == rmt.RMT_EDIVERGED
    with pytest.raises(rmt.RMTError) as ei:
        g.step(1)
    assert ei.value.status == rmt.RMT_ESTATE  # the error is sticky
    g.close()


def test_nan_in_the_velocity_is_reported_at_once_in_adaptive_mode():
    g = rmt.Grid(S.cavity_sphere(24))
    g.set_option("inject_nan_step", 1)
    g.step(1)
    with pytest.raises(rmt.RMTError) as ei:
        g.step(1)
    assert ei.value.status == rmt.RMT_EDIVERGED
    g.close()


def test_a_new_grid_starts_with_clean_error_words():
    """The host copy of a grid's error words starts at zero.  A grid whose steps diverged leaves
    non-zero words in its pinned buffer when it is destroyed; a new grid initialised by a read
    polls its words at its first step, before a copy of its own has landed, and must not see the
    old grid's words if the pinned block comes back to it."""
    for _ in range(3):
        bad = rmt.Grid(_fixed(S.cavity_sphere(24, precision="fp32")))
        bad.set_option("inject_nan_step", 1)
        bad.step(3)
        bad.read(rmt.RMT_F_U)  # the diverged words have landed in the pinned buffer
        bad.close()
        g = rmt.Grid(_fixed(S.cavity_sphere(24, precision="fp32")))
        g.read(rmt.RMT_F_LAYER, 0)  # initialises the grid (allocates its pinned words)
        g.step(2)
        assert np.all(np.isfinite(g.read(rmt.RMT_F_U)))
        g.close()


def test_a_clean_run_reports_nothing():
    g = rmt.Grid(_fixed(S.cavity_sphere(24, precision="fp32")))
    g.step(6)
    assert np.all(np.isfinite(g.read(rmt.RMT_F_U)))
    g.step(1)  # polls the error words of the earlier steps
    g.close()


def test_cycle_cap_gives_enoconverge():
    sc = S.cavity_sphere(24)
    g = rmt.Grid(dict(sc, mg_rtol=1e-14, mg_max_cycles=1))
    with pytest.raises(rmt.RMTError) as ei:
        g.step(1)
    assert ei.value.status == rmt.RMT_ENOCONVERGE
    with pytest.raises(rmt.RMTError) as ei:
        g.step(1)
    assert ei.value.status == rmt.RMT_ESTATE
    g.close()


def test_injected_allocation_failure_gives_enomem():
    g = rmt.Grid(S.cavity_sphere(16))
    g.set_option("inject_alloc", 5)
    with pytest.raises(rmt.RMTError) as ei:
        g.step(1)
    assert ei.value.status == rmt.RMT_ENOMEM
    g.close()


def test_batch_sync_reports_a_diverged_member():
    a = rmt.Grid(_fixed(S.cavity_sphere(24, precision="fp32")))
    b = rmt.Grid(_fixed(S.cavity_sphere(32, precision="fp32")))
    b.set_option("inject_nan_step", 1)
    bt = rmt.Batch()
    bt.add(a)
    bt.add(b)
    bt.step(3)
    with pytest.raises(rmt.RMTError) as ei:
        bt.sync()
    assert ei.value.status == rmt.RMT_EDIVERGED
    bt.close()
    assert np.all(np.isfinite(a.read(rmt.RMT_F_U)))  # the other member is unharmed
    a.close()
    b.close()


def test_server_evicts_a_diverged_job_and_the_others_finish():
    srv = rmt.Server(1 << 34)
    srv.set_option("inject_nan_step", 3)
    bad = srv.submit(_fixed(S.cavity_sphere(24, precision="fp32"), graph=0), 40)
    r, q = srv.poll()  # admits the bad job with the injection
    assert r == 1
    srv.set_option("inject_nan_step", -1)
    good = [srv.submit(_fixed(S.cavity_sphere(n, precision="fp32"), graph=0), 12) for n in (16, 20)]
    for _ in range(2000):
        r, q = srv.poll()
        if r == 0 and q == 0:
            break
    ib = srv.job(bad)
    assert ib["state"] == rmt.RMT_JOB_FAILED and ib["status"] == rmt.RMT_EDIVERGED
    assert ib["steps_done"] < 40  # evicted before its last step
    for j in good:
        inf = srv.job(j)
        assert inf["state"] == rmt.RMT_JOB_DONE and inf["steps_done"] == 12
        assert np.all(np.isfinite(srv.grid(j).read(rmt.RMT_F_U)))
    # the evicted job's memory went back to the budget: only the finished jobs stay resident
    assert srv.resident_bytes() == sum(srv.job(j)["device_bytes"] for j in good)
    srv.close()


def _translated_sphere(precision):
    """A sphere whose reference map puts it 0.42 away from its centre along x, so that its band
    straddles the point half a period from the centre."""
    n = 32
    sc = S._box(n, periodic=True)
    sc.update(precision=precision, dt=0.2 / n)
    c = (0.5, 0.5, 0.5)
    sc["solids"] = [S.solid(S.SPHERE, c, (0.15, 0.15, 0.15))]
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    xi = np.stack([np.mod(X - 0.42, 1.0), Y, Z]).reshape(-1)
    return sc, xi


def test_fp32_band_at_the_image_seam_is_reported():
    sc, xi = _translated_sphere("fp32")
    g = rmt.Grid(sc)
    with pytest.raises(rmt.RMTError) as ei:
        g.write(rmt.RMT_F_XI, xi, 0)
    assert ei.value.status == rmt.RMT_ERANGE
    g.close()
    sc, xi = _translated_sphere("fp64")
    g = rmt.Grid(sc)
    g.write(rmt.RMT_F_XI, xi, 0)  # the FP64 form stores xi itself: no seam
    g.step(1)
    g.close()


def test_fp32_reference_map_round_trip_keeps_the_displacement():
    """A written reference map comes back with the FP32 rounding of its displacement from the cell
    centres, not of the O(1) positions."""
    n = 32
    sc = S._box(n, periodic=True)
    sc.update(precision="fp32", dt=0.2 / n)
    sc["solids"] = [S.solid(S.SPHERE, (0.47, 0.52, 0.5), (0.2, 0.2, 0.2))]
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    d = 1e-3 * np.stack([np.sin(2 * np.pi * Y), np.cos(2 * np.pi * Z), np.sin(2 * np.pi * X)])
    xi = (np.stack([X, Y, Z]) + d).reshape(-1)
    g = rmt.Grid(sc)
    g.write(rmt.RMT_F_XI, xi, 0)
    got = g.read(rmt.RMT_F_XI, 0)
    lay = g.read(rmt.RMT_F_LAYER, 0)
    inside = np.tile(lay == 0, 3)
    err = np.abs(got[inside] - xi[inside]).max()
    assert err <= 1e-3 * 2**-23 * 2  # FP32 rounding of a 1e-3 displacement, not of xi ~ 0.5
    g.close()
