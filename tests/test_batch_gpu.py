"""Graph-captured steps, batches and the serving runtime: every result is the same as the grid
stepped alone (bit for bit: members share no data and every kernel is deterministic), the
footprint model equals what a grid allocates, and the server keeps to its budget."""
import numpy as np
import pytest

from paper_2104_00095_gb300 import rmt, scenes as S
from parity_util import needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]

FIELDS = (rmt.RMT_F_U, rmt.RMT_F_P, rmt.RMT_F_RHO)


def _fixed(sc, mac=4, fe=3):
    return dict(sc, mg_fixed_cycles=mac, mg_fixed_cycles_fe=fe)


def _same(a: rmt.Grid, b: rmt.Grid, tag=""):
    for f in FIELDS:
        assert np.array_equal(a.read(f), b.read(f)), f"{tag} field {f}"
    for m in range(len(a.scene.get("solids", []))):
        for f in (rmt.RMT_F_XI, rmt.RMT_F_LAYER):
            assert np.array_equal(a.read(f, m), b.read(f, m), equal_nan=True), f"{tag} body {m} field {f}"


def _mix():
    a = S.cavity_sphere(24, precision="fp32")
    b = S.swimmers(n=32, nbodies=2, seed=7, precision="fp32")
    c = S.settling(n=28, nbodies=2, seed=9, precision="fp64")
    d = S._box(20, periodic=False, lid=1.0)
    d.update(dt=0.2 / 20, precision="fp32")
    return [_fixed(x) for x in (a, b, c, d)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_step_equals_eager(prec):
    sc = _fixed(S.swimmers(n=32, nbodies=2, seed=5, precision=prec))
    eager = rmt.Grid(sc)
    graph = rmt.Grid(dict(sc, options={"graph": 1}))
    l0 = rmt.kernel_launches()
    eager.step(5)
    l1 = rmt.kernel_launches()
    graph.step(5)
    l2 = rmt.kernel_launches()
    _same(eager, graph, prec)
    assert l2 - l1 == l1 - l0  # a replayed graph counts its kernel nodes


def test_batch_equals_alone():
    scenes = _mix()
    alone = [rmt.Grid(s) for s in scenes]
    for g in alone:
        g.step(6)
    members = [rmt.Grid(s) for s in scenes]
    b = rmt.Batch()
    for g in members:
        b.add(g)
    b.step(4)
    # a member cannot be stepped on its own while in the batch
    with pytest.raises(rmt.RMTError) as ei:
        members[0].step(1)
    assert ei.value.status == rmt.RMT_ESTATE
    b.step(2)
    b.sync()
    for k, (a, m) in enumerate(zip(alone, members)):
        _same(a, m, f"member {k}")
    # leaving the batch: the grid carries on alone, still in step with its twin
    b.remove(members[1])
    members[1].step(2)
    alone[1].step(2)
    _same(alone[1], members[1], "after leaving")
    b.close()


def test_footprint_equals_allocation():
    for sc in _mix() + [S.cavity_sphere(16)]:
        g = rmt.Grid(sc)
        g.read(rmt.RMT_F_RHO)  # initialises
        assert g.device_bytes() == rmt.footprint(sc), sc["n"]


def test_server_mix_matches_alone_within_budget():
    scenes = _mix()
    steps = [7, 3, 5, 4]
    fp = [rmt.footprint(s) for s in scenes]
    budget = max(fp) + min(fp)  # never room for all: jobs must wait for memory
    srv = rmt.Server(budget)
    ids = [srv.submit(s, n) for s, n in zip(scenes, steps)]
    peak = 0
    for _ in range(10000):
        r, q = srv.poll()
        peak = max(peak, srv.resident_bytes())
        # finished jobs are released after their check below, freeing memory for the queue
        for i in [i for i in ids if i in srv.scenes]:
            inf = srv.job(i)
            if inf["state"] == rmt.RMT_JOB_DONE:
                sc = srv.scenes[i]
                twin = rmt.Grid(sc)
                twin.step(inf["steps_total"])
                _same(twin, srv.grid(i), f"job {i}")
                assert inf["t_submit"] <= inf["t_admit"] <= inf["t_done"]
                srv.release(i)
        if r == 0 and q == 0 and not srv.scenes:
            break
    assert peak <= budget
    for i in ids:
        with pytest.raises(rmt.RMTError):
            srv.job(i)  # released
    assert srv.cell_steps() == sum(np.prod(s["n"]) * n for s, n in zip(scenes, steps))
    srv.close()


def test_server_failed_job_does_not_stop_the_others():
    n = 16
    bad = S._box(n, periodic=False)
    bad.update(dt=0.2 / n)
    bad["solids"] = [S.solid(S.SPHERE, ((8 + 0.5) / n,) * 3, (0.6 / n,) * 3)]  # a one-cell body
    good = S.cavity_sphere(20)
    srv = rmt.Server(1 << 34)
    jb = srv.submit(_fixed(bad), 2)
    jg = srv.submit(_fixed(good), 3)
    for _ in range(1000):
        r, q = srv.poll()
        if r == 0 and q == 0:
            break
    ib, ig = srv.job(jb), srv.job(jg)
    assert ib["state"] == rmt.RMT_JOB_FAILED and ib["status"] == rmt.RMT_EDEGENERATE
    assert ig["state"] == rmt.RMT_JOB_DONE and ig["steps_done"] == 3
    srv.close()


def test_autotune_picks_a_schedule_that_meets_the_tolerance():
    sc = S.swimmers(n=64, nbodies=2, seed=11, precision="fp32")
    g = rmt.Grid(sc)
    with pytest.raises(rmt.RMTError) as ei:
        g.autotune(1e-6)  # needs a step's right-hand sides
    assert ei.value.status == rmt.RMT_ESTATE
    g.step(1)
    r = g.autotune(1e-6)
    assert r["mac_cycles"] >= 1 and r["fe_cycles"] >= 1 and r["mac_block"] in (1, 2, 4, 8)
    assert r["trials"] >= 96 + 81  # sweeps x relaxation x inner cycles, per solver
    assert r["mac_omega"] in (1.0, 1.15)
    # the tuned grid now steps fixed-cycle; the same options set by hand give the same result
    twin = rmt.Grid(sc)
    twin.step(1)
    for k in ("mac_pre", "mac_post", "mac_inner", "mac_block", "mac_cycles", "mac_zchunk", "fe_zchunk", "fe_pre",
              "fe_post", "fe_inner", "fe_block", "fe_omega", "fe_cycles", "mac_omega"):
        twin.set_option(k, r[k])
    g.step(2)
    twin.step(2)
    _same(g, twin, "tuned")
    n = sc["n"][0]
    um = [g.read(f) for f in (rmt.RMT_F_UMAC_X, rmt.RMT_F_UMAC_Y, rmt.RMT_F_UMAC_Z)]
    div = (np.diff(um[0].reshape(n, n, n + 1), axis=2) + np.diff(um[1].reshape(n, n + 1, n), axis=1) +
           np.diff(um[2].reshape(n + 1, n, n), axis=0)) * n
    assert np.max(np.abs(div)) <= 1e-4 * max(np.abs(u).max() for u in um) * n


def test_tile_z_chunks_do_not_change_the_result():
    """The z-chunk length of the plane-marching tiles (fused red-black sweep, FE tiles) only
    changes how the planes are split among blocks: a block recomputes the first-colour ring of its
    chunk's lower boundary with the same arithmetic, so every chunking gives the same bits."""
    sc = S.swimmers(n=128, nbodies=2, seed=7, precision="fp32")

    def run(mz, fz):
        g = rmt.Grid(dict(sc, mg_fixed_cycles=4, mg_fixed_cycles_fe=4,
                          options={"graph": 1, "mac_sweep": 2, "mac_zchunk": mz, "fe_zchunk": fz}))
        g.step(2)
        out = [g.read(f) for f in (rmt.RMT_F_U, rmt.RMT_F_P)]
        g.close()
        return out

    ref = run(0, 0)
    for mz, fz in ((16, 8), (48, 64)):
        for a, b in zip(run(mz, fz), ref):
            assert np.array_equal(a, b)
