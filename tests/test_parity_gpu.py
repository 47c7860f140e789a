"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Bar: integer outputs (layer labels) bit-exact; FP64 fields within rel-L2 1e-10 per step;
FP32 bulk with two-float refinement of the projections within rel-L2 1e-4 on u and xi after 10
steps."""
import numpy as np
import pytest
from scipy import ndimage

import oracle as O
from paper_2104_00095_gb300 import rmt, scenes as S
from parity_util import compare_state, needs_gpu, pair, rel_l2

# the multigrid schedule bench.py times (5 MAC and 4 FE V-cycles per solve)
BENCH_OPTIONS = {"fe_inner": 4, "mac_inner": 5, "mac_pre": 2, "mac_post": 2, "mac_omega": 1.15, "mac_coarse_pre": 2,
                 "mac_coarse_post": 2, "fe_pre": 2, "fe_post": 1, "fe_omega": 1.0, "graph": 1}
BENCH_CYCLES = {"mg_fixed_cycles": 5, "mg_fixed_cycles_fe": 4}

pytestmark = [pytest.mark.gpu, needs_gpu]

TOL64 = 1e-10


def _small_scenes():
    cav = S.cavity_sphere(32, steps=20)
    settle = S.settling(n=32, nbodies=3, seed=5)
    swim = S.swimmers(n=32, nbodies=2, seed=5, precision="fp64")
    rag = S._box(28, periodic=False, lid=1.0)
    rag.update(n=(20, 24, 28), hi=(20 / 28, 24 / 28, 1.0), dt=0.2 / 28, mu=0.02)
    rag["solids"] = [S.solid(S.ELLIPSOID, (0.36, 0.42, 0.5), (0.17, 0.1, 0.13),
                             S.random_rotation(np.random.default_rng(3)), rho_s=1.2, G=0.3, mu_a=0.02,
                             gamma_t=1.0)]
    return {"cavity32": cav, "settling32": settle, "swimmers32": swim, "ragged20x24x28": rag}


@pytest.mark.parametrize("name", ["cavity32", "settling32", "swimmers32", "ragged20x24x28"])
def test_initialisation_parity(name):
    sc = _small_scenes()[name]
    g, o = pair(sc)
    compare_state(g, o, len(sc["solids"]), 1e-12, tag=name)
    assert abs(g.dt - o.dt) == 0.0


def test_one_step_intermediates_cavity():
    sc = S.cavity_sphere(32)
    g, o = pair(sc)
    g.step(1)
    assert o.step(1) == 0
    for f in (rmt.RMT_F_DIVTAU_N, rmt.RMT_F_UFACE_X, rmt.RMT_F_UFACE_Y, rmt.RMT_F_UFACE_Z, rmt.RMT_F_UMAC_X,
              rmt.RMT_F_UMAC_Y, rmt.RMT_F_UMAC_Z, rmt.RMT_F_MAC_Q, rmt.RMT_F_ADV_U, rmt.RMT_F_DIVTAU_H,
              rmt.RMT_F_RHO_HALF, rmt.RMT_F_USTAR, rmt.RMT_F_PSI):
        e = rel_l2(g.read(f), o.read(f))
        assert e <= TOL64, f"intermediate {f}: rel-L2 {e:.3e}"
    e = rel_l2(g.read(rmt.RMT_F_XI_HALF, 0), o.read(O.F_XI_HALF, 0))
    assert e <= TOL64
    compare_state(g, o, 1, TOL64, tag="step 1")


@pytest.mark.parametrize("name,steps", [("cavity32", 20), ("settling32", 6), ("swimmers32", 6),
                                        ("ragged20x24x28", 5)])
def test_multistep_parity_fp64(name, steps):
    sc = _small_scenes()[name]
    g, o = pair(sc)
    for s in range(steps):
        g.step(1)
        assert o.step(1) == 0, o.error()
        compare_state(g, o, len(sc["solids"]), TOL64, tag=f"{name} step {s + 1}")


def test_pure_fluid_cavity_parity():
    sc = S._box(24, periodic=False, lid=1.0)
    sc.update(dt=0.2 / 24)
    g, o = pair(sc)
    for s in range(5):
        g.step(1)
        assert o.step(1) == 0
        compare_state(g, o, 0, TOL64, tag=f"fluid step {s + 1}")


@pytest.mark.parametrize("sweep", [1, 2])
def test_fp32_bulk_within_1e4_after_10_steps(sweep):
    """sweep 2 runs the fused red-black pass on every MAC level of the 32^3 cavity (32 down to 4,
    no-slip walls on every side); sweep 1 leaves these small levels to one pass per colour."""
    sc = S.cavity_sphere(32, precision="fp32")
    sc64 = dict(sc, precision="fp64")
    g = rmt.Grid(dict(sc, mg_rtol=1e-10, mg_max_cycles=200, options={"mac_sweep": sweep}))
    o = O.Oracle(sc64)
    g.step(10)
    assert o.step(10) == 0
    eu = rel_l2(g.read(rmt.RMT_F_U), o.read(O.F_U))
    xg, xo = g.read(rmt.RMT_F_XI, 0), o.read(O.F_XI, 0)
    both = np.isfinite(xg) & np.isfinite(xo)
    ex = np.linalg.norm(xg[both] - xo[both]) / np.linalg.norm(xo[both])
    # band presence may differ only on a thin shell where phi is within float rounding of zero
    assert np.count_nonzero(np.isfinite(xg) != np.isfinite(xo)) <= 0.01 * both.sum()
    assert eu <= 1e-4, eu
    assert ex <= 1e-4, ex


def _periodic_taylor_green(n, precision):
    """Triply periodic unit box without bodies, started from the 3-D Taylor-Green field
    u = (sin X cos Y cos Z, -cos X sin Y cos Z, 0), X = 2 pi x (divergence-free)."""
    sc = S._box(n, periodic=True)
    sc.update(mu=0.01, dt=0.2 / n, precision=precision)
    x = (np.arange(n) + 0.5) / n * 2 * np.pi
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = np.zeros((3, n, n, n))
    u[0] = np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -np.cos(X) * np.sin(Y) * np.cos(Z)
    return sc, u.reshape(-1)


def test_fp32_periodic_fluid_matches_fp64_oracle():
    """The FP32 form on a triply periodic grid, where the FE smoother and residual stage 16-byte
    rows and (mac_sweep 2) every MAC level runs the fused red-black pass, against the FP64 oracle
    after 10 steps of a Taylor-Green flow: without bodies the only FP32 error is rounding."""
    sc, u0 = _periodic_taylor_green(32, "fp32")
    g = rmt.Grid(dict(sc, mg_rtol=1e-10, mg_max_cycles=200, options={"mac_sweep": 2}))
    o = O.Oracle(dict(sc, precision="fp64"))
    g.write(rmt.RMT_F_U, u0)
    o.write(O.F_U, u0)
    g.step(10)
    assert o.step(10) == 0
    eu = rel_l2(g.read(rmt.RMT_F_U), o.read(O.F_U))
    ep = rel_l2(g.read(rmt.RMT_F_P), o.read(O.F_P))
    assert eu <= 1e-4, (eu, ep)
    assert ep <= 1e-3, (eu, ep)


def _fp32_against_oracle(sc, steps=10):
    """Relative L2 error of u and of every body's xi (cells holding xi on both paths) of the FP32
    form against the FP64 oracle after `steps` steps; band presence may differ only on a thin
    shell where phi is within float rounding of zero."""
    g = rmt.Grid(dict(sc, precision="fp32", mg_rtol=1e-10, mg_max_cycles=200, options={"mac_sweep": 2}))
    o = O.Oracle(dict(sc, precision="fp64", mg_rtol=1e-13, mg_max_cycles=200))
    g.step(steps)
    assert o.step(steps) == 0, o.error()
    eu = rel_l2(g.read(rmt.RMT_F_U), o.read(O.F_U))
    exs = []
    for m in range(len(sc["solids"])):
        xg, xo = g.read(rmt.RMT_F_XI, m), o.read(O.F_XI, m)
        both = np.isfinite(xg) & np.isfinite(xo)
        assert np.count_nonzero(np.isfinite(xg) != np.isfinite(xo)) <= 0.01 * both.sum()
        exs.append(np.linalg.norm(xg[both] - xo[both]) / np.linalg.norm(xo[both]))
    g.close()
    return eu, max(exs)


def test_fp32_swimmers_within_1e4_of_the_fp64_oracle():
    """The FP32 form on the swimmer scene (2 active ellipsoids, 32^3) after 10 steps.  Reference
    maps are stored as displacements from the cell centres, so FP32 rounding no longer enters
    the elastic stress at the level of O(1) positions (measured 4e-7 on u)."""
    eu, ex = _fp32_against_oracle(S.swimmers(n=32, nbodies=2, seed=5))
    assert eu <= 1e-4, (eu, ex)
    assert ex <= 1e-4, (eu, ex)


def test_fp32_swimmer_scene_64_eight_bodies_within_1e4():
    """The benchmark's swimmer scene (8 active ellipsoids, seed of the 256^3 scene) on a 64^3
    copy, FP32 against the FP64 oracle after 10 steps."""
    eu, ex = _fp32_against_oracle(S.swimmers(n=64, nbodies=8))
    assert eu <= 1e-4, (eu, ex)
    assert ex <= 1e-4, (eu, ex)


def test_fp32_settling_within_1e4():
    """The settling mixture (heavy and buoyant ellipsoids under gravity between no-slip walls) on
    a 48^3 copy with the 10 bodies that fit at this resolution, FP32 against the FP64 oracle after
    10 steps."""
    eu, ex = _fp32_against_oracle(S.settling(n=48, nbodies=10))
    assert eu <= 1e-4, (eu, ex)
    assert ex <= 1e-4, (eu, ex)


def _ragged_walls_fp32():
    sc = S._box(64, periodic=False, lid=1.0)
    sc.update(n=(68, 60, 64), hi=(68 / 64, 60 / 64, 1.0), dt=0.2 / 64, mu=0.01, precision="fp32")
    sc["solids"] = [S.solid(S.ELLIPSOID, (0.5, 0.45, 0.5), (0.2, 0.12, 0.15),
                            S.random_rotation(np.random.default_rng(4)), rho_s=1.3, G=0.4, mu_a=0.01)]
    return sc


@pytest.mark.parametrize("name,sweep", [("cavity128", 1), ("swimmers128", 1), ("ragged68x60x64", 2)])
def test_fused_sweep_matches_colour_passes(name, sweep):
    """The fused red-black pass (both colours per launch, out of place, z-chunked tiles with a
    recomputed first-colour ring) against one in-place pass per colour, on the fixed-cycle FP32
    schedule of the bench: no-slip walls on every side (cavity), a triply periodic box
    (swimmers), and walls with partial tiles along x and y (68 x 60 x 64).  The two compute the
    same sweep with the same operations; only the compiler's contraction of products into FMAs
    may differ, so the results agree far below the FP32 bar."""
    if name == "cavity128":
        sc = S.cavity_sphere(128, precision="fp32")
    elif name == "swimmers128":
        sc = S.swimmers(n=128, nbodies=2, seed=7, precision="fp32")
    else:
        sc = _ragged_walls_fp32()

    def run(mode):
        g = rmt.Grid(dict(sc, **BENCH_CYCLES, options=dict(BENCH_OPTIONS, mac_sweep=mode)))
        g.step(3)
        out = [g.read(f) for f in (rmt.RMT_F_U, rmt.RMT_F_P, rmt.RMT_F_RHO)]
        g.close()
        return out

    ref, fused = run(0), run(sweep)
    for a, b in zip(fused, ref):
        assert np.all(np.isfinite(a))
        assert rel_l2(a, b) <= 1e-6, rel_l2(a, b)


def test_runs_are_bit_identical():
    sc = S.settling(n=32, nbodies=3, seed=5)
    a, b = rmt.Grid(sc), rmt.Grid(sc)
    a.step(3)
    b.step(3)
    for f in (rmt.RMT_F_U, rmt.RMT_F_P, rmt.RMT_F_RHO):
        assert np.array_equal(a.read(f), b.read(f))
    for m in range(3):
        assert np.array_equal(a.read(rmt.RMT_F_XI, m), b.read(rmt.RMT_F_XI, m), equal_nan=True)


def test_degenerate_extrapolation_is_reported_on_both_paths():
    """A sphere holding one interior cell leaves every layer-1 fit with a single data point."""
    n = 16
    sc = S._box(n, periodic=False)
    sc.update(dt=0.2 / n)
    sc["solids"] = [S.solid(S.SPHERE, ((8 + 0.5) / n,) * 3, (0.6 / n,) * 3)]
    o = O.Oracle(sc)
    assert o.step(0) == 8  # RMT_EDEGENERATE
    with pytest.raises(rmt.RMTError) as ei:
        g = rmt.Grid(sc)
        g.step(0)
    assert ei.value.status == rmt.RMT_EDEGENERATE


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_uniform_translation_is_exact(prec, tol):
    """Periodic box, uniform velocity, unstressed sphere: xi = x - U t and u = U stay exact."""
    n = 32
    U = np.array([0.3, -0.2, 0.1])
    sc = S._box(n, periodic=True)
    sc.update(dt=0.2 / n, precision=prec)
    sc["solids"] = [S.solid(S.SPHERE, (0.5, 0.5, 0.5), (0.2,) * 3, rho_s=1.0, G=0.4)]
    g = rmt.Grid(sc)
    g.write(rmt.RMT_F_U, np.repeat(U, n**3))
    g.step(5)
    u = g.read(rmt.RMT_F_U).reshape(3, -1)
    assert np.max(np.abs(u - U[:, None])) < tol * 10
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    P = np.stack([X, Y, Z]).reshape(3, -1)
    xi = g.read(rmt.RMT_F_XI, 0).reshape(3, -1)
    ok = np.isfinite(xi[0])
    d = xi[:, ok] - (P[:, ok] - U[:, None] * 5 * 0.2 / n)
    d -= np.round(d)
    assert np.max(np.abs(d)) < tol


# ------------------------------------------------------------------ full-size properties
def _taxicab_layers_local(lay, per, L):
    """Brute-force layer labels from the layer-0 mask of lay, on a box around the band
    (periodic axes wrapped by index arithmetic)."""
    nz, ny, nx = lay.shape
    idx = np.argwhere(lay >= 0)
    out = {}
    lo, hi = idx.min(0) - (L + 2), idx.max(0) + (L + 3)
    rng = [np.arange(lo[a], hi[a]) for a in range(3)]
    sub_ok = True
    for a, n in enumerate((nz, ny, nx)):
        if not per:
            rng[a] = np.clip(rng[a], 0, n - 1)
            rng[a] = np.unique(rng[a])
        else:
            rng[a] = rng[a] % n
            if len(np.unique(rng[a])) < len(rng[a]):
                sub_ok = False
    if not sub_ok:
        return None
    sub = lay[np.ix_(rng[0], rng[1], rng[2])]
    d = ndimage.distance_transform_cdt(sub != 0, metric="taxicab")
    ref = np.where(d <= L, d, -1)
    return sub, ref


@pytest.mark.parametrize("cfg", ["swimmers256_fp32", "settling128_fp64"])
def test_full_size_properties(cfg):
    if cfg == "swimmers256_fp32":
        sc = S.swimmers(n=256, steps=1)
        # the launch configuration bench.py times
        sc.update(BENCH_CYCLES, options=BENCH_OPTIONS)
        xtol = 1e-6  # FP32 fits of an affine map: a few units in the last place of x ~ O(1)
    else:
        sc = S.settling(n=128, steps=1)
        sc.update(mg_rtol=1e-12)
        xtol = 1e-12
    n = sc["n"][0]
    per = sc["bc"][0] == S.PERIODIC
    g = rmt.Grid(sc)
    # initialisation: the extrapolated reference map of an undeformed body is x itself
    x = (np.arange(n) + 0.5) / n
    for m in range(len(sc["solids"])):
        lay = g.read(rmt.RMT_F_LAYER, m).reshape(n, n, n).astype(int)
        r = _taxicab_layers_local(lay, per, sc["band_layers"])
        if r is not None:
            sub, ref = r
            assert np.array_equal(sub, ref), f"body {m}: layer labels differ from the taxicab distance"
        xi = g.read(rmt.RMT_F_XI, m).reshape(3, n, n, n)
        band = lay >= 1
        c = np.asarray(sc["solids"][m]["center"])
        for a, ax in enumerate((2, 1, 0)):
            coord = np.broadcast_to(x.reshape([-1 if q == ax else 1 for q in range(3)]), (n, n, n))
            dd = xi[a][band] - coord[band]
            if per:
                dd -= np.round(dd)
            assert np.max(np.abs(dd)) < xtol * 10, f"body {m} comp {a}"
    g.step(1)
    # the MAC-projected face velocities are discretely divergence-free
    um = [g.read(f) for f in (rmt.RMT_F_UMAC_X, rmt.RMT_F_UMAC_Y, rmt.RMT_F_UMAC_Z)]
    div = (np.diff(um[0].reshape(n, n, n + 1), axis=2) + np.diff(um[1].reshape(n, n + 1, n), axis=1) +
           np.diff(um[2].reshape(n + 1, n, n), axis=0)) * n
    scale = max(np.abs(u).max() for u in um) * n
    assert np.max(np.abs(div)) <= (1e-4 if sc["precision"] == "fp32" else 1e-9) * max(scale, 1e-30)
    for f in (rmt.RMT_F_U, rmt.RMT_F_P, rmt.RMT_F_RHO):
        assert np.all(np.isfinite(g.read(f)))


@pytest.mark.parametrize("n,prec", [(44, "fp64"), (112, "fp32")])
def test_uneven_multigrid_hierarchies(n, prec):
    """Periodic sizes whose hierarchy reaches odd levels: 44 -> 22 -> 11 and 112 -> 56 -> 28 ->
    14 -> 7, where the MAC smoother switches to Jacobi sweeps (an odd periodic side has no
    consistent red-black colouring; the finest level itself must have even periodic sides, which
    rmt_create_grid checks)."""
    sc = S.swimmers(n=n, nbodies=1, seed=21, precision=prec)
    g = rmt.Grid(sc)
    if prec == "fp64":
        o = O.Oracle(sc)
        g.step(1)
        assert o.step(1) == 0
        compare_state(g, o, 1, TOL64, tag=f"n={n}")
    else:
        g.step(2)
        um = [g.read(f) for f in (rmt.RMT_F_UMAC_X, rmt.RMT_F_UMAC_Y, rmt.RMT_F_UMAC_Z)]
        div = (np.diff(um[0].reshape(n, n, n + 1), axis=2) + np.diff(um[1].reshape(n, n + 1, n), axis=1) +
               np.diff(um[2].reshape(n + 1, n, n), axis=0)) * n
        assert np.max(np.abs(div)) <= 1e-4 * max(np.abs(u).max() for u in um) * n
        assert np.all(np.isfinite(g.read(rmt.RMT_F_U)))


@pytest.mark.parametrize("scene", ["swimmers64", "swimmers256", "settling128"])
def test_bench_cycle_counts_stay_close_to_the_converged_solve(scene):
    """The fixed-cycle configuration that bench.py times (5 MAC cycles after one two-float
    residual, 2 red-black sweeps each way over-relaxed by 1.15 on the finest level and 2 on the
    others, 4 FE cycles after one two-float residual with 2 + 1 Jacobi sweeps of weight 1) against
    adaptive solves to 1e-9, after 6 and 12 steps in FP32:
    the swimmer scene on a small copy and on the benchmark's own 256^3 grid (an FP32 V-cycle's
    accuracy on smooth modes falls with n, so the small case alone does not cover the
    benchmark), and the settling mixture between no-slip walls."""
    if scene == "swimmers64":
        mk = lambda: S.swimmers(n=64, nbodies=2, seed=13, precision="fp32")
    elif scene == "swimmers256":
        mk = lambda: S.swimmers(n=256, nbodies=8, seed=1003, precision="fp32")
    else:
        mk = lambda: S.settling(n=128, precision="fp32")

    def run(**kw):
        sc = mk()
        sc.update(kw)
        g = rmt.Grid(sc)
        out = []
        for _ in range(2):
            g.step(6)
            out.append((g.read(rmt.RMT_F_U), g.read(rmt.RMT_F_P)))
        g.close()
        return out
    ref = run(mg_rtol=1e-9, mg_max_cycles=60, options={"fe_inner": 2})
    got = run(**BENCH_CYCLES, options=BENCH_OPTIONS)
    for (u, p), (u_ref, p_ref) in zip(got, ref):
        assert rel_l2(u, u_ref) <= 1e-5
        assert rel_l2(p - p.mean(), p_ref - p_ref.mean()) <= 1e-5


@pytest.mark.parametrize("dw_cells", [0.0, 2.0])
def test_wall_repulsion_parity(dw_cells):
    """A sphere close to the bottom wall with wall repulsion (SI "Contact with a wall"): state
    and repulsion field against the oracle, step by step."""
    n = 24
    h = 1.0 / n
    sc = S._box(n, periodic=False)
    sc.update(dt=0.1 * h, wall_dw=dw_cells * h, gravity=(0.0, 0.0, -1.0))
    sc["solids"] = [S.solid(S.SPHERE, (0.5, 0.45, 0.2 + 0.3 * h), (0.2,) * 3, rho_s=1.5, G=0.3, rep_A=12.0)]
    g, o = pair(sc)
    for s in range(4):
        g.step(1)
        assert o.step(1) == 0, o.error()
        compare_state(g, o, 1, TOL64, tag=f"repulsion step {s + 1}")
        ar, ao = g.read(rmt.RMT_F_REPULSION), o.read(O.F_REPULSION)
        assert np.count_nonzero(ao) > 0
        assert np.array_equal(ar != 0, ao != 0)
        assert rel_l2(ar, ao) <= TOL64


def test_initial_pressure_iterations_parity():
    """SI "Initialization" item 2 on both paths: same iteration count, same pressure, and the
    steps after it stay in parity."""
    sc = S.cavity_sphere(24)
    g, o = pair(sc)
    it_g = g.init_pressure(8, 1e-4)
    rc, it_o = o.init_pressure(8, 1e-4)
    assert rc == 0 and it_g == it_o >= 2
    assert rel_l2(g.read(rmt.RMT_F_P), o.read(O.F_P)) <= TOL64
    compare_state(g, o, 1, TOL64, tag="after the initial pressure iterations")
    for s in range(2):
        g.step(1)
        assert o.step(1) == 0
        compare_state(g, o, 1, TOL64, tag=f"step {s + 1} after them")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_body_stats_parity(prec):
    """Body diagnostics (main text "Swimming"; SI "Swimming statistics"; SI "Pre-stretched
    sphere", eq. elas) of every active body after a few steps against the oracle's.  FP64: the
    two states are in parity.  FP32: the GPU state (u and each body's xi) is written into the
    oracle first, so both evaluate the diagnostics on the same FP32 state (the oracle
    re-extrapolates the band of the written xi in FP64)."""
    sc = S.swimmers(n=32, nbodies=2, seed=5, precision=prec)
    g, o = pair(sc)
    g.step(3)
    assert o.step(3) == 0
    assert o.write(O.F_U, g.read(rmt.RMT_F_U)) == 0
    if prec == "fp32":
        for m in range(len(sc["solids"])):
            assert o.write(O.F_XI, g.read(rmt.RMT_F_XI, m), m) == 0
    for m in range(len(sc["solids"])):
        a, b = g.body_stats(m), o.body_stats(m)
        assert a.shape == (7,) and np.all(np.isfinite(a))
        assert b[3] != 0.0 and b[4] > 0.0 and b[5] > 0.0 and b[6] > 0.0
        if prec == "fp64":
            np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-12 * np.abs(b[:5]).max())
        else:
            # xi is stored to ~1e-7 absolute, so centred differences of it over 2h carry ~3e-6:
            # J and the (second-order small) elastic energy are compared to that resolution
            uscale = np.abs(g.read(rmt.RMT_F_U)).max()
            np.testing.assert_allclose(a[:3], b[:3], rtol=0, atol=1e-6 * uscale)
            np.testing.assert_allclose(a[3:5], b[3:5], rtol=1e-3)
            assert abs(a[6] - b[6]) <= 1e-5
            assert abs(a[5] - b[5]) <= 2e-2 * b[5]
    # deterministic: the same call twice gives the same bits
    assert np.array_equal(g.body_stats(0), g.body_stats(0))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_float_field_io_matches_the_fp64_calls(precision):
    """rmt_read_fields_float / rmt_write_fields_float against the FP64 calls: reads are the FP64
    values rounded to float (exact for u and p of an FP32 grid, which are stored as floats; xi of
    a body goes through the conversion path), and a step after writing u as floats equals the
    step after writing the same values through the FP64 call, bit for bit."""
    import torch

    sc = S.swimmers(n=32, nbodies=2, seed=5, precision=precision)
    a, b = rmt.Grid(sc), rmt.Grid(sc)
    a.step(2)
    b.step(2)
    for f in (rmt.RMT_F_U, rmt.RMT_F_P, rmt.RMT_F_RHO):
        ref = a.read(f)
        got = a.read_float(f)
        assert got.dtype == np.float32 and np.array_equal(got, ref.astype(np.float32)), f
        if precision == "fp32" and f != rmt.RMT_F_RHO:
            assert np.array_equal(got.astype(np.float64), ref), f  # stored as floats: no rounding
    xi = a.read(rmt.RMT_F_XI, 1)
    xf = a.read_float(rmt.RMT_F_XI, 1)
    assert np.array_equal(np.isnan(xf), np.isnan(xi))
    ok = ~np.isnan(xi)
    assert np.array_equal(xf[ok], xi[ok].astype(np.float32))
    # device destination
    d = torch.empty(a.field_len(rmt.RMT_F_U), dtype=torch.float32, device="cuda")
    a.read_float_ptr(rmt.RMT_F_U, d.data_ptr(), d.numel() * 4, 1)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), a.read_float(rmt.RMT_F_U))
    # the same new velocity written both ways
    u = (a.read(rmt.RMT_F_U) * 0.9).astype(np.float32)
    a.write_float(rmt.RMT_F_U, u)
    b.write(rmt.RMT_F_U, u.astype(np.float64))
    assert np.array_equal(a.read(rmt.RMT_F_U), b.read(rmt.RMT_F_U))
    a.step(1)
    b.step(1)
    for f in (rmt.RMT_F_U, rmt.RMT_F_P):
        assert np.array_equal(a.read(f), b.read(f)), f
    # from page-locked memory the write stays asynchronous; the next step is ordered after it
    pin = torch.from_numpy(u * np.float32(1.1)).pin_memory()
    a.write_float_ptr(rmt.RMT_F_U, pin.data_ptr(), pin.numel() * 4, 0)
    b.write(rmt.RMT_F_U, pin.numpy().astype(np.float64))
    a.step(1)
    b.step(1)
    for f in (rmt.RMT_F_U, rmt.RMT_F_P):
        assert np.array_equal(a.read(f), b.read(f)), f
    with pytest.raises(rmt.RMTError):
        a.write_float(rmt.RMT_F_U, u[:-1])
    a.close()
    b.close()

