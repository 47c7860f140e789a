"""Physics validation of the GPU path beyond parity (SI "Pre-stretched sphere"; main text
"Settling sphere in a square cylinder" with Stokes' law): scaling, convergence under grid
refinement, relaxation and settling speed, measured with the body diagnostics."""
import math

import numpy as np
import pytest

from paper_2104_00095_gb300 import rmt, scenes as S
from parity_util import needs_gpu

pytestmark = [pytest.mark.gpu, needs_gpu]

LAM = 1.21  # the SI text's pre-stretch


def _prestretched(n, case, dt, precision="fp64"):
    sc = S.prestretched_sphere(n, case, dt=dt, precision=precision)
    sc.update(mg_rtol=1e-12 if precision == "fp64" else 1e-9, mg_max_cycles=200)
    g = rmt.Grid(sc)
    g.write(rmt.RMT_F_XI, S.prestretch_xi(sc, LAM), 0)
    return g


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_prestretched_sphere_scaling_is_exact(prec):
    """Table str_params cases A1 and A2 share R and gamma = R sqrt(rho G) / mu: with A1's step
    twice A2's, u scales by 1/2 and p and every stress by 1/4, all powers of two, so the two
    runs agree bit for bit under that scaling, energy curve E / E_0 included (the collapse the
    SI reports for these two cases, made exact)."""
    h = 1.0 / 32
    g2 = _prestretched(32, "A2", 0.1 * h, prec)
    g1 = _prestretched(32, "A1", 0.2 * h, prec)
    e1, e2 = [g1.body_stats(0)[5]], [g2.body_stats(0)[5]]
    for _ in range(4):
        g1.step(5)
        g2.step(5)
        e1.append(g1.body_stats(0)[5])
        e2.append(g2.body_stats(0)[5])
    u1, u2 = g1.read(rmt.RMT_F_U), g2.read(rmt.RMT_F_U)
    assert np.abs(u2).max() > 1e-3
    assert np.array_equal(2 * u1, u2)
    assert np.array_equal(4 * g1.read(rmt.RMT_F_P), g2.read(rmt.RMT_F_P))
    assert np.array_equal(g1.read(rmt.RMT_F_XI, 0), g2.read(rmt.RMT_F_XI, 0), equal_nan=True)
    assert np.array_equal(4 * np.array(e1), np.array(e2))
    assert np.all(np.diff(e2) < 0)  # relaxing


def _relax(n, T=0.2):
    """Case A2 from rest to time T; dt = T / steps within the step limits of the scheme."""
    h = 1.0 / n
    mu, _, _, G = S.STR_PARAMS["A2"]
    steps = math.ceil(T / min(0.2 * h, 0.8 * h * h / (6 * mu), 0.5 * h / math.sqrt(G)))
    g = _prestretched(n, "A2", T / steps)
    s0 = g.body_stats(0)
    E = [s0[5]]
    for _ in range(4):
        g.step(steps // 4)
        E.append(g.body_stats(0)[5])
    if steps % 4:
        g.step(steps % 4)
        E.append(g.body_stats(0)[5])
    return s0, g.body_stats(0), np.array(E)


def test_prestretched_sphere_relaxes_and_converges():
    """Case A2 (R = 0.2, G = 1, mu = 0.01; SI "Pre-stretched sphere" item 1) up to T = 0.2:
    the initial energy is the closed form of eq. elas for the uniform stretch; the sphere
    relaxes towards its rest shape over the first quarter of an oscillation (tau_osc = R
    sqrt(rho / G) = 0.2), so the energy falls monotonically to a small fraction of E_0; and the
    volume change, ||J - 1|| and the energy at T shrink as h is refined (the SI reports orders
    1.44 and 1.04 for the first two)."""
    res = {n: _relax(n) for n in (32, 48, 64)}
    dv, jn, eT = {}, {}, {}
    for n, (s0, s1, E) in res.items():
        phi_el = 0.5 * 1.0 * (LAM ** 2 + 2 / LAM - 3)
        assert s0[5] == pytest.approx(phi_el * s0[4], rel=1e-9)
        assert s0[6] < 1e-9
        assert np.all(np.diff(E) < 0)
        assert E[-1] < 0.02 * E[0]
        dv[n] = abs(s1[4] / s0[4] - 1)
        jn[n], eT[n] = s1[6], s1[5]
        assert dv[n] < 2e-3
    assert dv[32] > dv[48] > dv[64]
    assert jn[32] > jn[48] > jn[64]
    assert abs(eT[32] - eT[64]) > abs(eT[48] - eT[64])


def test_prestretched_sphere_convergence_rates():
    """Case A2 at T = 0.2 on 32^3 ... 128^3 (SI "Pre-stretched sphere", Fig. str_conv): both
    measures vanish for the exact solution, so their values are the errors, fitted as B h^s over the
    five grids.  The SI reports s = 1.44 for the volume and 1.04 for ||J - 1||; this scheme gives
    about 1.1 and 0.8 (the readings of the paper it takes differ from the paper's own code in the
    projection and the extrapolation details).  The windows exclude a stalled (s ~ 0) and a
    second-order (s ~ 2) behaviour."""
    ns = (32, 48, 64, 96, 128)
    res = {n: _relax(n) for n in ns}
    h = np.array([1.0 / n for n in ns])
    dv = np.array([abs(res[n][1][4] / res[n][0][4] - 1) for n in ns])
    jn = np.array([res[n][1][6] for n in ns])
    s_v = np.polyfit(np.log(h), np.log(dv), 1)[0]
    s_j = np.polyfit(np.log(h), np.log(jn), 1)[0]
    assert 0.9 < s_v < 1.8, (s_v, dv)
    assert 0.65 < s_j < 1.3, (s_j, jn)


def _released(case, n=64, periods=2.5):
    """E(t) / E_0 of a Table str_params case released from the pre-stretch, sampled every few
    steps up to `periods` oscillation times tau_osc = R sqrt(rho_s / G)."""
    mu, rs, R, G = S.STR_PARAMS[case]
    tau_osc = R * math.sqrt(rs / G)
    sc = S.prestretched_sphere(n, case)
    sc.update(mg_fixed_cycles=6, mg_fixed_cycles_fe=6, options={"graph": 1})
    g = rmt.Grid(sc)
    g.write(rmt.RMT_F_XI, S.prestretch_xi(sc, LAM), 0)
    nsteps = int(math.ceil(periods * tau_osc / g.dt))
    every = max(1, nsteps // 160)
    t, E = [0.0], [g.body_stats(0)[5]]
    k = 0
    while k < nsteps:
        g.step(every)
        k += every
        t.append(k * g.dt)
        E.append(g.body_stats(0)[5])
    g.close()
    return np.array(t) / tau_osc, np.array(E) / E[0]


def _first_min_and_max(t, e):
    """time of the first energy minimum (parabolic refinement) and the value of the first maximum
    after it"""
    q = next(q for q in range(1, len(e) - 1) if e[q] < e[q - 1] and e[q] <= e[q + 1])
    den = e[q - 1] - 2 * e[q] + e[q + 1]
    tq = t[q] + (0.5 * (e[q - 1] - e[q + 1]) / den if den != 0 else 0.0) * (t[1] - t[0])
    r = next(r for r in range(q + 1, len(e) - 1) if e[r] > e[r - 1] and e[r] >= e[r + 1])
    return tq, e[r]


def test_gamma_scaling_of_the_released_sphere():
    """Table str_params (SI "Pre-stretched sphere", scaling study), each case at 64^3 until 2.5
    oscillation times tau_osc = R sqrt(rho_s / G).  With gamma = R sqrt(rho G) / mu the only
    dimensionless group when rho_s = rho_f and mu_a = mu:
    * the cases of one gamma (A1-A4, gamma = 20) collapse approximately in t / tau_osc (the same
      as t / tau_diss at fixed gamma): the first energy minimum within 6 % of their mean and the
      first rebound E_max / E_0 within 20 % of A1's (A1 and A2 share R and collapse exactly, see
      test_prestretched_sphere_scaling_is_exact; A3's sphere spans only 6.4 cells);
    * less damping per oscillation as gamma grows (B1, B2, A1, B3: gamma = 10, 15.8, 20, 30): the
      rebound grows strictly with gamma while the oscillation time stays within 25 % of A1's;
    * a solid denser or lighter than the fluid (C1, C2, gamma and tau_diss formed with rho_s, both
      equal to A1's) rebounds like A1 (within 10 %) but its minimum moves away from A1's by more
      than twice the spread of the A cases: rescaling by tau_diss no longer aligns the curves."""
    res = {c: _first_min_and_max(*_released(c)) for c in S.STR_PARAMS}
    tA = np.array([res[c][0] for c in ("A1", "A2", "A3", "A4")])
    spread = np.abs(tA - tA.mean()).max() / tA.mean()
    assert spread < 0.06, res
    for c in ("A2", "A3", "A4"):
        assert abs(res[c][1] / res["A1"][1] - 1) < 0.2, res
    reb = [res[c][1] for c in ("B1", "B2", "A1", "B3")]
    assert all(a < b for a, b in zip(reb, reb[1:])), res
    for c in ("B1", "B2", "B3"):
        assert abs(res[c][0] / res["A1"][0] - 1) < 0.25, res
    for c in ("C1", "C2"):
        assert abs(res[c][1] / res["A1"][1] - 1) < 0.1, res
        assert abs(res[c][0] / res["A1"][0] - 1) > 2 * spread, res


def test_prestretched_sphere_overshoots():
    """gamma = 20 (case A2) means many oscillations before the fluid damps them: the sphere
    passes through its rest shape and stretches the other way, so the energy has a deep
    minimum near t = tau_osc and grows again after it."""
    n = 32
    g = _prestretched(n, "A2", 0.2 / n)
    E = [g.body_stats(0)[5]]
    for _ in range(24):
        g.step(4)
        E.append(g.body_stats(0)[5])
    E = np.array(E)
    # the first local minimum, and the rebound after it
    k = next(q for q in range(1, len(E) - 1) if E[q] < E[q - 1] and E[q] <= E[q + 1])
    assert E[k] < 0.05 * E[0]
    assert E[k:].max() > 10 * E[k]


def test_settling_sphere_matches_stokes_drag_of_a_periodic_array():
    """A heavy sphere (R = 0.1, rho_s = 1.5, mu = 0.05: particle Reynolds number 0.06) in the
    triply periodic unit box, set up like the main text's settling runs (mu_a = mu, gamma_t =
    0, eps = h/2).  The box as a whole accelerates under the net weight, so the sphere's speed
    is taken relative to the box-mean velocity; it approaches Stokes' law u_0 = 2 (rho_s -
    rho_f) g R^2 / (9 mu) reduced by the periodic-array drag factor (Hasimoto 1959), 0.72 u_0
    here.  5 % covers the blur zone's uncertainty in the hydrodynamic radius (a tenth of a
    cell at R = 4.8 h moves u by 4 %), the neglected O(c^{8/3}) terms and the Oseen correction."""
    n = 48
    sc = S.stokes_sphere(n, precision="fp32")
    sc.update(mg_rtol=1e-9, mg_max_cycles=200)
    g = rmt.Grid(sc)
    R, mu, rs = 0.1, 0.05, 1.5
    u0 = 2 * (rs - 1.0) * 1.0 * R * R / (9 * mu)
    c = 4.0 / 3.0 * math.pi * R ** 3
    u_h = u0 * (1 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c * c)
    steps = int(round(2.5 / g.dt))
    rel = []
    for _ in range(10):
        g.step(steps // 10)
        st = g.body_stats(0)
        uz = g.read(rmt.RMT_F_U).reshape(3, -1)[2]
        rel.append(uz.mean() - st[2])  # settling speed relative to the box (downwards > 0)
        assert abs(st[0]) < 1e-3 * u0 and abs(st[1]) < 1e-3 * u0  # falls straight down
    rel = np.array(rel)
    assert np.all(np.diff(rel[:6]) > 0)  # accelerates towards the terminal speed
    assert abs(rel[-1] / u_h - 1) < 0.05
    assert abs(rel[-1] / rel[-2] - 1) < 0.01  # terminal


def test_cavity_sphere_convergence_rates():
    """The lid-driven cavity with a soft sphere (config of the main text's cavity run: R = 0.2, G =
    0.1, Re = 100) at T = 0.5 on 32^3 ... 96^3, the step kept within the explicit viscous limit
    (SI Fig. object_conv).  The sphere's volume error against the exact 4/3 pi R^3 falls at second
    order (the SI: 2.08) and ||J - 1|| at about 1.2 (the SI: 1.16); the windows exclude the
    neighbouring integer orders."""
    ns = (32, 48, 64, 96)
    V0 = 4.0 / 3.0 * math.pi * 0.2 ** 3
    dv, jn = [], []
    for n in ns:
        sc = S.cavity_sphere(n)
        h = 1.0 / n
        steps = math.ceil(0.5 / min(0.2 * h, 0.8 * h * h / (6 * 0.01)))
        sc.update(mg_rtol=1e-11, mg_max_cycles=200, dt=0.5 / steps)
        g = rmt.Grid(sc)
        g.step(steps)
        st = g.body_stats(0)
        dv.append(abs(st[4] - V0) / V0)
        jn.append(st[6])
        g.close()
    h = np.log([1.0 / n for n in ns])
    s_v = np.polyfit(h, np.log(dv), 1)[0]
    s_j = np.polyfit(h, np.log(jn), 1)[0]
    assert 1.7 < s_v < 2.4, (s_v, dv)
    assert 0.95 < s_j < 1.5, (s_j, jn)
