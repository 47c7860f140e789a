"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types an oracle formula: each compares the oracle with a
closed form, an invariant, a textbook solution or a brute-force computation.
"""
import ctypes as C

import numpy as np
import pytest
from scipy import ndimage

import oracle as O
from paper_2104_00095_gb300 import scenes as S

L = O.lib()


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# --------------------------------------------------------------------------- Heaviside
def test_heaviside_closed_form_points():
    """eq. sm_heavi: H(-eps)=0, H(0)=1/2, H(eps)=1, constant outside the blur zone."""
    eps = 0.037
    assert L.orc_heaviside(-eps, eps) == 0.0
    assert L.orc_heaviside(-2 * eps, eps) == 0.0
    assert L.orc_heaviside(0.0, eps) == 0.5
    assert L.orc_heaviside(eps, eps) == 1.0
    assert L.orc_heaviside(3 * eps, eps) == 1.0
    # odd symmetry about (0, 1/2)
    for p in np.linspace(-eps, eps, 17):
        assert abs(L.orc_heaviside(p, eps) + L.orc_heaviside(-p, eps) - 1.0) < 1e-15


def test_heaviside_c2_and_derivative():
    """H has a continuous second derivative (paper text after eq. sm_heavi); H' integrates
    to 1 and eps*H' lies in [0,1]; H' is the derivative of H (finite differences)."""
    eps = 0.05
    xs = np.linspace(-1.5 * eps, 1.5 * eps, 3001)
    Hs = np.array([L.orc_heaviside(x, eps) for x in xs])
    dH = np.array([L.orc_dheaviside(x, eps) for x in xs])
    fd = np.gradient(Hs, xs)
    assert np.max(np.abs(fd - dH)) < 1e-3 / eps
    assert np.all(eps * dH >= 0) and np.all(eps * dH <= 1.0 + 1e-15)
    assert abs(np.trapezoid(dH, xs) - 1.0) < 1e-6
    # second derivative continuous at +-eps: H'' -> 0 from inside
    d = 1e-5 * eps
    for e in (-eps, eps):
        h2 = (L.orc_dheaviside(e - np.sign(e) * d, eps) - L.orc_dheaviside(e - np.sign(e) * 2 * d, eps)) / d
        assert abs(h2) < 1e-3 / eps**2


# --------------------------------------------------------------------------- slopes
def _slope(q, ok=(1, 1, 1, 1, 1), h=1.0):
    qa = np.asarray(q, dtype=np.float64)
    oka = (C.c_int * 5)(*ok)
    return L.orc_limited_slope(_dp(qa), oka, h)


def test_slope_exact_on_linear_data():
    for a, b, h in [(0.3, 1.7, 0.1), (-2.0, -0.25, 0.03), (1.0, 0.0, 1.0)]:
        q = [a + b * h * s for s in range(-2, 3)]
        assert abs(_slope(q, h=h) - b) < 1e-12 * max(1, abs(b))


def test_slope_fourth_order_on_smooth_data():
    """Away from extrema the limited slope equals the 4th-order centred slope:
    error against the exact derivative falls ~16x per halving of h."""
    errs = []
    for h in (0.02, 0.01, 0.005):
        x0 = 0.3
        q = [np.sin(x0 + s * h) for s in range(-2, 3)]
        errs.append(abs(_slope(q, h=h) - np.cos(x0)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12 < r1 < 20 and 12 < r2 < 20


def test_slope_no_new_extrema_and_zero_at_extremum():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        q = np.cumsum(rng.random(5) * rng.choice([-1, 1]))  # monotone
        s = _slope(q)
        left, right = q[2] - 0.5 * s, q[2] + 0.5 * s
        lo, hi = min(q[1], q[3]), max(q[1], q[3])
        assert lo - 1e-12 <= left <= hi + 1e-12 and lo - 1e-12 <= right <= hi + 1e-12
    assert _slope([0.0, 1.0, 2.0, 1.0, 0.0]) == 0.0
    assert _slope([1.0, 0.0, -1.0, 0.0, 1.0]) == 0.0
    # missing inner neighbour -> zero; missing outer -> second-order limited slope
    assert _slope([0, 1, 2, 3, 4], ok=(1, 0, 1, 1, 1)) == 0.0
    assert abs(_slope([9, 1, 2, 3, 9], ok=(0, 1, 1, 1, 0)) - 1.0) < 1e-15


# --------------------------------------------------------------------------- Godunov
def _burgers_riemann_at_zero(uL, uR):
    """Entropy solution of u_t + (u^2/2)_x = 0 with data (uL, uR) sampled at x/t = 0."""
    if uL > uR:  # shock with speed (uL+uR)/2
        s = 0.5 * (uL + uR)
        return uL if s > 0 else uR
    if uL >= 0:  # rarefaction fan
        return uL
    if uR <= 0:
        return uR
    return 0.0


def test_godunov_normal_is_burgers_riemann_solution():
    rng = np.random.default_rng(3)
    for _ in range(5000):
        uL, uR = rng.normal(size=2)
        if abs(uL + uR) < 1e-12:
            continue
        assert L.orc_godunov_normal(uL, uR, 0.0) == _burgers_riemann_at_zero(uL, uR)
    for uL, uR in [(0.0, 1.0), (-1.0, 0.0), (0.0, 0.0), (-1.0, 1.0), (2.0, 3.0), (-3.0, -2.0)]:
        assert L.orc_godunov_normal(uL, uR, 0.0) == _burgers_riemann_at_zero(uL, uR)


def test_upwind_tolerance_only_changes_near_zero_velocities():
    """With a tolerance t the choices differ from the exact rule only where |u_L|, |u_L + u_R|
    or |u_n| is within t of zero; there the normal velocity is taken as 0."""
    rng = np.random.default_rng(13)
    t = 1e-9
    for _ in range(5000):
        uL, uR = rng.normal(size=2) * rng.choice([1.0, 1e-9])
        a, b = L.orc_godunov_normal(uL, uR, 0.0), L.orc_godunov_normal(uL, uR, t)
        if a != b:
            assert b == 0.0 and (abs(uL) <= t or abs(uL + uR) <= t or abs(uR) <= t)
        q1, q2 = rng.normal(size=2)
        un = rng.normal() * rng.choice([1.0, 1e-10])
        if abs(un) <= t:
            assert L.orc_upwind(q1, q2, un, t) == 0.5 * (q1 + q2)
        else:
            assert L.orc_upwind(q1, q2, un, t) == L.orc_upwind(q1, q2, un, 0.0)


# --------------------------------------------------------------------------- stress
def _tau(A, G=1.0):
    Aa = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
    out = np.zeros(9)
    assert L.orc_neohookean(_dp(Aa), G, _dp(out)) == 1
    return out.reshape(3, 3)


def test_zero_stress_identity_and_rotation():
    """tau_s = G(B - tr(B)/3 I) vanishes for xi = x and for rigid rotations (F = R)."""
    assert np.max(np.abs(_tau(np.eye(3), 0.7))) == 0.0
    rng = np.random.default_rng(11)
    for _ in range(50):
        R = S.random_rotation(rng)
        # xi = R^T (x - c) + c  ->  grad xi = R^T, F = R, B = I
        assert np.max(np.abs(_tau(R.T, 2.0))) < 1e-14


def test_uniaxial_stretch_and_simple_shear():
    lam, G = 1.21, 0.5
    F = np.diag([lam, lam**-0.5, lam**-0.5])
    t = _tau(np.linalg.inv(F), G)
    s = (lam**2 + 2.0 / lam) / 3.0
    assert np.allclose(t, G * np.diag([lam**2 - s, 1 / lam - s, 1 / lam - s]), atol=1e-14)
    gam = 0.3
    F = np.eye(3)
    F[0, 1] = gam
    t = _tau(np.linalg.inv(F), G)
    assert abs(t[0, 1] - G * gam) < 1e-14 and abs(t[1, 0] - G * gam) < 1e-14
    assert abs(t[0, 0] - G * (1 + gam**2 - (3 + gam**2) / 3)) < 1e-14


def test_stress_frame_indifference():
    rng = np.random.default_rng(5)
    for _ in range(20):
        F = np.eye(3) + 0.2 * rng.normal(size=(3, 3))
        Q = S.random_rotation(rng)
        t1 = _tau(np.linalg.inv(F))
        t2 = _tau(np.linalg.inv(Q @ F))
        assert np.allclose(t2, Q @ t1 @ Q.T, atol=1e-12)


# --------------------------------------------------------------------------- mixing
def _mix(Hm):
    H = np.asarray(Hm, dtype=np.float64)
    w = np.zeros(max(1, len(H)))
    Hmix = L.orc_mix_weights(len(H), _dp(H), _dp(w))
    return Hmix, w[: len(H)]


def test_mixing_rule_hand_cases():
    """SI eq. mod_heaviside and the combination rule above it."""
    H, w = _mix([0.3])
    assert abs(H - 0.3) < 1e-16 and abs(w[0] - 0.7) < 1e-16
    H, w = _mix([0.8, 0.9])  # sum(1-H) = 0.3 <= 1: plain sum
    assert abs(H - 0.7) < 1e-15 and np.allclose(w, [0.2, 0.1], atol=1e-16)
    H, w = _mix([0.2, 0.3])  # sum = 1.5 > 1: normalised, H = 0
    assert H == 0.0 and np.allclose(w, [0.8 / 1.5, 0.7 / 1.5], atol=1e-16)
    H, w = _mix([])
    assert H == 1.0


# --------------------------------------------------------------------------- level sets
def test_phi0_sphere_and_ellipsoid():
    sph = O.make_solid_desc(S.solid(S.SPHERE, (0.5, 0.4, 0.3), (0.2, 0.2, 0.2)))
    for X, d in [((0.5, 0.4, 0.3), -0.2), ((0.9, 0.4, 0.3), 0.2), ((0.5, 0.4, 0.5), 0.0)]:
        assert abs(L.orc_phi0(C.byref(sph), _dp(np.array(X))) - d) < 1e-15
    rng = np.random.default_rng(2)
    R = S.random_rotation(rng)
    a = np.array([0.15, 0.05, 0.08])
    c = np.array([0.4, 0.5, 0.6])
    ell = O.make_solid_desc(S.solid(S.ELLIPSOID, c, a, R))
    for _ in range(100):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        surf = c + R @ (a * v)  # a point on the surface
        assert abs(L.orc_phi0(C.byref(ell), _dp(surf))) < 1e-14
        inside = c + R @ (0.5 * a * v)
        assert L.orc_phi0(C.byref(ell), _dp(inside)) < 0
    for ax in range(3):  # exact distance along the principal axes
        e = np.zeros(3)
        e[ax] = 1.0
        X = c + R @ (e * (a[ax] + 0.03))
        assert abs(L.orc_phi0(C.byref(ell), _dp(X)) - 0.03) < 1e-14
    # equal semi-axes reduce to the sphere
    ell2 = O.make_solid_desc(S.solid(S.ELLIPSOID, c, (0.2, 0.2, 0.2), R))
    sph2 = O.make_solid_desc(S.solid(S.SPHERE, c, (0.2, 0.2, 0.2)))
    for _ in range(50):
        X = rng.random(3)
        assert abs(L.orc_phi0(C.byref(ell2), _dp(X)) - L.orc_phi0(C.byref(sph2), _dp(X))) < 1e-14


# --------------------------------------------------------------------------- layers
def _brute_layers(inside, periodic, Lmax):
    """Taxicab (face-neighbour) distance to the interior, computed with scipy's chamfer
    transform; periodic axes handled by tiling."""
    if periodic:
        t = np.tile(~inside, (3, 3, 3))
        d = ndimage.distance_transform_cdt(t, metric="taxicab")
        n = inside.shape
        d = d[n[0]:2 * n[0], n[1]:2 * n[1], n[2]:2 * n[2]]
    else:
        d = ndimage.distance_transform_cdt(~inside, metric="taxicab")
    out = np.where(d <= Lmax, d, -1)
    return out


@pytest.mark.parametrize("periodic,shape", [(False, S.SPHERE), (True, S.ELLIPSOID), (False, S.ELLIPSOID)])
def test_layers_match_brute_force_distance(periodic, shape):
    n = 20
    sc = S._box(n, periodic=periodic)
    rng = np.random.default_rng(4)
    c = (0.93, 0.5, 0.47) if periodic else (0.52, 0.47, 0.5)
    sc["solids"] = [S.solid(shape, c, (0.21, 0.13, 0.17), S.random_rotation(rng))]
    o = O.Oracle(sc)
    lay = o.read(O.F_LAYER).reshape(n, n, n).astype(int)  # [z][y][x]
    phi = o.read(O.F_PHI).reshape(n, n, n)
    inside = lay == 0
    assert np.all(phi[inside] < 0)
    ref = _brute_layers(inside, periodic, 4)
    assert np.array_equal(lay, ref)


def test_layers_stop_at_walls():
    n = 16
    sc = S._box(n, periodic=False)
    sc["solids"] = [S.solid(S.SPHERE, (0.5, 0.5, 0.2), (0.12,) * 3)]
    o = O.Oracle(sc)
    lay = o.read(O.F_LAYER).reshape(n, n, n).astype(int)
    assert np.array_equal(lay, _brute_layers(lay == 0, False, 4))
    assert lay[0].max() >= 0  # the band reaches the z=0 wall and stops there


# --------------------------------------------------------------------------- extrapolation
@pytest.mark.parametrize("periodic", [False, True])
def test_extrapolation_reproduces_affine_maps(periodic):
    """The WLS fit reproduces any affine xi exactly (main text: local linear model)."""
    n = 20
    sc = S._box(n, periodic=periodic)
    rng = np.random.default_rng(8)
    c = np.array([0.5, 0.48, 0.52])
    sc["solids"] = [S.solid(S.ELLIPSOID, c, (0.2, 0.12, 0.15), S.random_rotation(rng))]
    o = O.Oracle(sc)
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    P = np.stack([X, Y, Z]).reshape(3, -1)
    A = S.random_rotation(rng) @ np.diag([1.2, 0.9, 1.0 / 1.08])
    A = A / np.cbrt(np.linalg.det(A))
    b = c - A @ c + np.array([0.01, -0.02, 0.015])
    xi = A @ P + b[:, None]
    assert o.write(O.F_XI, xi.reshape(-1)) == 0
    lay = o.read(O.F_LAYER)
    got = o.read(O.F_XI).reshape(3, -1)
    band = lay >= 1
    assert band.sum() > 500
    assert np.max(np.abs(got[:, band] - xi[:, band])) < 1e-12
    # and the layer-0 cells are exactly those whose mapped point is inside
    phi = o.read(O.F_PHI)
    assert np.all(phi[lay == 0] < 0) and np.all(phi[lay >= 1] >= -1e-12)


# --------------------------------------------------------------------------- projections
def _fresh(n, periodic):
    sc = S._box(n, periodic=periodic)
    sc["dt"] = 0.01
    return O.Oracle(sc)


@pytest.mark.parametrize("periodic", [False, True])
def test_mac_projection_divergence_free_and_idempotent(periodic):
    n = 12
    o = _fresh(n, periodic)
    rng = np.random.default_rng(1)
    rho = 1.0 + 0.5 * rng.random(n**3)
    nf = n**2 * (n + 1)
    U = [rng.normal(size=nf) for _ in range(3)]
    shp = [(n, n, n + 1), (n, n + 1, n), (n + 1, n, n)]
    for d in range(3):
        u = U[d].reshape(shp[d])
        if periodic:  # the two copies of the periodic face agree
            sl = [slice(None)] * 3
            sl[2 - d] = -1
            s0 = [slice(None)] * 3
            s0[2 - d] = 0
            u[tuple(sl)] = u[tuple(s0)]
        else:
            sl = [slice(None)] * 3
            sl[2 - d] = 0
            u[tuple(sl)] = 0.0
            sl[2 - d] = -1
            u[tuple(sl)] = 0.0
    q = np.zeros(n**3)
    dt = 0.01
    assert L.orc_mac_project(o._g, _dp(rho), _dp(U[0]), _dp(U[1]), _dp(U[2]), dt, _dp(q)) == 0
    div = np.zeros((n, n, n))
    for d in range(3):
        u = U[d].reshape(shp[d])
        div += np.diff(u, axis=2 - d) * n
    assert np.max(np.abs(div)) < 1e-10 * max(1.0, max(np.abs(x).max() for x in U) * n)
    U2 = [x.copy() for x in U]
    q2 = np.zeros(n**3)
    assert L.orc_mac_project(o._g, _dp(rho), _dp(U2[0]), _dp(U2[1]), _dp(U2[2]), dt, _dp(q2)) == 0
    for d in range(3):
        assert np.max(np.abs(U2[d] - U[d])) < 1e-10


def test_fe_operator_identities():
    n = 8
    o = _fresh(n, False)
    rng = np.random.default_rng(9)
    NN = (n + 1) ** 3
    beta = np.ones(n**3)
    one = np.ones(NN)
    out = np.zeros(NN)
    L.orc_fe_apply(o._g, _dp(beta), _dp(one), _dp(out))
    assert np.max(np.abs(out)) < 1e-15
    # linear function: K psi vanishes at interior nodes (consistency of the FE Laplacian)
    xn = np.arange(n + 1) / n
    Zn, Yn, Xn = np.meshgrid(xn, xn, xn, indexing="ij")
    lin = (0.3 * Xn - 0.7 * Yn + 0.2 * Zn).reshape(-1)
    L.orc_fe_apply(o._g, _dp(beta), _dp(lin), _dp(out))
    inner = out.reshape(n + 1, n + 1, n + 1)[1:-1, 1:-1, 1:-1]
    assert np.max(np.abs(inner)) < 1e-15
    # weak divergence is minus the adjoint of the cell gradient: psi.f(V) = h^3 sum V.G psi
    psi = rng.normal(size=NN)
    V = rng.normal(size=3 * n**3)
    f = np.zeros(NN)
    L.orc_fe_weak_div(o._g, _dp(V), _dp(f))
    G = np.zeros(3 * n**3)
    L.orc_cell_grad(o._g, _dp(psi), _dp(G))
    assert abs(psi @ f - (V @ G) / n**3) < 1e-12 * np.abs(psi).sum()
    # element stiffness: the 27-point stencil of an interior node with beta = 1
    e = np.zeros(NN)
    mid = (n // 2) + (n + 1) * ((n // 2) + (n + 1) * (n // 2))
    e[mid] = 1.0
    L.orc_fe_apply(o._g, _dp(beta), _dp(e), _dp(out))
    st = out.reshape(n + 1, n + 1, n + 1)[n // 2 - 1:n // 2 + 2, n // 2 - 1:n // 2 + 2, n // 2 - 1:n // 2 + 2] * n
    # exact integrals of grad N_i . grad N_j for trilinear hats on a uniform grid
    assert abs(st[1, 1, 1] - 8.0 / 3.0) < 1e-14
    assert abs(st[1, 1, 0]) < 1e-14  # edge neighbours
    assert abs(st[1, 0, 0] + 1.0 / 6.0) < 1e-14  # face diagonals
    assert abs(st[0, 0, 0] + 1.0 / 12.0) < 1e-14  # body diagonals


def test_fe_solve_manufactured_second_order():
    """Neumann problem with psi = cos(pi x)cos(pi y)cos(pi z): V = grad psi sampled at cell
    centres; the FE solution converges to psi at second order."""
    errs = []
    for n in (8, 16):
        o = _fresh(n, False)
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        V = np.concatenate([(-np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y) * np.cos(np.pi * Z)).ravel(),
                            (-np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y) * np.cos(np.pi * Z)).ravel(),
                            (-np.pi * np.cos(np.pi * X) * np.cos(np.pi * Y) * np.sin(np.pi * Z)).ravel()])
        rho = np.ones(n**3)
        psi = np.zeros((n + 1) ** 3)
        assert L.orc_fe_solve(o._g, _dp(rho), _dp(V), _dp(psi)) == 0
        xn = np.arange(n + 1) * h
        Zn, Yn, Xn = np.meshgrid(xn, xn, xn, indexing="ij")
        ex = (np.cos(np.pi * Xn) * np.cos(np.pi * Yn) * np.cos(np.pi * Zn)).ravel()
        ex -= ex.mean()
        errs.append(np.max(np.abs(psi - ex)))
    assert errs[0] / errs[1] > 3.3


# --------------------------------------------------------------------------- whole steps
def test_quiescent_unstressed_sphere_stays_at_rest():
    """u = 0, xi = x, no gravity, no lid: every term of eq. dis_full_mmt vanishes."""
    sc = S._box(16, periodic=False)
    sc.update(dt=0.2 / 16)
    sc["solids"] = [S.solid(S.SPHERE, (0.5, 0.5, 0.5), (0.2,) * 3, rho_s=1.3, G=0.5)]
    o = O.Oracle(sc)
    xi0 = o.read(O.F_XI)
    assert o.step(3) == 0
    # rounding only: grad xi of xi = x is the identity up to the spacing's rounding
    assert np.max(np.abs(o.read(O.F_U))) < 1e-12
    xi = o.read(O.F_XI)
    ok = np.isfinite(xi0) & np.isfinite(xi)
    assert np.max(np.abs(xi[ok] - xi0[ok])) < 1e-13
    assert np.array_equal(np.isfinite(xi0), np.isfinite(xi))


def test_rigidly_rotated_sphere_has_no_stress():
    """xi = R^T (x - c) + c describes an unstressed body: the whole step keeps u = 0."""
    n = 16
    sc = S._box(n, periodic=False)
    sc.update(dt=0.2 / n)
    c = np.array([0.5, 0.5, 0.5])
    sc["solids"] = [S.solid(S.SPHERE, c, (0.22,) * 3, rho_s=1.0, G=1.0)]
    o = O.Oracle(sc)
    R = S.random_rotation(np.random.default_rng(12))
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    P = np.stack([X, Y, Z]).reshape(3, -1)
    xi = R.T @ (P - c[:, None]) + c[:, None]
    assert o.write(O.F_XI, xi.reshape(-1)) == 0
    assert o.step(2) == 0
    assert np.max(np.abs(o.read(O.F_U))) < 1e-12


def test_uniform_translation_advects_reference_map_exactly():
    """Periodic box, uniform u = U, unstressed sphere: u stays U and xi = x - U t exactly
    (affine transport, eq. xi_adv), because the limited slopes, the Taylor states and the
    upwinding are exact on linear data."""
    n = 16
    U = np.array([0.3, -0.2, 0.1])
    sc = S._box(n, periodic=True)
    sc.update(dt=0.2 / n)
    sc["solids"] = [S.solid(S.SPHERE, (0.5, 0.5, 0.5), (0.2,) * 3, rho_s=1.0, G=0.4)]
    o = O.Oracle(sc)
    o.write(O.F_U, np.repeat(U, n**3))
    steps = 4
    assert o.step(steps) == 0
    t = steps * 0.2 / n
    u = o.read(O.F_U).reshape(3, -1)
    assert np.max(np.abs(u - U[:, None])) < 1e-12
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    P = np.stack([X, Y, Z]).reshape(3, -1)
    xi = o.read(O.F_XI).reshape(3, -1)
    ok = np.isfinite(xi[0])
    assert ok.sum() > 500
    exp = P - U[:, None] * t
    diff = xi[:, ok] - exp[:, ok]
    diff -= np.round(diff)  # periodic images
    assert np.max(np.abs(diff)) < 1e-12


def test_viscous_shear_wave_decays_at_the_right_rate():
    """Pure fluid, periodic: u = (sin 2 pi z, 0, 0) decays like exp(-4 pi^2 nu t);
    the error falls at least first order under refinement (SI: the scheme is about
    first order in space and time)."""
    errs = []
    nu = 0.05
    T = 0.05
    for n in (8, 16, 32):
        sc = S._box(n, periodic=True)
        sc.update(mu=nu, dt=0.0)
        o = O.Oracle(sc)
        dt = o.dt
        steps = int(round(T / dt))
        z = (np.arange(n) + 0.5) / n
        Z = np.broadcast_to(z[:, None, None], (n, n, n))
        u0 = np.zeros((3, n, n, n))
        u0[0] = np.sin(2 * np.pi * Z)
        o.write(O.F_U, u0.reshape(-1))
        assert o.step(steps) == 0
        u = o.read(O.F_U).reshape(3, n, n, n)
        ex = np.sin(2 * np.pi * Z) * np.exp(-4 * np.pi**2 * nu * steps * dt)
        errs.append(np.sqrt(np.mean((u[0] - ex) ** 2)))
    assert errs[0] / errs[1] > 2.0 and errs[1] / errs[2] > 2.0


# --------------------------------------------------------------------------- wall repulsion
def test_repulsion_magnitude_meets_its_defining_conditions():
    """A_rep (SI "Contact with a wall") is the largest of three accelerations, each fixed by a
    condition the paper states: check each condition where its term is the largest."""
    V, dw, Lmin, g = 4.0 / 3.0 * np.pi * 0.1 ** 3, 1.0 / 64, 0.2, 1.0
    vrep = dw * Lmin ** 2
    # approach at U: the centre of mass, decelerated by V_rep A / V, stops within d_w at t = 2 d_w / U
    U = 3.0
    a = L.orc_rep_accel(V, U, dw, Lmin, 1.0, 1.0, 0.0, 1e-6)
    acm = vrep * a / V
    ts = U / acm
    assert ts == pytest.approx(2 * dw / U, rel=1e-12)
    assert U * ts - 0.5 * acm * ts ** 2 == pytest.approx(dw, rel=1e-12)
    # resting on the wall: the repulsion on the breached cells carries the body's net weight
    rho_s = 3.0
    a = L.orc_rep_accel(V, 1e-6, dw, Lmin, rho_s, 1.0, g, 1e-6)
    assert rho_s * vrep * a == pytest.approx(abs(rho_s - 1.0) * V * g, rel=1e-12)
    # neither: the safety floor U_safe^2 / d_w
    assert L.orc_rep_accel(V, 1e-6, dw, Lmin, 1.0, 1.0, 0.0, 4.5) == pytest.approx(4.5 ** 2 / dw, rel=1e-15)
    # and it is the maximum of the three
    terms = [4.5 ** 2 / dw, V * U ** 2 / (2 * dw * vrep), abs(rho_s - 1.0) * V * g / (rho_s * vrep)]
    assert L.orc_rep_accel(V, U, dw, Lmin, rho_s, 1.0, g, 4.5) == pytest.approx(max(terms), rel=1e-15)


def _wall_sphere(n=16, rep=8.0, dw=0.0):
    sc = S._box(n, periodic=False)
    h = 1.0 / n
    sc.update(dt=0.1 * h, wall_dw=dw)
    sc["solids"] = [S.solid(S.SPHERE, (0.5, 0.5, 0.22 + 0.3 * h), (0.22,) * 3, rho_s=1.0, G=0.2, rep_A=rep)]
    return sc


@pytest.mark.parametrize("dw_cells", [0.0, 2.0])
def test_repulsion_field_matches_eq_wall_acc(dw_cells):
    """The acceleration the oracle adds to u* equals eq. wall_acc evaluated independently from
    the body's half-step reference map: sphere phi = |xi - c| - R, transition width h, inward
    normal of the breached wall (here the bottom one), zero elsewhere."""
    n = 16
    h = 1.0 / n
    sc = _wall_sphere(n, rep=8.0, dw=dw_cells * h)
    o = O.Oracle(sc)
    assert o.step(1) == 0
    a = o.read(O.F_REPULSION).reshape(3, n, n, n)
    xh = o.read(O.F_XI_HALF, 0).reshape(3, n, n, n)
    c = np.array(sc["solids"][0]["center"])
    phi = np.sqrt(sum((xh[q] - c[q]) ** 2 for q in range(3))) - 0.22
    f = np.where(phi <= -h, 1.0, np.where(phi < h, 0.5 - phi / (2 * h), 0.0))
    f = np.where(np.isfinite(xh[0]), f, 0.0)
    dw = dw_cells * h if dw_cells > 0 else h
    kk = np.arange(n)
    near_bottom = ((kk + 0.5) * h < dw)[:, None, None]
    expect_z = np.where(near_bottom, 8.0 * f, 0.0)
    assert np.allclose(a[2], expect_z, rtol=0, atol=1e-14)
    assert np.count_nonzero(a[2]) > 0
    # the sphere reaches no other wall: no x or y component
    assert np.all(a[0] == 0.0) and np.all(a[1] == 0.0)


def test_repulsion_pushes_the_body_off_the_wall():
    """With repulsion the body near the bottom wall starts to move up; without it, at rest."""
    n = 16
    w = {}
    for rep in (0.0, 8.0):
        o = O.Oracle(_wall_sphere(n, rep=rep))
        assert o.step(3) == 0
        u = o.read(O.F_U).reshape(3, n, n, n)
        lay = o.read(O.F_LAYER, 0).reshape(n, n, n)
        w[rep] = u[2][lay == 0].mean()
    assert abs(w[0.0]) < 1e-12
    assert w[8.0] > 1e-4


# --------------------------------------------------------------------------- initial pressure
def _taylor_green(n, iters, tol):
    """2-D Taylor-Green vortex u = (sin x cos y, -cos x sin y, 0) in a periodic [0,2pi]^2 box
    (4 cells deep); its pressure is p = (cos 2x + cos 2y)/4 (rho = 1)."""
    Lx = 2 * np.pi
    h = Lx / n
    sc = S._box(n, periodic=True)
    sc.update(n=(n, n, 4), hi=(Lx, Lx, 4 * h), mu=0.01, dt=0.1 * h)
    o = O.Oracle(sc)
    x = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, x, indexing="xy")
    u = np.zeros((3, 4, n, n))
    u[0] = np.sin(X) * np.cos(Y)
    u[1] = -np.cos(X) * np.sin(Y)
    o.write(O.F_U, u.reshape(-1))
    rc, it = o.init_pressure(iters, tol)
    p = o.read(O.F_P).reshape(4, n, n)
    xn = np.arange(n) * h
    Xn, Yn = np.meshgrid(xn, xn, indexing="xy")
    pe = 0.25 * (np.cos(2 * Xn) + np.cos(2 * Yn))
    return rc, it, np.abs(p - (pe - pe.mean())[None]).max(), o, u


def test_initial_pressure_iterations_recover_the_taylor_green_pressure():
    """SI "Initialization" item 2: the iterations turn p = 0 into the pressure the velocity
    field needs; for the Taylor-Green vortex that is known in closed form, and the error falls
    at second order with h."""
    rc16, it16, e16, o, u = _taylor_green(16, 30, 1e-6)
    rc32, it32, e32, _, _ = _taylor_green(32, 30, 1e-6)
    assert rc16 == 0 and rc32 == 0
    assert it16 < 30 and it32 < 30  # the estimate converged before the cap
    assert e16 < 0.02 and e32 < 0.006  # amplitude of p is 0.5
    assert e16 / e32 > 3.0
    # nothing but p changed
    assert np.array_equal(o.read(O.F_U), u.reshape(-1))


def test_initial_pressure_iterations_leave_a_quiescent_state_alone():
    sc = S.cavity_sphere(16)
    sc["wall_u"] = [[0.0] * 3 for _ in range(6)]
    o = O.Oracle(sc)
    before = {f: o.read(f) for f in (O.F_U, O.F_RHO)}
    xi = o.read(O.F_XI, 0)
    rc, it = o.init_pressure(5, 1e-8)
    assert rc == 0 and 1 <= it <= 5
    assert np.abs(o.read(O.F_P)).max() < 1e-10  # rounding noise of a state at rest
    for f, v in before.items():
        assert np.array_equal(o.read(f), v)
    assert np.array_equal(o.read(O.F_XI, 0), xi, equal_nan=True)


# --------------------------------------------------------------------------- swimmer diagnostics
def _solid_fraction(phi, eps):
    """1 - H_eps(phi) of eq. sm_heavi, written out here."""
    H = np.where(phi <= -eps, 0.0, np.where(phi >= eps, 1.0,
                 0.5 * (1 + phi / eps + np.sin(np.pi * phi / eps) / np.pi)))
    return 1.0 - H


def test_body_stats_uniform_flow_and_volume():
    """A uniform velocity is the centroid velocity of every body and does no active work; the
    volume is the integral of the solid fraction (close to 4/3 pi R^3)."""
    n = 24
    sc = S._box(n, periodic=True)
    sc.update(dt=0.2 / n)
    R = 0.25
    sc["solids"] = [S.solid(S.SPHERE, (0.5, 0.5, 0.5), (R,) * 3, active_A=0.7, active_omega=2 * np.pi,
                            active_len=0.5)]
    o = O.Oracle(sc)
    U = np.array([0.3, -0.1, 0.2])
    o.write(O.F_U, np.repeat(U, n ** 3))
    st = o.body_stats(0)
    assert np.allclose(st[:3], U, rtol=0, atol=1e-14)
    assert st[3] == 0.0
    phi, lay = o.read(O.F_PHI, 0), o.read(O.F_LAYER, 0)
    w = np.where(lay >= 0, _solid_fraction(phi, 1.5 / n), 0.0)
    assert st[4] == pytest.approx(w.sum() / n ** 3, rel=1e-13)
    assert st[4] == pytest.approx(4 / 3 * np.pi * R ** 3, rel=0.05)  # blur of 1.5 h


def test_body_stats_active_power_brute_force():
    """u = (c X^2 Z, 0, 0) on an undeformed body aligned with the axes: only the xx active
    stress acts, and sigma_a : grad u = (3/2) Z sigma_0(X) (2/3) 2 c X Z = 2 c X Z^2 sigma_0(X)
    (the centred difference of a quadratic is exact), summed by hand over the solid fraction."""
    n = 32
    sc = S._box(n, periodic=True)
    sc.update(dt=0.2 / n)
    ctr = np.array([0.5, 0.5, 0.5])
    A_, w_, l_ = 0.7, 2 * np.pi, 0.45
    sc["solids"] = [S.solid(S.ELLIPSOID, ctr, (0.3, 0.12, 0.12), active_A=A_, active_omega=w_, active_len=l_)]
    o = O.Oracle(sc)
    x = (np.arange(n) + 0.5) / n
    Z3, Y3, X3 = np.meshgrid(x, x, x, indexing="ij")
    Xr, Zr = X3 - ctr[0], Z3 - ctr[2]
    c = 0.8
    u = np.zeros((3, n, n, n))
    u[0] = c * Xr ** 2 * Zr
    o.write(O.F_U, u.reshape(-1))
    st = o.body_stats(0)
    phi, lay = o.read(O.F_PHI, 0).reshape(n, n, n), o.read(O.F_LAYER, 0).reshape(n, n, n)
    wfrac = np.where(lay >= 0, _solid_fraction(phi, 1.5 / n), 0.0)
    s0 = A_ * np.sin(2 * np.pi * Xr / l_)  # t = 0
    P = -np.sum(wfrac * 2 * c * Xr * Zr ** 2 * s0) / n ** 3
    assert abs(P) > 1e-6
    assert st[3] == pytest.approx(P, rel=1e-12)
    # a flow whose stretching is odd in X does no net work on this symmetric body
    u[0] = c * Xr * Zr
    o.write(O.F_U, u.reshape(-1))
    assert abs(o.body_stats(0)[3]) < 1e-12 * abs(P) + 1e-18


def test_body_stats_rigid_rotation_has_no_centroid_velocity():
    n = 24
    sc = S._box(n, periodic=True)
    sc.update(dt=0.2 / n)
    sc["solids"] = [S.solid(S.SPHERE, (0.5, 0.5, 0.5), (0.25,) * 3)]
    o = O.Oracle(sc)
    x = (np.arange(n) + 0.5) / n - 0.5
    Z3, Y3, X3 = np.meshgrid(x, x, x, indexing="ij")
    om = np.array([0.3, -0.5, 0.8])
    u = np.stack([om[1] * Z3 - om[2] * Y3, om[2] * X3 - om[0] * Z3, om[0] * Y3 - om[1] * X3])
    o.write(O.F_U, u.reshape(-1))
    st = o.body_stats(0)
    assert np.abs(st[:3]).max() < 1e-14


def _affine_xi(n, ctr, M):
    """xi = ctr + M (x - ctr) at every cell centre of the periodic unit box ([3][N] layout)."""
    x = (np.arange(n) + 0.5) / n
    Z3, Y3, X3 = np.meshgrid(x, x, x, indexing="ij")
    r = np.stack([X3 - ctr[0], Y3 - ctr[1], Z3 - ctr[2]]).reshape(3, -1)
    return (np.asarray(ctr)[:, None] + M @ r).reshape(-1)


@pytest.mark.parametrize("stretch", ["isochoric", "rotated"])
def test_body_stats_elastic_energy_of_a_uniform_stretch(stretch):
    """SI "Pre-stretched sphere", eq. elas: a body deformed by a uniform F has the energy density
    G/2 (sum_i lambda_i^2 - 3 - 2 ln(lambda_1 lambda_2 lambda_3)) everywhere (lambda_i the
    principal stretches of F; tr(F^T F) is invariant under rotations), so the energy is that
    density times the body's volume, and J - 1 = prod lambda_i - 1 at every cell.  The affine
    reference map is xi = c + F^-1 (x - c)."""
    n = 32
    G_ = 1.7
    sc = S._box(n, periodic=True)
    sc.update(dt=0.2 / n)
    ctr = np.array([0.5, 0.5, 0.5])
    sc["solids"] = [S.solid(S.SPHERE, ctr, (0.2,) * 3, G=G_)]
    o = O.Oracle(sc)
    if stretch == "isochoric":  # the paper's pre-stretch: lambda along x, 1/sqrt(lambda) across
        lam = np.array([1.21, 1.21 ** -0.5, 1.21 ** -0.5])
        Q = np.eye(3)
    else:
        lam = np.array([1.1, 0.93, 1.04])
        Q = S.random_rotation(np.random.default_rng(3))
    F = Q @ np.diag(lam) @ Q.T
    assert o.write(O.F_XI, _affine_xi(n, ctr, np.linalg.inv(F)), 0) == 0
    st = o.body_stats(0)
    phi_el = 0.5 * G_ * (np.sum(lam ** 2) - 3 - 2 * np.log(np.prod(lam)))
    assert phi_el > 0
    assert st[5] == pytest.approx(phi_el * st[4], rel=1e-10)
    assert st[6] == pytest.approx(abs(np.prod(lam) - 1), abs=1e-11)
    assert st[4] == pytest.approx(4 / 3 * np.pi * 0.2 ** 3 * np.prod(lam), rel=0.05)


def test_body_stats_undeformed_body_has_no_elastic_energy():
    n = 24
    sc = S._box(n, periodic=True)
    sc.update(dt=0.2 / n)
    sc["solids"] = [S.solid(S.ELLIPSOID, (0.5, 0.5, 0.5), (0.3, 0.15, 0.1))]
    o = O.Oracle(sc)
    st = o.body_stats(0)
    assert abs(st[5]) < 1e-12 * st[4] and st[6] < 1e-12


def test_prestretched_sphere_scaling_is_exact():
    """SI "Pre-stretched sphere" item 2 (Table str_params, cases A1 and A2): the two runs share
    R and gamma = R sqrt(rho G) / mu, so with time scaled by tau_diss (A1's step twice A2's)
    they are the same problem with u scaled by 1/2 and every stress and p by 1/4.  Each factor
    is a power of two, so the discrete runs agree bit for bit under that scaling: a term with a
    misplaced dt, mu, G or rho breaks it."""
    n, h = 16, 1.0 / 16
    runs = {}
    for case, dt in (("A2", 0.1 * h), ("A1", 0.2 * h)):
        sc = S.prestretched_sphere(n, case, dt=dt)
        o = O.Oracle(sc)
        assert o.write(O.F_XI, S.prestretch_xi(sc), 0) == 0
        e0 = o.body_stats(0)[5]
        assert o.step(3) == 0, o.error()
        runs[case] = (o.read(O.F_U), o.read(O.F_P), o.read(O.F_XI, 0), e0, o.body_stats(0))
    (u1, p1, x1, e01, s1), (u2, p2, x2, e02, s2) = runs["A1"], runs["A2"]
    assert np.abs(u2).max() > 1e-3 and e02 > 0
    assert np.array_equal(2 * u1, u2)
    assert np.array_equal(4 * p1, p2)
    assert np.array_equal(x1, x2, equal_nan=True)
    assert 4 * e01 == e02 and 4 * s1[5] == s2[5]
    assert s2[5] < e02  # the stretched sphere starts to relax
