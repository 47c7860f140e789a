"""Pins of the oracle's least-squares extrapolation weights, its search-radius fallback and its
face stress, each against an independent computation written from the paper.

* eq. weight (SI "Weighting scheme for weighted least squares-based extrapolation"): on a
  non-affine reference map every band value must equal a weighted least-squares fit computed
  here with numpy's lstsq from the paper's definition (kernel 2^-(r_i+r_j+r_k), the factor
  max(0, x'.n_e/|x'|) with x' = x_e - x_d for layers 1 and 2 only, n_e the normalised gradient
  of phi_0(xi) at e from a kernel-only fit).  Each plausible mistake (the sign of x', the clip
  at zero, the kernel, the layer switch) is shown to move the result far beyond the tolerance.
* degenerate systems (main text "Extrapolation of xi"): where the 5^3 box holds only coplanar
  data the fit must be repeated with a 7^3 box, not skipped to 9^3.
* face stress (SI "Stress calculations", eq. mixed_stresses; main text "Swimming" for the active
  stress): for a smooth non-affine map, the oracle's cell divergence of the blended face stress
  must converge at second order to the divergence of the continuous stress field, which is
  differentiated here by fourth-order finite differences of its closed form.
"""
import numpy as np
import pytest

import oracle as O
from paper_2104_00095_gb300 import scenes as S

# ----------------------------------------------------------------------------- helpers


def _centres(n):
    return (np.arange(n) + 0.5) / n


def _grid_points(n):
    x = _centres(n)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return np.stack([X, Y, Z])  # [3][n][n][n], x fastest in memory


def _sphere_grad_dir(X, c):
    """direction of grad_X phi_0 for a sphere centred at c (phi_0 = |X - c| - R)."""
    return np.asarray(X) - np.asarray(c)


def _fit(offs, vals, w):
    """Weighted affine fit xi_d ~ a + G (x_d - x_e) by lstsq on sqrt(w)-scaled rows; offs in
    cell units.  Returns (a[3], G[3][3] with G[:, b] the derivative along axis b per cell),
    or None when fewer than 4 points carry weight or the rows do not span R^4."""
    keep = w > 0
    if keep.sum() < 4:
        return None
    M = np.hstack([np.ones((keep.sum(), 1)), offs[keep]])
    sw = np.sqrt(w[keep])[:, None]
    A = M * sw
    s = np.linalg.svd(A, compute_uv=False)
    if s[-1] <= 1e-9 * s[0]:
        return None
    coef, *_ = np.linalg.lstsq(A, vals[keep] * sw, rcond=None)
    return coef[0], coef[1:].T  # value, gradient [component][axis]


def _expected(xi, lay, e, le, n, centre, variant="paper", rs_list=(2, 3, 4)):
    """xi_e by the paper's weighted least squares, from the data of the cells with layer < le.
    variant names a deliberate mistake (used to show that the pin detects it)."""
    i, j, k = e
    for rs in rs_list:
        offs, vals = [], []
        for dk in range(-rs, rs + 1):
            for dj in range(-rs, rs + 1):
                for di in range(-rs, rs + 1):
                    p, q, r = i + di, j + dj, k + dk
                    if not (0 <= p < n and 0 <= q < n and 0 <= r < n):
                        continue
                    ld = lay[r, q, p]
                    if ld < 0 or ld >= le:
                        continue
                    offs.append((di, dj, dk))
                    vals.append(xi[:, r, q, p])
        if not offs:
            continue
        offs = np.array(offs, dtype=float)
        vals = np.array(vals)
        ssum = np.abs(offs).sum(axis=1)
        kern = {"kernel_max": 2.0 ** -np.abs(offs).max(axis=1),
                "kernel_4": 4.0 ** -ssum}.get(variant, 2.0 ** -ssum)
        switch = {"switch_1": 1, "switch_3": 3}.get(variant, 2)
        f0 = _fit(offs, vals, kern)
        if f0 is None:
            continue
        if le > switch:
            return f0[0], rs
        a0, G0 = f0
        gX = _sphere_grad_dir(a0, centre)
        v = G0.T @ gX  # grad_x phi_0(xi) = (grad xi)^T grad_X phi_0
        if not np.linalg.norm(v) > 0:
            continue
        nrm = v / np.linalg.norm(v)
        xp = -offs  # x' = x_e - x_d, in cell units
        if variant == "sign":
            xp = offs
        cs = xp @ nrm / np.linalg.norm(xp, axis=1)
        w = cs * kern
        if variant == "noclip":
            w = np.abs(cs) * kern
        f1 = _fit(offs, vals, w)
        if f1 is None:
            continue
        return f1[0], rs
    return None, None


# ------------------------------------------------------------------ eq. weight, by hand


def _quadratic_map(P, c, kappa):
    """A smooth non-affine reference map about c: xi = x + kappa q(x - c)."""
    r = P - np.asarray(c)[:, None, None, None]
    q = np.stack([r[1] ** 2 - 0.5 * r[2] * r[0], r[2] * r[0] + 0.7 * r[1] ** 2, r[0] ** 2 - r[1] * r[2]])
    return P + kappa * q


def test_wls_weights_on_a_non_affine_map():
    n = 16
    c = np.array([0.52, 0.49, 0.505])
    sc = S._box(n, periodic=False)
    sc["solids"] = [S.solid(S.SPHERE, c, (0.27, 0.27, 0.27))]
    o = O.Oracle(sc)
    xi = _quadratic_map(_grid_points(n), c, 1.5)
    assert o.write(O.F_XI, xi.reshape(-1)) == 0
    lay = o.read(O.F_LAYER).reshape(n, n, n).astype(int)
    got = o.read(O.F_XI).reshape(3, n, n, n)
    # layer-0 values are the written map itself
    assert np.array_equal(got[:, lay == 0], xi[:, lay == 0])
    worst, mutated = 0.0, {"sign": 0.0, "noclip": 0.0, "kernel_max": 0.0, "kernel_4": 0.0, "switch_1": 0.0,
                           "switch_3": 0.0}
    checked = {1: 0, 2: 0, 3: 0, 4: 0}
    scale = np.abs(got[:, lay >= 0]).max()
    for (k, j, i) in zip(*np.nonzero(lay >= 1)):
        le = lay[k, j, i]
        exp, rs = _expected(got, lay, (i, j, k), le, n, c)
        assert exp is not None and rs == 2
        err = np.abs(got[:, k, j, i] - exp).max() / scale
        worst = max(worst, err)
        checked[le] += 1
        for var in mutated:
            alt, _ = _expected(got, lay, (i, j, k), le, n, c, variant=var)
            if alt is not None:
                mutated[var] = max(mutated[var], np.abs(alt - got[:, k, j, i]).max() / scale)
    assert min(checked.values()) > 50, checked
    assert worst < 1e-12, worst
    # each mistake moves some band value by far more than the tolerance
    for var, d in mutated.items():
        assert d > 1e-5, (var, d)


# ------------------------------------------------------------- r_s fallback, by hand


def test_wls_radius_fallback_takes_the_7_box():
    """Layer 0 is a 9 x 9 plane of cells plus one cell two below its centre.  The layer-1 cell
    above the centre sees only the plane in its 5^3 box (coplanar data: singular), the extra cell
    enters at r_s = 3, and the 9^3 box would add more plane cells: the oracle must return the
    7^3 fit."""
    n, i0, j0, z0 = 16, 8, 8, 8
    h = 1.0 / n
    c = np.array([0.5, 0.5, 0.5])
    sc = S._box(n, periodic=False)
    sc["solids"] = [S.solid(S.SPHERE, c, (0.3, 0.3, 0.3))]
    o = O.Oracle(sc)
    P = _grid_points(n)
    xref = np.array([(i0 + 0.5) * h, (j0 + 0.5) * h, (z0 + 0.5) * h])
    r = P - xref[:, None, None, None]
    xi_full = c[:, None, None, None] + 0.5 * r + 0.5 * np.stack([r[1] ** 2, r[0] * r[1], r[0] ** 2 + r[1] ** 2])
    xi = np.full((3, n, n, n), np.nan)
    sel = np.zeros((n, n, n), bool)
    sel[z0, j0 - 4:j0 + 5, i0 - 4:i0 + 5] = True
    sel[z0 - 2, j0, i0] = True
    xi[:, sel] = xi_full[:, sel]
    o.write(O.F_XI, xi.reshape(-1))  # cells beside the plane stay degenerate: not checked here
    lay = o.read(O.F_LAYER).reshape(n, n, n).astype(int)
    got = o.read(O.F_XI).reshape(3, n, n, n)
    assert np.array_equal(lay == 0, sel)
    e = (i0, j0, z0 + 1)
    assert lay[e[2], e[1], e[0]] == 1
    exp2, _ = _expected(got, lay, e, 1, n, c, rs_list=(2,))
    exp3, rs = _expected(got, lay, e, 1, n, c)
    exp4, _ = _expected(got, lay, e, 1, n, c, rs_list=(4,))
    assert exp2 is None and rs == 3
    v = got[:, e[2], e[1], e[0]]
    assert np.abs(v - exp3).max() < 1e-12
    assert np.abs(v - exp4).max() > 1e-5  # the 9^3 fit is a different value


# ------------------------------------------------------------------ face stress, manufactured


def _heaviside(phi, eps):
    """eq. sm_heavi."""
    out = np.where(phi <= -eps, 0.0, 1.0)
    mid = np.abs(phi) < eps
    out = np.where(mid, 0.5 * (1 + phi / eps + np.sin(np.pi * phi / eps) / np.pi), out)
    return out


def _continuous_stress(P, c, kappa, R, G, eps, act):
    """The blended solid stress (1 - H(phi_0(xi))) (tau_s + sigma_a) of the continuous map
    xi = x + kappa q(x - c) at points P [3][...]: F = (grad xi)^-1, tau_s = G (F F^T - tr/3 I)
    (SI "Stress calculations"), sigma_a = (3 Z s0 / 2)(e e^T - I/3) with e = F E_X / |F E_X|,
    s0 = A sin(2 pi X / l) at t = 0 (main text "Swimming"; body frame = world frame here)."""
    r = P - np.asarray(c).reshape(3, *([1] * (P.ndim - 1)))
    q = np.stack([r[1] ** 2 - 0.5 * r[2] * r[0], r[2] * r[0] + 0.7 * r[1] ** 2, r[0] ** 2 - r[1] * r[2]])
    xi = P + kappa * q
    Jq = np.zeros((3, 3) + P.shape[1:])  # d q_a / d x_b
    Jq[0, 1] = 2 * r[1]; Jq[0, 2] = -0.5 * r[0]; Jq[0, 0] = -0.5 * r[2]
    Jq[1, 2] = r[0]; Jq[1, 0] = r[2]; Jq[1, 1] = 1.4 * r[1]
    Jq[2, 0] = 2 * r[0]; Jq[2, 1] = -r[2]; Jq[2, 2] = -r[1]
    A = np.eye(3).reshape(3, 3, *([1] * (P.ndim - 1))) + kappa * Jq
    Am = np.moveaxis(A, (0, 1), (-2, -1))
    F = np.linalg.inv(Am)
    B = F @ np.swapaxes(F, -1, -2)
    tr = np.trace(B, axis1=-2, axis2=-1)
    tau = G * (B - tr[..., None, None] / 3.0 * np.eye(3))
    if act is not None:
        A_amp, ell = act
        Xb, Zb = xi[0] - c[0], xi[2] - c[2]
        s0 = A_amp * np.sin(2 * np.pi * Xb / ell)
        f = F[..., :, 0]
        e = f / np.linalg.norm(f, axis=-1, keepdims=True)
        tau = tau + (1.5 * Zb * s0)[..., None, None] * (e[..., :, None] * e[..., None, :] - np.eye(3) / 3.0)
    phi = np.linalg.norm(xi - np.asarray(c).reshape(3, *([1] * (P.ndim - 1))), axis=0) - R
    w = 1.0 - _heaviside(phi, eps)
    return w[..., None, None] * tau


def _divergence(P, c, kappa, R, G, eps, act, delta=2e-3):
    """div of the continuous stress at points P by fourth-order central differences."""
    div = np.zeros_like(P)
    for b in range(3):
        vals = []
        for s in (-2, -1, 1, 2):
            Q = P.copy()
            Q[b] += s * delta
            vals.append(_continuous_stress(Q, c, kappa, R, G, eps, act)[..., :, b])
        d = (vals[0] - 8 * vals[1] + 8 * vals[2] - vals[3]) / (12 * delta)
        div += np.moveaxis(d, -1, 0)
    return div


def _oracle_divtau(n, c, kappa, R, G, eps, act):
    sc = S._box(n, periodic=False)
    sc.update(mu=0.01, eps_h=eps * n, dt=0.2 / n)
    sol = S.solid(S.SPHERE, c, (R, R, R), G=G, mu_a=0.01)
    if act is not None:
        sol.update(active_A=act[0], active_omega=2 * np.pi, active_len=act[1])
    sc["solids"] = [sol]
    o = O.Oracle(sc)
    P = _grid_points(n)
    r = P - np.asarray(c)[:, None, None, None]
    q = np.stack([r[1] ** 2 - 0.5 * r[2] * r[0], r[2] * r[0] + 0.7 * r[1] ** 2, r[0] ** 2 - r[1] * r[2]])
    o.write(O.F_XI, (P + kappa * q).reshape(-1))
    lay = o.read(O.F_LAYER).reshape(n, n, n)
    assert o.step(1) == 0, o.error()
    div = o.read(O.F_DIVTAU_N).reshape(3, n, n, n)
    # cells whose whole 3^3 neighbourhood holds the written map (no extrapolated values)
    inner = np.ones((n, n, n), bool)
    l0 = lay == 0
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                inner &= np.roll(l0, (dk, dj, di), axis=(0, 1, 2))
    inner[[0, -1], :, :] = inner[:, [0, -1], :] = inner[:, :, [0, -1]] = False
    return P, div, inner


@pytest.mark.parametrize("act", [None, (0.5, 0.5)], ids=["passive", "active"])
def test_face_stress_divergence_converges_at_second_order(act):
    c, kappa, R, G, eps = np.array([0.5, 0.5, 0.5]), 0.4, 0.3, 1.0, 0.12
    errs, blur_cells = [], []
    for n in (24, 32, 48):
        P, div, inner = _oracle_divtau(n, c, kappa, R, G, eps, act)
        r = P - c[:, None, None, None]
        xi = P + kappa * np.stack([r[1] ** 2 - 0.5 * r[2] * r[0], r[2] * r[0] + 0.7 * r[1] ** 2,
                                   r[0] ** 2 - r[1] * r[2]])
        phi = np.linalg.norm(xi - c[:, None, None, None], axis=0) - R
        # the same region of the body at every resolution, phi_0(xi) <= -0.08, where every face
        # stencil stays inside the written map (checked by `inner`); relative L2 error there
        sel = inner & (phi <= -0.08)
        assert np.array_equal(sel, phi <= -0.08)
        ref = _divergence(P[:, sel], c, kappa, R, G, eps, act)
        errs.append(np.linalg.norm(div[:, sel] - ref) / np.linalg.norm(ref))
        blur_cells.append(int(np.count_nonzero(sel & (phi > -eps))))
    orders = [np.log(errs[q] / errs[q + 1]) / np.log(m / n) for q, (n, m) in enumerate([(24, 32), (32, 48)])]
    # the blend is exercised (cells inside the blur zone), and the error falls at second order
    assert min(blur_cells) > 100, blur_cells
    assert errs[-1] < 6e-3, errs
    assert all(1.8 < q < 2.3 for q in orders), (errs, orders)
