"""Seeded synthetic scenes shaped like the paper's examples (arXiv 2104.00095).

This module only draws inputs: grid sizes, boundary conditions, material constants and
body placements.  It holds none of the method's arithmetic, so that both the CUDA path
and the FP64 oracle can be fed from it.  Every generator uses numpy's PCG64 with the
seed it is given.

Scene dict keys: n, lo, hi, bc (6 ints: -x,+x,-y,+y,-z,+z), wall_u (6x3), rho_f, mu,
eps_h, band_layers, dt (0 = library picks), gravity, steps, precision ("fp64" or
"fp32"), solids (list of dicts: shape, center, semi_axes, rot 3x3 body->world,
rho_s, G, mu_a, gamma_t, active_A, active_omega, active_len).
"""
from __future__ import annotations

import numpy as np

NOSLIP, PERIODIC = 0, 1
SPHERE, ELLIPSOID = 0, 1


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform rotation on SO(3) from a uniform unit quaternion (Shoemake 1992)."""
    u1, u2, u3 = rng.random(3)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    w, x, y, z = (a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3))
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _box(n: int, periodic: bool, lid: float = 0.0) -> dict:
    bc = [PERIODIC] * 6 if periodic else [NOSLIP] * 6
    wall_u = [[0.0, 0.0, 0.0] for _ in range(6)]
    if lid and not periodic:
        wall_u[5] = [lid, 0.0, 0.0]  # the +z face moves in +x
    return dict(n=(n, n, n), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=bc, wall_u=wall_u,
                rho_f=1.0, mu=0.01, eps_h=1.5, band_layers=4, dt=0.0,
                gravity=(0.0, 0.0, 0.0), solids=[], steps=1, precision="fp64")


def solid(shape=SPHERE, center=(0.5, 0.5, 0.5), semi_axes=(0.2, 0.2, 0.2), rot=None, rho_s=1.0,
          G=0.1, mu_a=0.01, gamma_t=0.0, active_A=0.0, active_omega=0.0, active_len=1.0, rep_A=0.0) -> dict:
    return dict(shape=shape, center=tuple(float(c) for c in center),
                semi_axes=tuple(float(a) for a in semi_axes),
                rot=np.eye(3) if rot is None else np.asarray(rot, dtype=np.float64),
                rho_s=float(rho_s), G=float(G), mu_a=float(mu_a), gamma_t=float(gamma_t),
                active_A=float(active_A), active_omega=float(active_omega),
                active_len=float(active_len), rep_A=float(rep_A))


def cavity_sphere(n: int = 32, steps: int = 20, precision: str = "fp64") -> dict:
    """Lid-driven cavity with one soft sphere (main text, "Lid-driven cubic cavity with a
    sphere"): unit box, lid speed 1 on z=1, rho=1, mu=0.01, R=0.2 at (0.6,0.5,0.5), G=0.1,
    mu_a=0.01, eps=1.5h, four layers, dt=0.2h."""
    s = _box(n, periodic=False, lid=1.0)
    s.update(mu=0.01, dt=0.2 / n, steps=steps, precision=precision)
    s["solids"] = [solid(SPHERE, (0.6, 0.5, 0.5), (0.2, 0.2, 0.2), rho_s=1.0, G=0.1, mu_a=0.01)]
    return s


def _place(rng, radii, n, periodic, margin_cells, band, tries=200000):
    """Rejection placement of bounding spheres (no overlap; wall margin on walled boxes)."""
    h = 1.0 / n
    centers = []
    for r in radii:
        for _ in range(tries):
            if periodic:
                c = rng.random(3)
            else:
                m = r + (band + 1 + margin_cells) * h
                if m >= 0.5:
                    raise ValueError("body too large for the box")
                c = m + (1.0 - 2.0 * m) * rng.random(3)
            ok = True
            for c2, r2 in centers:
                d = c - c2
                if periodic:
                    d -= np.round(d)
                if np.linalg.norm(d) < r + r2:
                    ok = False
                    break
            if ok:
                centers.append((c, r))
                break
        else:
            raise RuntimeError("placement failed; lower the body count or sizes")
    return [c for c, _ in centers]


def settling(n: int = 128, nbodies: int = 20, steps: int = 200, seed: int = 1002,
             precision: str = "fp64") -> dict:
    """Settling mixture (shape of the main text's 150-ellipsoid run): no-slip unit box,
    gravity -1 in z, rho_f=1, mu=0.02, ellipsoids with semi-axes U[0.06,0.12], uniform
    orientations, half heavy (1.5) and half buoyant (0.5), G=0.5, mu_a=mu."""
    rng = _rng(seed)
    s = _box(n, periodic=False)
    s.update(mu=0.02, gravity=(0.0, 0.0, -1.0), steps=steps, precision=precision)
    axes = [rng.uniform(0.06, 0.12, size=3) for _ in range(nbodies)]
    eps = 1.5 / n
    centers = _place(rng, [a.max() + eps for a in axes], n, False, 0, s["band_layers"])
    for b in range(nbodies):
        rho_s = 1.5 if b < nbodies // 2 else 0.5
        s["solids"].append(solid(ELLIPSOID, centers[b], axes[b], random_rotation(rng), rho_s=rho_s,
                                 G=0.5, mu_a=0.02))
    return s


def swimmers(n: int = 256, nbodies: int = 8, steps: int = 500, seed: int = 1003,
             precision: str = "fp32") -> dict:
    """Active-stress swimmers in a triply periodic unit box (shape of the main text's
    "Swimming" section): ellipsoids (0.15,0.04,0.04), G=1, mu=mu_a=0.01, rho=1, active
    amplitude A=0.5, omega=2 pi, wavelength = body length 0.3."""
    rng = _rng(seed)
    s = _box(n, periodic=True)
    s.update(mu=0.01, steps=steps, precision=precision)
    axes = np.array([0.15, 0.04, 0.04])
    eps = 1.5 / n
    centers = _place(rng, [axes.max() + eps] * nbodies, n, True, 0, s["band_layers"])
    for b in range(nbodies):
        s["solids"].append(solid(ELLIPSOID, centers[b], axes, random_rotation(rng), rho_s=1.0, G=1.0,
                                 mu_a=0.01, active_A=0.5, active_omega=2 * np.pi,
                                 active_len=2 * axes[0]))
    return s


def batched(nsims: int = 64, steps: int = 100, seed: int = 1004, sizes=(32, 48, 64, 96, 128),
            precision: str = "fp32") -> list:
    """Batch of independent lid-driven cavities, each with 1-6 soft spheres (radii U[0.08,0.2],
    densities U[0.5,1.5], shear moduli U[0.05,1])."""
    rng = _rng(seed)
    out = []
    for _ in range(nsims):
        n = int(rng.choice(sizes))
        s = _box(n, periodic=False, lid=1.0)
        s.update(mu=0.01, steps=steps, precision=precision)
        nb = int(rng.integers(1, 7))
        # rejection: non-overlapping spheres (blur width apart) one cell inside the walls; a
        # draw of radii that cannot be placed is drawn again
        for _attempt in range(100):
            radii = rng.uniform(0.08, 0.2, size=nb)
            try:
                centers = _place(rng, [r + 1.5 / n for r in radii], n, False, 0, 0, tries=2000)
                break
            except RuntimeError:
                continue
        else:
            raise RuntimeError("batched scene: no placement found")
        for b in range(nb):
            s["solids"].append(solid(SPHERE, centers[b], (radii[b],) * 3, rho_s=rng.uniform(0.5, 1.5),
                                     G=rng.uniform(0.05, 1.0), mu_a=0.01))
        out.append(s)
    return out


def serving_stream(njobs: int = 32, rate: float = 4.0, seed: int = 1005, sizes=range(48, 193, 16),
                   steps=(100, 2000), precision: str = "fp32") -> list:
    """Poisson arrivals of settling- or swimmer-like jobs with 1-10 bodies; returns a list of
    (arrival_time_s, scene)."""
    rng = _rng(seed)
    t = 0.0
    out = []
    sizes = list(sizes)
    for j in range(njobs):
        t += rng.exponential(1.0 / rate)
        n = int(rng.choice(sizes))
        nb = int(rng.integers(1, 11))
        st = int(rng.integers(steps[0], steps[1] + 1))
        sub = int(rng.integers(0, 2**31 - 1))
        if rng.random() < 0.5:
            sc = settling(n=n, nbodies=nb, steps=st, seed=sub, precision=precision)
        else:
            sc = swimmers(n=n, nbodies=nb, steps=st, seed=sub, precision=precision)
        out.append((t, sc))
    return out


def scaled(scene: dict, n: int) -> dict:
    """The same scene on an n^3 grid (bodies and constants unchanged; dt re-picked unless the
    scene fixes it in units of h)."""
    s = dict(scene)
    s["n"] = (n, n, n)
    s["solids"] = [dict(b) for b in scene["solids"]]
    if scene.get("dt", 0.0) > 0.0:
        s["dt"] = scene["dt"] * scene["n"][0] / n
    return s


# Table str_params of the SI ("Pre-stretched sphere"): mu, rho_s / rho_f, R, G per case
STR_PARAMS = {
    "A1": (0.005, 1.0, 0.2, 0.25), "A2": (0.01, 1.0, 0.2, 1.0), "A3": (0.005, 1.0, 0.1, 1.0),
    "A4": (0.0075, 1.0, 0.3, 0.25), "B1": (0.005, 1.0, 0.1, 0.25), "B2": (0.02, 1.0, 0.2, 2.5),
    "B3": (0.005, 1.0, 0.3, 0.25), "C1": (0.005, 0.5625, 4.0 / 15.0, 0.25), "C2": (0.005, 2.25, 2.0 / 15.0, 0.25),
}


def prestretched_sphere(n: int = 32, case: str = "A2", dt: float = 0.0, precision: str = "fp64") -> dict:
    """Pre-stretched sphere (SI "Pre-stretched sphere"; Table str_params): periodic unit box,
    rho_f = 1, one neo-Hookean sphere of radius R at the centre with mu_a = mu and gamma_t = 0,
    released from rest at t = 0 in a volume-preserving stretch (see prestretch_xi).  The
    scene's sphere is the reference (unstretched) body."""
    mu, rs, R, G = STR_PARAMS[case]
    s = _box(n, periodic=True)
    s.update(mu=mu, dt=dt, precision=precision)
    s["solids"] = [solid(SPHERE, (0.5, 0.5, 0.5), (R, R, R), rho_s=rs, G=G, mu_a=mu)]
    return s


def prestretch_xi(scene: dict, lam: float = 1.21) -> np.ndarray:
    """Initial reference map of a body stretched by lam along x and by 1/sqrt(lam) along y and
    z about its centre: xi = c + diag(1/lam, sqrt(lam), sqrt(lam)) (x - c) at every cell centre
    ([3][nz][ny][nx], the layout of the field reads and writes).  The SI text gives lam = 1.21;
    the caption of its figure says 1.44."""
    n = scene["n"]
    c = np.asarray(scene["solids"][0]["center"])
    h = (np.asarray(scene["hi"]) - np.asarray(scene["lo"])) / np.asarray(n)
    ax = [scene["lo"][d] + (np.arange(n[d]) + 0.5) * h[d] for d in range(3)]
    Z3, Y3, X3 = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    inv = (1.0 / lam, np.sqrt(lam), np.sqrt(lam))
    return np.stack([c[0] + inv[0] * (X3 - c[0]), c[1] + inv[1] * (Y3 - c[1]),
                     c[2] + inv[2] * (Z3 - c[2])]).reshape(-1)


def stokes_sphere(n: int = 48, R: float = 0.1, mu: float = 0.05, rho_s: float = 1.5, G: float = 1.0,
                  dt: float = 0.0, precision: str = "fp64") -> dict:
    """One heavy sphere in a triply periodic unit box under gravity -1 in z (a simple cubic
    array of settling spheres), set up like the main text's settling runs ("Settling sphere in
    a square cylinder"): rho_f = 1, mu_a = mu, gamma_t = 0, a blur half-width of h/2 and G large
    enough that the sphere stays nearly rigid."""
    s = _box(n, periodic=True)
    s.update(mu=mu, dt=dt, gravity=(0.0, 0.0, -1.0), precision=precision, eps_h=0.5)
    s["solids"] = [solid(SPHERE, (0.5, 0.5, 0.5), (R, R, R), rho_s=rho_s, G=G, mu_a=mu)]
    return s
