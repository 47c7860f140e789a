"""Host-side checks of the index arithmetic and staging schedules of two tiled multigrid kernels
(csrc/rmt_mg.cu), restated in Python thread by thread:

* the fused red-black sweep (k_rbgs_sweep): a block marches a z-chunk of a 64 x 8 tile, staging
  x, rho and b planes through a ring of cp.async slots, updating the first colour on the tile and
  a one-cell ring, then the second colour one plane behind.  The emulation checks every shared
  read against the plane it must hold and the copy group it must have waited for, checks that
  no thread reads or writes what another thread writes between two barriers, that every cell is
  written exactly once and in bounds, and that the result equals two in-place colour passes of
  the 7-point operator (walls, periodic axes, partial tiles, tiles wider than the grid);
* the FE tile's 16-byte staging (k_fe_tile, VEC): one chunk per thread and plane covers every
  shared element the stencil window reads, with sources in bounds and 16-byte aligned.

These run on the CPU; the kernels themselves are compared with the oracle by the GPU tests."""
import itertools

import numpy as np
import pytest

# ------------------------------------------------------------------ fused red-black sweep
GX, GY = 64, 8
GW, GH = GX + 8, GY + 4
GP = GW * GH
GR = 6
GCH = GW // 4
GNCH = 3 * GH * GCH
GT = 256


def _wrap(v, n, per):
    if per:
        return v % n
    return v if 0 <= v < n else -1


def _two_colour_passes(x, b, rho, n, per, c0, w, ih2):
    """Two in-place colour passes of red-black Gauss-Seidel on the 7-point operator with face
    coefficient 2/(rho_a + rho_b) (no face across a wall)."""
    x = x.copy()
    nx, ny, nz = n
    for col in (c0, 1 - c0):
        xo = x.copy()  # a colour's cells read only the other colour
        for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
            if (i + j + k) & 1 != col:
                continue
            off = dg = 0.0
            for d, s in ((0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1)):
                q = [i, j, k]
                q[d] = _wrap(q[d] + s, n[d], per[d])
                if q[d] < 0:
                    continue
                beta = 2.0 / (rho[k, j, i] + rho[q[2], q[1], q[0]])
                off += beta * xo[q[2], q[1], q[0]]
                dg += beta
            ax = (dg * xo[k, j, i] - off) * ih2
            diag = dg * ih2
            if diag > 0:
                x[k, j, i] = xo[k, j, i] + w * (b[k, j, i] - ax) / diag
    return x


class _Interval:
    """Shared-memory accesses between two barriers, by thread."""

    def __init__(self):
        self.r, self.w = {}, {}

    def read(self, t, d):
        self.r.setdefault(d, set()).add(t)

    def write(self, t, d):
        self.w.setdefault(d, set()).add(t)

    def close(self):
        for d, ws in self.w.items():
            assert len(ws) == 1, f"shared element {d} written by threads {sorted(ws)[:4]}"
            others = self.r.get(d, set()) - ws
            assert not others, f"shared element {d} written by {ws} and read by {sorted(others)[:4]}"
        self.r.clear()
        self.w.clear()


def _emulate_sweep(x, b, rho, n, per, c0, w, ih2, zc):
    nx, ny, nz = n
    pst, ntot = nx * ny, nx * ny * nz
    src = [x.ravel(), rho.ravel(), b.ravel()]
    xout = np.full(ntot, np.nan)
    written = np.zeros(ntot, int)
    perx, pery, perz = per
    for bz, by, bx in itertools.product(range(-(-nz // zc)), range(-(-ny // GY)), range(-(-nx // GX))):
        i0, j0, k0 = bx * GX, by * GY, bz * zc
        k1 = min(k0 + zc, nz)
        sm = np.full((3 * GR + 3) * GP, np.nan)
        tag = np.full(sm.size, -10**6)
        grp = np.full(sm.size, -1)
        state = {"cur": 0, "done": -1}
        iv = _Interval()
        chunks = []  # per thread: (array, shared offset in slot 0, in-plane source or None)
        for t in range(GT):
            mine = []
            for s in range(3):
                c = t + GT * s
                if c >= GNCH:
                    continue
                a, rc = divmod(c, GH * GCH)
                r, cc = divmod(rc, GCH)
                gy, gx = _wrap(j0 - 2 + r, ny, pery), _wrap(i0 - 4 + 4 * cc, nx, perx)
                mine.append((a, a * GR * GP + r * GW + 4 * cc, gy * nx + gx if gy >= 0 and gx >= 0 else None))
            chunks.append(mine)

        def adv(s, d, m):
            return s + d - m if s + d >= m else s + d

        def issue(p, slot):
            assert slot == (p - k0 + 2) % GR
            pz = (p + nz if perz else -1) if p < 0 else ((p - nz if perz else -1) if p >= nz else p)
            for t in range(GT):
                for a, soff, off in chunks[t]:
                    d = soff + slot * GP
                    assert 0 <= d and d + 4 <= 3 * GR * GP and d % 4 == 0
                    if pz >= 0 and off is not None:
                        g = pz * pst + off
                        assert 0 <= g and g + 4 <= ntot and g % 4 == 0
                        sm[d:d + 4] = src[a][g:g + 4]
                    else:
                        sm[d:d + 4] = 0.0
                    tag[d:d + 4] = p
                    grp[d:d + 4] = state["cur"]
                    for u in range(4):
                        iv.write(t, d + u)

        def commit():
            state["cur"] += 1

        def wait(keep):
            state["done"] = state["cur"] - 1 - keep

        def staged(t, a, base, o, p):
            assert base == (a * GR + (p - k0 + 2) % GR) * GP and 0 <= o < GP
            d = base + o
            assert tag[d] == p, ("stale plane", a, p, tag[d])
            assert grp[d] <= state["done"], ("copy group not waited for", p)
            iv.read(t, d)
            return sm[d]

        def red(t, base, o, p):
            assert base == (3 * GR + (p - k0 + 3) % 3) * GP and 0 <= o < GP
            d = base + o
            assert tag[d] == p, ("stale first-colour plane", p, tag[d])
            iv.read(t, d)
            return sm[d]

        def put(t, base, o, p, v):
            assert base == (3 * GR + (p - k0 + 3) % 3) * GP and 0 <= o < GP
            sm[base + o] = v
            tag[base + o] = p
            iv.write(t, base + o)

        def update(rc, rn, xn, xc, bc):
            off = dg = 0.0
            for f in range(6):
                r = 1.0 / (rc + rn[f]) if rn[f] > 0 else 0.0
                off += r * xn[f]
                dg += r
            ax = (dg * xc - off) * 2 * ih2
            diag = dg * 2 * ih2
            return xc + w * (bc - ax) / diag if diag > 0 else xc

        def store(q, nbase):
            for t in range(GX * GY // 4):
                r, cc = divmod(t, GX // 4)
                gj, gi = j0 + r, i0 + 4 * cc
                if gj < ny and gi < nx:
                    for u in range(4):
                        v = red(t, nbase, (r + 2) * GW + 4 + 4 * cc + u, q)
                        g = q * pst + gj * nx + gi + u
                        assert 0 <= g < ntot
                        xout[g] = v
                        written[g] += 1

        lanes = []
        for t in range(GT):
            lane, wp = t & 31, t >> 5
            pp, jj = 16 * (wp & 1) + (lane & 15), 2 * (wp >> 1) + (lane >> 4)
            has_ring, hp, hj = t < GX + 2 * GY, 0, 0
            if t < GX:
                hp, hj = 16 * (t >> 5) + (t & 15), GY if t & 16 else -1
            elif has_ring:
                r = t - GX
                hp, hj = (-1, r) if r < GY else (GX // 2, r - GY)
            lanes.append((pp, jj, has_ring, hp, hj))

        issue(k0 - 2, 0)
        issue(k0 - 1, 1)
        issue(k0, 2)
        commit()
        issue(k0 + 1, 3)
        commit()
        sq, rq = 1, 2
        for q in range(k0 - 1, k1 + 1):
            wait(1)
            iv.close()  # barrier
            if q + 3 <= k1 + 1:
                issue(q + 3, adv(sq, 3, GR))
            commit()
            sm1, sm2, sp1 = adv(sq, GR - 1, GR), adv(sq, GR - 2, GR), adv(sq, 1, GR)
            X0, Xm1, Xp1 = sq * GP, sm1 * GP, sp1 * GP
            R0, Rm1, Rm2, Rp1 = (GR + sq) * GP, (GR + sm1) * GP, (GR + sm2) * GP, (GR + sp1) * GP
            B0, Bm1 = (2 * GR + sq) * GP, (2 * GR + sm1) * GP
            N0, Nm1, Nm2 = (3 * GR + rq) * GP, (3 * GR + adv(rq, 2, 3)) * GP, (3 * GR + adv(rq, 1, 3)) * GP
            if q - 2 >= k0:
                store(q - 2, Nm2)
            zin = perz or 0 <= q < nz
            carry = []
            for t, (pp, jj, has_ring, hp, hj) in enumerate(lanes):
                for first_pair, (p2, jr) in enumerate([(pp, jj)] + ([(hp, hj)] if has_ring else [])):
                    e = (c0 + j0 + jr + q) & 1
                    o = (jr + 2) * GW + 4 + 2 * p2 + e
                    rn = [staged(t, 1, R0, o - 1, q), staged(t, 1, R0, o + 1, q), staged(t, 1, R0, o - GW, q),
                          staged(t, 1, R0, o + GW, q), staged(t, 1, Rm1, o, q - 1), staged(t, 1, Rp1, o, q + 1)]
                    xn = [staged(t, 0, X0, o - 1, q), staged(t, 0, X0, o + 1, q), staged(t, 0, X0, o - GW, q),
                          staged(t, 0, X0, o + GW, q), staged(t, 0, Xm1, o, q - 1), staged(t, 0, Xp1, o, q + 1)]
                    rc, xc = staged(t, 1, R0, o, q), staged(t, 0, X0, o, q)
                    v = update(rc, rn, xn, xc, staged(t, 2, B0, o, q))
                    ci = o - (jr + 2) * GW - 4
                    real = zin and (pery or 0 <= j0 + jr < ny) and (perx or 0 <= i0 + ci < nx)
                    v = v if real else 0.0
                    put(t, N0, o, q, v)
                    if first_pair == 0:
                        carry.append((o, rc, rn[4], xn[4], v))  # reused by the second colour
            iv.close()  # barrier
            if q - 1 >= k0:
                for t, (pp, jj, _, _, _) in enumerate(lanes):
                    o, rc, rlo, xlo, vq = carry[t]
                    # the second colour's cell at plane q-1 is the first colour's cell at plane q
                    assert o == (jj + 2) * GW + 4 + 2 * pp + ((1 - c0 + j0 + jj + q - 1) & 1)
                    if j0 + jj < ny and i0 + o - (jj + 2) * GW - 4 < nx:
                        rn = [staged(t, 1, Rm1, o - 1, q - 1), staged(t, 1, Rm1, o + 1, q - 1),
                              staged(t, 1, Rm1, o - GW, q - 1), staged(t, 1, Rm1, o + GW, q - 1),
                              staged(t, 1, Rm2, o, q - 2), rc]
                        xn = [red(t, Nm1, o - 1, q - 1), red(t, Nm1, o + 1, q - 1), red(t, Nm1, o - GW, q - 1),
                              red(t, Nm1, o + GW, q - 1), red(t, Nm2, o, q - 2), vq]
                        put(t, Nm1, o, q - 1, update(rlo, rn, xn, xlo, staged(t, 2, Bm1, o, q - 1)))
            sq, rq = adv(sq, 1, GR), adv(rq, 1, 3)
        wait(0)
        iv.close()
        if k1 - 1 >= k0:
            store(k1 - 1, (3 * GR + adv(rq, 1, 3)) * GP)
    assert (written == 1).all(), (written.min(), written.max())
    return xout.reshape(nz, ny, nx)


@pytest.mark.parametrize("n,per,zc", [
    ((64, 8, 6), (1, 1, 1), 4),    # periodic, one tile, two chunks
    ((64, 12, 5), (0, 0, 0), 2),   # walls, partial tile along y, three chunks
    ((68, 8, 4), (0, 1, 0), 3),    # walls along x with a partial tile, periodic y
    ((8, 8, 4), (1, 1, 1), 1),     # periodic grid narrower than the tile (wrapped images)
])
@pytest.mark.parametrize("c0", [0, 1])
def test_fused_sweep_schedule_equals_two_colour_passes(n, per, zc, c0):
    rng = np.random.default_rng(sum(n) + 10 * zc + c0)
    nx, ny, nz = n
    x = rng.standard_normal((nz, ny, nx))
    b = rng.standard_normal((nz, ny, nx))
    rho = rng.uniform(0.5, 1.5, (nz, ny, nx))
    ref = _two_colour_passes(x, b, rho, n, per, c0, 1.0, 4.0)
    got = _emulate_sweep(x, b, rho, n, per, c0, 1.0, 4.0, zc)
    assert np.abs(got - ref).max() < 1e-12


# ------------------------------------------------------------------ FE tile, 16-byte staging
FX, FY = 32, 8
VXC, VBC, VRC = (FX + 8) // 4, (FX + 4) // 4, FX // 4
VNX, VNR, VNB = (FY + 2) * VXC, FY * VRC, (FY + 1) * VBC


@pytest.mark.parametrize("nn,ny,i0,j0", [(256, 256, 224, 248), (48, 40, 32, 32), (8, 8, 0, 0)])
def test_fe_tile_16_byte_staging_covers_the_window(nn, ny, i0, j0):
    """Periodic x (nodes = cells = nn along x, nn % 4 == 0); a wall or period along y with ny
    nodes.  Chunks: x rows j0-1 .. j0+FY with nodes i0-4 .. i0+FX+3, b rows j0 .. j0+FY-1 with
    nodes i0 .. i0+FX-1, beta rows j0-1 .. j0+FY-1 with cells i0-4 .. i0+FX-1."""
    assert nn % 4 == 0 and VNX + VNR + VNB <= FX * FY
    cover = {"x": np.zeros((FY + 2, FX + 8), int), "b": np.zeros((FY, FX), int), "beta": np.zeros((FY + 1, FX + 4), int)}
    for t in range(FX * FY):
        if t < VNX:
            r, cc = divmod(t, VXC)
            arr, src_col = "x", (i0 - 4 + 4 * cc) % nn
        elif t < VNX + VNR:
            r, cc = divmod(t - VNX, VRC)
            arr, src_col = "b", (i0 + 4 * cc) % nn
        elif t < VNX + VNR + VNB:
            r, cc = divmod(t - VNX - VNR, VBC)
            arr, src_col = "beta", (i0 - 4 + 4 * cc) % nn
        else:
            continue
        assert src_col % 4 == 0 and src_col + 4 <= nn  # one aligned 16-byte chunk of a row
        cover[arr][r, 4 * cc:4 * cc + 4] += 1
    for a in cover.values():
        assert (a == 1).all()  # every staged element exactly once
    # the window of thread (tx, ty): x nodes i-1..i+1, j-1..j+1 at columns tx+3.., rows ty..;
    # beta cells i-1..i, j-1..j at columns tx+3.., rows ty..; b at (ty, tx)
    for ty, tx in itertools.product(range(FY), range(FX)):
        for c, a in itertools.product(range(3), range(3)):
            assert 0 <= ty + c < FY + 2 and 0 <= tx + 3 + a < FX + 8
            assert (i0 - 4 + tx + 3 + a) == i0 + tx - 1 + a  # the staged column holds node i-1+a
        for c, a in itertools.product(range(2), range(2)):
            assert 0 <= ty + c < FY + 1 and 0 <= tx + 3 + a < FX + 4
            assert (i0 - 4 + tx + 3 + a) == i0 + tx - 1 + a  # cell i-1+a
