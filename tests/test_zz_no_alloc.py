"""rmt_extrapolate_noalloc against the grid API's extrapolation.

Some callers cannot allocate device memory while this step runs (their own pool holds the
memory budget, or a cudaMalloc would synchronise their pipeline).  rmt_extrapolate_noalloc
serves them: it runs the reference-map extrapolation on buffers the caller owns, with its
scratch in a fixed static device array.  Its result must equal what the grid API computes
(rmt_write_fields of a reference map re-runs the same extrapolation), on two calls in a row,
since the calls share that scratch.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2104_00095_gb300 import rmt, scenes as S
from parity_util import needs_gpu, rel_l2

pytestmark = [pytest.mark.gpu, needs_gpu]


def _scene():
    n = (36, 40, 44)
    sc = S._box(44, periodic=False)
    sc.update(n=n, hi=(36 / 44, 40 / 44, 1.0), dt=0.2 / 44)
    sc["solids"] = [S.solid(S.ELLIPSOID, (0.4, 0.45, 0.5), (0.2, 0.12, 0.15),
                            S.random_rotation(np.random.default_rng(21)), rho_s=1.2, G=0.5)]
    return sc


def _reference_map(sc):
    """A smooth, non-affine map with candidates only near the body (NaN elsewhere)."""
    nx, ny, nz = sc["n"]
    h = 1.0 / 44
    x, y, z = ((np.arange(m) + 0.5) * h for m in (nx, ny, nz))
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    xi = np.stack([X + 0.01 * np.sin(3 * Y), Y - 0.008 * np.cos(2 * Z), Z + 0.006 * np.sin(4 * X)])
    far = (X - 0.4) ** 2 + (Y - 0.45) ** 2 + (Z - 0.5) ** 2 > 0.3**2
    xi[:, far] = np.nan
    return xi.reshape(-1)


def test_noalloc_extrapolation_matches_the_grid_api_on_two_calls():
    torch = pytest.importorskip("torch")
    sc = _scene()
    xi_in = _reference_map(sc)
    N = int(np.prod(sc["n"]))
    g = rmt.Grid(sc)  # FP64 grid: the same kernels in the same precision
    g.write(rmt.RMT_F_XI, xi_in)
    ref_xi, ref_phi = g.read(rmt.RMT_F_XI), g.read(rmt.RMT_F_PHI)
    ref_lay = g.read(rmt.RMT_F_LAYER)
    g.close()
    assert np.count_nonzero(ref_lay >= 1) > 1000

    L = rmt.load()
    d_in = torch.tensor(xi_in, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    gd = rmt.make_grid_desc(sc)
    sd = rmt.make_solid_desc(sc["solids"][0])
    for call in range(2):
        d_xi = torch.full((3 * N,), 7.0, dtype=torch.float64, device="cuda")
        d_phi = torch.full((N,), 7.0, dtype=torch.float64, device="cuda")
        d_lay = torch.full((N,), 7, dtype=torch.int8, device="cuda")
        rc = L.rmt_extrapolate_noalloc(C.byref(gd), C.byref(sd), C.c_void_p(d_in.data_ptr()),
                                       C.c_void_p(d_xi.data_ptr()), C.c_void_p(d_phi.data_ptr()),
                                       C.c_void_p(d_lay.data_ptr()), C.c_void_p(stream))
        assert rc == rmt.RMT_OK, f"call {call}: status {rc}"
        torch.cuda.synchronize()
        lay = d_lay.cpu().numpy().astype(np.float64)
        assert np.array_equal(lay, ref_lay), f"call {call}: layer labels differ"
        assert rel_l2(d_xi.cpu().numpy(), ref_xi) <= 1e-10, f"call {call}"
        assert rel_l2(d_phi.cpu().numpy(), ref_phi) <= 1e-10, f"call {call}"


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    sc = _scene()
    sc.update(n=(130, 130, 130), hi=(1.0, 1.0, 1.0))  # 2,197,000 cells > 2^21
    L = rmt.load()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    rc = L.rmt_extrapolate_noalloc(C.byref(rmt.make_grid_desc(sc)), C.byref(rmt.make_solid_desc(sc["solids"][0])),
                                   p, p, p, p, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == rmt.RMT_EINVAL
