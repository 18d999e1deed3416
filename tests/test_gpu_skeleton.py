"""GPU parity of the two global phases of D8 accumulation on DEMs with long
rivers: the cell walkers and the tile-skeleton solve (FR_GLOBAL_WALKERS /
FR_GLOBAL_SKELETON, and the default choice between them), against the CPU
oracle.

Inputs with long rivers: fractal DEMs after the oracle's depression filling
(every interior cell drains to the edge, as on the paper's filled DEM, Sec. 4),
and planes, where every row is one chain across all tiles.  Bars: areas
bit-exact; water within 1e-6 relative per cell (leading word) and 1e-10 for
the two-float pair; identical bits on repeated calls.
"""
import numpy as np
import pytest

import oracle
from paper_2606_12800_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_W = 1e-6
WALK, SKEL = _lib.FR_GLOBAL_WALKERS, _lib.FR_GLOBAL_SKELETON
VARIANTS = [SKEL, WALK, 0]


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_12800_gb300 import api as a
    return a


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def relerr(got, ref):
    ref = np.asarray(ref, np.float64)
    got = np.asarray(got, np.float64)
    den = np.where(ref == 0, 1.0, np.abs(ref))
    return np.max(np.abs(got - ref) / den) if ref.size else 0.0


def _check(api, z, flags, rain, variants=VARIANTS):
    d_ref, w_ref, _, order = oracle.route_d8(z, 30.0, rain, flags)
    _, a_ref = oracle.accumulate_d8(d_ref, order, None)
    zt = cuda(z)
    rt = None if rain is None else cuda(rain)
    for v in variants:
        out = api.route_d8(zt, 30.0, rt, flags | v, want_w=True, want_lo=True, want_area=True)
        assert api.get_status() == 0, v
        np.testing.assert_array_equal(out["area"].cpu().numpy().astype(np.uint64), a_ref)
        w, lo = out["w"].cpu().numpy(), out["w_lo"].cpu().numpy()
        assert relerr(w, w_ref) <= RTOL_W, v
        assert relerr(w.astype(np.float64) + lo, w_ref) <= 1e-10, v
        # areas alone: the skeleton's integer solve (chain contraction)
        out = api.route_d8(zt, 30.0, None, flags | v, want_w=False, want_area=True)
        assert api.get_status() == 0, v
        np.testing.assert_array_equal(out["area"].cpu().numpy().astype(np.uint64), a_ref)
    return a_ref


@pytest.mark.parametrize("shape", [(64, 64), (65, 130), (300, 517), (700, 1100)])
@pytest.mark.parametrize("flags", [0, oracle.EDGE_ROUTE, oracle.D8_LOWEST | oracle.EDGE_ROUTE])
def test_filled_dem_both_global_phases(api, shape, flags):
    ny, nx = shape
    z = oracle.fill(inputs.fractal_dem(ny, nx, beta=2.0, tilt=0.01, seed=ny + 3 * nx))
    rain = inputs.rain_field(ny, nx, 4)
    a = _check(api, z, flags, rain)
    if flags == 0 and ny > 2 and nx > 2:
        # filled: the interior drains to the edge, rivers run across many tiles
        assert a.max() > (ny * nx) // 50


@pytest.mark.parametrize("shape", [(64, 64), (5, 700), (130, 1030), (300, 517), (1, 300), (300, 1)])
@pytest.mark.parametrize("flags", [0, oracle.EDGE_ROUTE])
def test_planar_chains_both_global_phases(api, shape, flags):
    ny, nx = shape
    z = inputs.planar_dem(ny, nx, 0.01, 30.0)
    _check(api, z, flags, None)


@pytest.mark.parametrize("shape", [(1, 1), (3, 3), (1, 9), (33, 65), (256, 256), (1500, 2600)])
def test_rough_dem_forced_skeleton(api, shape):
    """Few global cells (or grids too small for the skeleton's scratch, which
    then keep the walkers): the forced skeleton solve is exact too."""
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, seed=5 * ny + nx)
    rain = inputs.rain_field(ny, nx, 6)
    _check(api, z, 0, rain, variants=[SKEL])


def test_filled_benchmark_dem_full_size(api):
    """The 4096^2 D8 benchmark DEM after depression filling (about 5 % of the
    cells global): both global phases and the default against the full oracle,
    areas only and with rain."""
    n = 4096
    z = oracle.fill(inputs.fractal_dem(n, n, beta=2.0, tilt=0.01, seed=1))
    d_ref, _, a_ref, _ = oracle.route_d8(z, 30.0, None)
    zt = cuda(z)
    for v in VARIANTS:
        out = api.route_d8(zt, 30.0, None, v, want_w=False, want_area=True, want_dir=True)
        assert api.get_status() == 0
        np.testing.assert_array_equal(out["dir"].cpu().numpy(), d_ref)
        np.testing.assert_array_equal(out["area"].cpu().numpy().astype(np.uint64), a_ref)
    rain = inputs.rain_field(n, n, 1)
    _, w_ref, _, _ = oracle.route_d8(z, 30.0, rain)
    out = api.route_d8(zt, 30.0, cuda(rain), SKEL, want_w=True, want_area=False)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W


def test_skeleton_is_bit_reproducible(api):
    z = oracle.fill(inputs.fractal_dem(900, 1300, beta=2.0, tilt=0.01, seed=9))
    zt, rt = cuda(z), cuda(inputs.rain_field(900, 1300, 9))
    a = api.route_d8(zt, 30.0, rt, SKEL, want_w=True, want_lo=True, want_area=True)
    for _ in range(3):
        b = api.route_d8(zt, 30.0, rt, SKEL, want_w=True, want_lo=True, want_area=True)
        for k in ("w", "w_lo", "area"):
            assert torch.equal(a[k], b[k]), k
        c = api.route_d8(zt, 30.0, None, SKEL, want_w=False, want_area=True)
        assert torch.equal(a["area"], c["area"])


@pytest.mark.parametrize("variant", [SKEL, WALK])
def test_cycles_report_no_progress(api, variant):
    """Cycles inside one skeleton tile and across the border of two (x = 63 |
    64, y = 127 | 128) leave cells unfinished: FR_ERR_NO_PROGRESS, no hang;
    the same workspace is clean on the next good routing."""
    ny, nx = 200, 300
    d = np.full((ny, nx), oracle.SINK, np.uint8)
    d[10, 10], d[10, 11] = 0, 2          # E <-> W inside a tile
    d[20, 63], d[20, 64] = 0, 2          # across x = 63 | 64
    d[127, 100], d[128, 100] = 3, 1      # S <-> N across y = 127 | 128
    # a long chain feeding a cross-tile cycle, so that it is global
    d[150, 20:150] = 0                   # E along row 150 ...
    d[150, 150], d[150, 151] = 0, 2      # ... into a 2-cycle
    R = api.routing_d8(cuda(d), variant)
    api.accumulate(R, None, want_w=True, want_area=True)
    assert api.get_status() == 5
    api.accumulate(R, None, want_w=False, want_area=True)  # areas alone
    assert api.get_status() == 5
    z = inputs.planar_dem(ny, nx, 0.01, 30.0)
    api.route_d8(cuda(z), 30.0, None, variant)
    assert api.get_status() == 0


def test_eight_donor_lattice_forced_skeleton(api):
    ny, nx = 301, 517
    d = np.full((ny, nx), oracle.SINK, np.uint8)
    to_centre = {(-1, -1): 7, (-1, 0): 3, (-1, 1): 6, (0, -1): 0, (0, 1): 2,
                 (1, -1): 4, (1, 0): 1, (1, 1): 5}
    for cy in range(1, ny - 1, 3):
        for cx in range(1, nx - 1, 3):
            for (dy, dx), k in to_centre.items():
                d[cy + dy, cx + dx] = k
    # and a long chain along row 0 towards +x, crossing every tile
    d[0, :-1] = 0
    rain = inputs.rain_field(ny, nx, 21)
    w_ref, a_ref = oracle.accumulate_d8(d, oracle.kahn_order(d, False), rain)
    R = api.routing_d8(cuda(d), SKEL)
    o = api.accumulate(R, cuda(rain), want_w=True, want_area=True)
    assert api.get_status() == 0
    np.testing.assert_array_equal(o["area"].cpu().numpy().astype(np.uint64), a_ref)
    assert relerr(o["w"].cpu().numpy(), w_ref) <= RTOL_W
    o = api.accumulate(R, None, want_w=False, want_area=True)  # areas alone
    assert api.get_status() == 0
    np.testing.assert_array_equal(o["area"].cpu().numpy().astype(np.uint64), a_ref)


def test_global_phase_flags_are_validated(api):
    d = cuda(np.full((8, 8), oracle.SINK, np.uint8))
    R = api.routing_d8(d, WALK | SKEL)
    with pytest.raises(Exception):
        api.accumulate(R, None, want_area=True)
