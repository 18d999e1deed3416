"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (stated per test): D8 receiver codes, donor counts, MFD masks and unit-rain
areas bit-exact; real-valued water within 1e-6 relative of the FP64 oracle per
cell (the fp32 two-float leading word); the two-float pair within 1e-10 for D8.
"""
import numpy as np
import pytest

import oracle
from paper_2606_12800_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_W = 1e-6


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


SHAPES = [(1, 1), (1, 7), (9, 1), (3, 3), (33, 65), (64, 32), (65, 33), (97, 131), (256, 256),
          (300, 517)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("flags", [0, oracle.EDGE_ROUTE, oracle.D8_LOWEST,
                                   oracle.EDGE_ROUTE | oracle.D8_LOWEST, oracle.D4,
                                   oracle.D4 | oracle.EDGE_ROUTE | oracle.D8_LOWEST])
def test_receivers_d8_bit_exact(api, shape, flags):
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, seed=ny * 7 + nx)
    d, n = api.receivers_d8(cuda(z), 30.0, flags, indeg=True)
    d_ref = oracle.receivers_d8(z, 30.0, flags)
    np.testing.assert_array_equal(d.cpu().numpy(), d_ref)
    np.testing.assert_array_equal(n.cpu().numpy(), oracle.indegree(d_ref, False))


TMA_SHAPES = [(64, 128), (65, 132), (129, 260), (31, 1028), (1000, 1028), (4097, 8), (8, 4096),
              (513, 640)]


@pytest.mark.parametrize("shape", TMA_SHAPES)
@pytest.mark.parametrize("flags", [0, oracle.EDGE_ROUTE, oracle.D8_LOWEST, oracle.D4,
                                   oracle.D4 | oracle.EDGE_ROUTE | oracle.D8_LOWEST])
def test_receivers_d8_tma_path_bit_exact(api, shape, flags):
    """Grids whose rows are whole 16-byte units take the TMA-pipelined kernel
    (boxes across the grid's edges read NaN): codes bit-exact against the
    oracle, including partial tiles on both far edges."""
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, seed=ny + 13 * nx)
    d = api.receivers_d8(cuda(z), 30.0, flags)
    np.testing.assert_array_equal(d.cpu().numpy(), oracle.receivers_d8(z, 30.0, flags))
    assert api.get_status() == 0


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("flags", [0, oracle.EDGE_ROUTE, oracle.D4 | oracle.EDGE_ROUTE])
def test_route_d8_parity(api, shape, flags):
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, seed=ny * 3 + nx)
    rain = inputs.rain_field(ny, nx, 5)
    out = api.route_d8(cuda(z), 30.0, cuda(rain), flags, want_w=True, want_lo=True,
                       want_area=True, want_dir=True)
    d_ref, w_ref, _, order = oracle.route_d8(z, 30.0, rain, flags)
    _, a_ref = oracle.accumulate_d8(d_ref, order, None)
    np.testing.assert_array_equal(out["dir"].cpu().numpy(), d_ref)
    np.testing.assert_array_equal(out["area"].cpu().numpy().astype(np.uint64), a_ref)
    w = out["w"].cpu().numpy()
    lo = out["w_lo"].cpu().numpy()
    assert relerr(w, w_ref) <= RTOL_W
    assert relerr(w.astype(np.float64) + lo, w_ref) <= 1e-10
    assert api.get_status() == 0


@pytest.mark.parametrize("shape", [(64, 64), (300, 517), (5, 700)])
@pytest.mark.parametrize("flags", [0, oracle.EDGE_ROUTE, oracle.D8_LOWEST])
def test_planar_deep_chains(api, shape, flags):
    """Plane toward +x: every row is one long chain crossing many tiles, so
    almost every cell is reached by the cross-tile walkers."""
    ny, nx = shape
    z = inputs.planar_dem(ny, nx, 0.01, 30.0)
    out = api.route_d8(cuda(z), 30.0, None, flags, want_w=True, want_area=True)
    _, w_ref, a_ref, _ = oracle.route_d8(z, 30.0, None, flags)
    np.testing.assert_array_equal(out["area"].cpu().numpy().astype(np.uint64), a_ref)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W
    assert api.get_status() == 0


def test_unit_rain_only_and_determinism(api):
    z = inputs.fractal_dem(700, 900, seed=11)
    zt = cuda(z)
    a1 = api.route_d8(zt, 30.0, None, 0, want_w=False, want_area=True)["area"]
    a2 = api.route_d8(zt, 30.0, None, 0, want_w=False, want_area=True)["area"]
    assert torch.equal(a1, a2)
    rain = cuda(inputs.rain_field(700, 900, 11))
    w1 = api.route_d8(zt, 30.0, rain, 0, want_w=True, want_lo=True, want_area=False)
    w2 = api.route_d8(zt, 30.0, rain, 0, want_w=True, want_lo=True, want_area=False)
    assert torch.equal(w1["w"], w2["w"]) and torch.equal(w1["w_lo"], w2["w_lo"])
    _, _, a_ref, _ = oracle.route_d8(z, 30.0)
    np.testing.assert_array_equal(a1.cpu().numpy().astype(np.uint64), a_ref)


@pytest.mark.parametrize("shape", [(1, 9), (3, 3), (33, 65), (97, 131), (256, 256), (300, 517)])
@pytest.mark.parametrize("flags", [0, oracle.EDGE_ROUTE, oracle.DINF, oracle.DINF | oracle.EDGE_ROUTE])
def test_receivers_mfd(api, shape, flags):
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, beta=2.2, tilt=0.0, seed=ny + nx)
    m, f, n = api.receivers_mfd(cuda(z), 30.0, 1.1, flags, frac=True, indeg=True)
    m_ref, f_ref = oracle.receivers_mfd(z, 30.0, 1.1, flags)
    np.testing.assert_array_equal(m.cpu().numpy(), m_ref)
    np.testing.assert_array_equal(n.cpu().numpy(), oracle.indegree(m_ref, True))
    f = f.cpu().numpy().astype(np.float64)
    assert np.all((f == 0) == (f_ref == 0))
    nz = f_ref > 0
    if nz.any():
        assert np.max(np.abs(f[nz] - f_ref[nz]) / f_ref[nz]) <= 2e-6


@pytest.mark.parametrize("shape", [(1, 9), (33, 65), (97, 131), (256, 256), (300, 517)])
@pytest.mark.parametrize("flags", [0, oracle.EDGE_ROUTE, oracle.DINF])
def test_route_mfd_parity(api, shape, flags):
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, beta=2.2, tilt=0.0, seed=2 * ny + nx)
    rain = inputs.rain_field(ny, nx, 3)
    out = api.route_mfd(cuda(z), 30.0, 1.1, cuda(rain), flags, want_lo=True, want_mask=True)
    m_ref, f_ref, w_ref, _ = oracle.route_mfd(z, 30.0, 1.1, rain, flags)
    np.testing.assert_array_equal(out["mask"].cpu().numpy(), m_ref)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W
    assert api.get_status() == 0


def test_mfd_dataflow_is_deterministic(api):
    """The MFD tile solve finalises cells in an order that depends on
    scheduling, but each cell sums its dependencies in a fixed order: the
    route and the adjoint must be bit-identical from run to run."""
    z = inputs.fractal_dem(1500, 1300, beta=2.2, tilt=0.0, seed=17)
    zt = cuda(z)
    rain = cuda(inputs.rain_field(1500, 1300, 17))
    runs = [api.route_mfd(zt, 30.0, 1.1, rain, 0, want_lo=True, want_mask=True) for _ in range(3)]
    for r in runs[1:]:
        assert torch.equal(r["w"], runs[0]["w"]) and torch.equal(r["w_lo"], runs[0]["w_lo"])
    R = api.routing_mfd(runs[0]["mask"], zt, 30.0, 1.1)
    g1 = api.adjoint(R, runs[0]["w"], runs[0]["w_lo"], want_dz=True)
    g2 = api.adjoint(R, runs[0]["w"], runs[0]["w_lo"], want_dz=True)
    assert torch.equal(g1[0], g2[0]) and torch.equal(g1[1], g2[1])
    assert api.get_status() == 0


def _bowl(ny, nx, seed):
    """A bowl with a little seeded roughness: every path converges on the
    centre, so the tile solves see deep chains and cells that many donors
    complete at about the same time."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r2 = ((y - ny / 2) ** 2 + (x - nx / 2) ** 2) * 0.01
    return (r2 + 1e-3 * np.random.default_rng(seed).random((ny, nx))).astype(np.float32)


def _plane_x(ny, nx, seed):
    """A plane falling towards +x with seeded jitter: every cell drains to its
    three eastern neighbours, so dependencies cross the whole grid."""
    x = np.arange(nx, dtype=np.float64)[None, :].repeat(ny, 0)
    return (1000.0 - 0.3 * x + 1e-3 * np.random.default_rng(seed).random((ny, nx))).astype(np.float32)


@pytest.mark.parametrize("make", [_bowl, _plane_x])
@pytest.mark.parametrize("shape", [(130, 140), (300, 517)])
def test_route_mfd_converging_and_crossing_flows(api, make, shape):
    ny, nx = shape
    z = make(ny, nx, ny + nx)
    rain = inputs.rain_field(ny, nx, 4)
    out = api.route_mfd(cuda(z), 30.0, 1.1, cuda(rain), 0, want_lo=True, want_mask=True)
    m_ref, f_ref, w_ref, order = oracle.route_mfd(z, 30.0, 1.1, rain)
    np.testing.assert_array_equal(out["mask"].cpu().numpy(), m_ref)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W
    R = api.routing_mfd(out["mask"], cuda(z), 30.0, 1.1)
    dLdr, _ = api.adjoint(R, out["w"], out["w_lo"], want_dz=False)
    g_ref = oracle.adjoint(order, w_ref, frac=f_ref)
    assert relerr(dLdr.cpu().numpy(), g_ref) <= RTOL_W
    assert api.get_status() == 0


@pytest.mark.parametrize("shape", [(33, 65), (256, 256), (300, 517)])
def test_adjoint_d8(api, shape):
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, seed=nx)
    rain = inputs.rain_field(ny, nx, 1)
    out = api.route_d8(cuda(z), 30.0, cuda(rain), 0, want_w=True, want_lo=True, want_dir=True,
                       want_area=False)
    R = api.routing_d8(out["dir"])
    dLdr, _ = api.adjoint(R, out["w"], out["w_lo"])
    d_ref, w_ref, _, order = oracle.route_d8(z, 30.0, rain)
    g_ref = oracle.adjoint(order, w_ref, dir_=d_ref)
    assert relerr(dLdr.cpu().numpy(), g_ref) <= RTOL_W
    # arbitrary incoming gradient
    gbar = np.random.default_rng(0).random((ny, nx), dtype=np.float32)
    dLdr, _ = api.adjoint(R, out["w"], out["w_lo"], dLdw=cuda(gbar))
    g_ref = oracle.adjoint(order, w_ref, dir_=d_ref, gbar=gbar.astype(np.float64))
    assert relerr(dLdr.cpu().numpy(), g_ref) <= RTOL_W
    assert api.get_status() == 0


@pytest.mark.parametrize("shape", [(33, 65), (256, 256), (300, 517)])
def test_adjoint_mfd(api, shape):
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, beta=2.2, tilt=0.0, seed=nx + 1)
    rain = inputs.rain_field(ny, nx, 2)
    zt = cuda(z)
    m = api.receivers_mfd(zt, 30.0, 1.1)
    R = api.routing_mfd(m, zt, 30.0, 1.1)
    o = api.accumulate(R, cuda(rain), want_w=True, want_lo=True)
    dLdr, dLdz = api.adjoint(R, o["w"], o["w_lo"], want_dz=True)
    m_ref, f_ref, w_ref, order = oracle.route_mfd(z, 30.0, 1.1, rain)
    g_ref = oracle.adjoint(order, w_ref, frac=f_ref)
    dz_ref = oracle.mfd_grad_z(z, 30.0, 1.1, f_ref, w_ref, g_ref)
    assert relerr(dLdr.cpu().numpy(), g_ref) <= RTOL_W
    dz = dLdz.cpu().numpy().astype(np.float64)
    scale = np.abs(dz_ref).max()
    assert np.max(np.abs(dz - dz_ref)) <= 1e-4 * scale
    big = np.abs(dz_ref) > 1e-2 * scale
    assert np.max(np.abs(dz[big] - dz_ref[big]) / np.abs(dz_ref[big])) <= 1e-3
    assert api.get_status() == 0


def test_mass_balance(api):
    ny, nx = 400, 300
    z = inputs.fractal_dem(ny, nx, seed=4)
    rain = inputs.rain_field(ny, nx, 4)
    rt = cuda(rain)
    out = api.route_d8(cuda(z), 30.0, rt, 0, want_w=True, want_lo=True, want_area=True,
                       want_dir=True)
    R = api.routing_d8(out["dir"])
    mb = api.mass_balance(R, rt, out["w"], out["w_lo"], out["area"]).cpu().numpy()
    d_ref, w_ref, _, _ = oracle.route_d8(z, 30.0, rain)
    s_ref, r_ref = oracle.mass_balance(w_ref, rain, dir_=d_ref)
    assert mb[2] == nx * ny
    assert abs(mb[1] - r_ref) <= 1e-12 * r_ref
    assert abs(mb[0] - s_ref) <= 1e-12 * s_ref
    assert abs(mb[0] - mb[1]) <= 1e-10 * mb[1]
    mb2 = api.mass_balance(R, rt, out["w"], out["w_lo"], out["area"]).cpu().numpy()
    assert np.array_equal(mb, mb2)


def _sink_sum_dem(kind, ny, nx, api):
    if kind == "plane":
        x = np.arange(nx, dtype=np.float64)[None, :]
        y = np.arange(ny, dtype=np.float64)[:, None]
        return cuda(np.ascontiguousarray((1000.0 - x - 0.37 * y).astype(np.float32)))
    zt = cuda(inputs.fractal_dem(ny, nx, beta=2.0, tilt=0.01, seed=nx + ny))
    if kind == "filled":
        zt = api.fill(zt)[0]
    return zt


@pytest.mark.parametrize("kind,shape", [("rough", (1, 9)), ("rough", (3, 3)), ("rough", (300, 517)),
                                        ("rough", (704, 1024)), ("filled", (600, 640)),
                                        ("plane", (256, 384))])
@pytest.mark.parametrize("gflags", [0, _lib.FR_GLOBAL_WALKERS, _lib.FR_GLOBAL_SKELETON])
def test_mass_balance_sink_sums(api, kind, shape, gflags):
    """FR_SINK_SUMS_IN_WORKSPACE: the area term from the accumulation's sums
    (local phase) and the global cells' sinks equals the full pass over the
    stored areas bit for bit, through the cell walkers and the skeleton
    solve, with and without a rain field."""
    ny, nx = shape
    zt = _sink_sum_dem(kind, ny, nx, api)
    d = api.receivers_d8(zt)
    Rs = api.routing_d8(d, gflags | _lib.FR_SINK_SUMS_IN_WORKSPACE)
    area = api.accumulate(Rs, None, want_w=False, want_area=True)["area"]
    fused = api.mass_balance(Rs, area=area).cpu().numpy()
    full = api.mass_balance(api.routing_d8(d, gflags), area=area).cpu().numpy()
    assert fused.tobytes() == full.tobytes()
    assert fused[2] == nx * ny and fused[1] == nx * ny and fused[0] == 0.0
    rt = cuda(inputs.rain_field(ny, nx, 5))
    fused_r = api.mass_balance(Rs, rain=rt, area=area).cpu().numpy()
    full_r = api.mass_balance(api.routing_d8(d, gflags), rain=rt, area=area).cpu().numpy()
    assert fused_r.tobytes() == full_r.tobytes()
    assert api.get_status() == 0


def test_mass_balance_sink_sums_count_only_sink_codes(api):
    """Codes pointing out of the grid act as no receiver in the accumulation
    but are not FR_SINK: both forms of the mass balance leave them out."""
    ny, nx = 300, 400
    z = cuda(inputs.fractal_dem(ny, nx, beta=2.0, tilt=0.01, seed=9))
    d = api.receivers_d8(z)
    d[0, 5:300] = 1     # N from the top row: out of the grid
    d[100:200, 0] = 2   # W from the left column
    Rs = api.routing_d8(d, _lib.FR_SINK_SUMS_IN_WORKSPACE)
    area = api.accumulate(Rs, None, want_w=False, want_area=True)["area"]
    fused = api.mass_balance(Rs, area=area).cpu().numpy()
    full = api.mass_balance(api.routing_d8(d), area=area).cpu().numpy()
    assert fused.tobytes() == full.tobytes()
    a = area.cpu().numpy()
    assert fused[2] == nx * ny - a[0, 5:300].sum() - a[100:200, 0].sum()
    # the flag needs areas and no water
    w = api.accumulate(Rs, None, want_w=True, want_area=True)
    with pytest.raises(RuntimeError):
        api.mass_balance(Rs, w=w["w"], area=w["area"])
    with pytest.raises(RuntimeError):
        api.mass_balance(Rs)
    assert api.get_status() == 0


def test_cycle_reports_no_progress(api):
    """A routing with a cycle (two cells pointing at each other) must finish
    and leave FR_ERR_NO_PROGRESS in the status word (no hang)."""
    ny, nx = 40, 70
    d = np.full((ny, nx), oracle.SINK, np.uint8)
    d[10, 10] = 0   # E  -> (11, 10)
    d[10, 11] = 2   # W  -> (10, 10)
    d[20, 63] = 0   # a cycle across a tile border (x = 63 | 64)
    d[20, 64] = 2
    R = api.routing_d8(cuda(d))
    api.accumulate(R, None, want_w=True, want_area=True)
    assert api.get_status() == 5
    # a good routing afterwards on the same workspace is clean again
    z = inputs.fractal_dem(ny, nx, seed=1)
    api.route_d8(cuda(z), 30.0)
    assert api.get_status() == 0


def _pit_lattice(ny, nx):
    """3 x 3 blocks whose eight outer cells all drain into the centre (a sink):
    every centre has eight donors, all of them leaves."""
    d = np.full((ny, nx), oracle.SINK, np.uint8)
    to_centre = {(-1, -1): 7, (-1, 0): 3, (-1, 1): 6, (0, -1): 0, (0, 1): 2,
                 (1, -1): 4, (1, 0): 1, (1, 1): 5}  # code of the cell at (dy, dx) from the centre
    for cy in range(1, ny - 1, 3):
        for cx in range(1, nx - 1, 3):
            for (dy, dx), k in to_centre.items():
                d[cy + dy, cx + dx] = k
    return d


@pytest.mark.parametrize("shape", [(64, 96), (301, 517)])
def test_eight_donor_cells(api, shape):
    """Cells with eight donors are completed exactly once, whatever the order of
    the donors' arrivals and of the cell's own count (repeated launches, both
    tile geometries through the batched route)."""
    ny, nx = shape
    d = _pit_lattice(ny, nx)
    rain = inputs.rain_field(ny, nx, 21)
    w_ref, a_ref = oracle.accumulate_d8(d, oracle.kahn_order(d, False), rain)
    assert a_ref.max() == 9
    R = api.routing_d8(cuda(d))
    rt = cuda(rain)
    for _ in range(5):
        o = api.accumulate(R, rt, want_w=True, want_area=True)
        assert api.get_status() == 0
        np.testing.assert_array_equal(o["area"].cpu().numpy().astype(np.uint64), a_ref)
        assert relerr(o["w"].cpu().numpy(), w_ref) <= RTOL_W
    # the batched route with each tile geometry, from a DEM whose D8 codes are
    # the lattice's: each block a cone falling towards its centre
    yy, xx = np.mgrid[0:ny, 0:nx]
    cy, cx = 1 + 3 * ((yy - 1) // 3).clip(0), 1 + 3 * ((xx - 1) // 3).clip(0)
    z = (np.maximum(np.abs(yy - cy), np.abs(xx - cx)) + 0.25 * (np.abs(yy - cy) + np.abs(xx - cx))
         + 10.0).astype(np.float32)
    d_z = oracle.receivers_d8(z, 30.0)
    w_z, a_z = oracle.accumulate_d8(d_z, oracle.kahn_order(d_z, False), rain)
    for _ in range(3):
        outs = api.route_batch([cuda(z)] * 4, [rt] * 4, "d8", want_w=True, want_area=True,
                               autotune=True)
        assert api.batch_status(outs) == 0
        for o in outs:
            np.testing.assert_array_equal(o["route"].cpu().numpy(), d_z)
            np.testing.assert_array_equal(o["area"].cpu().numpy().astype(np.uint64), a_z)
            assert relerr(o["w"].cpu().numpy(), w_z) <= RTOL_W


def test_routing_pointing_outside_grid_is_a_sink(api):
    """Caller-supplied codes that point out of the grid act as no receiver."""
    ny, nx = 16, 16
    d = np.full((ny, nx), oracle.SINK, np.uint8)
    d[0, :] = 1    # N from the top row: outside
    d[:, 0] = 2    # W from the left column: outside
    d[5, 5] = 0    # E -> (6, 5)
    R = api.routing_d8(cuda(d))
    out = api.accumulate(R, None, want_w=True, want_area=True)
    a = out["area"].cpu().numpy()
    assert a[5, 6] == 2 and a.sum() == ny * nx + 1
    assert api.get_status() == 0


@pytest.mark.parametrize("shape,seed", [((2048, 1536), 3), ((1500, 2600), 7), ((700, 1100), 2)])
def test_route_d8_large(api, shape, seed):
    """Many tiles: cross-tile chains, halo overlaps and walkers all occur."""
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, seed=seed)
    rain = inputs.rain_field(ny, nx, seed)
    out = api.route_d8(cuda(z), 30.0, cuda(rain), 0, want_w=True, want_lo=True, want_area=True)
    assert api.get_status() == 0
    d_ref, w_ref, _, order = oracle.route_d8(z, 30.0, rain)
    _, a_ref = oracle.accumulate_d8(d_ref, order, None)
    np.testing.assert_array_equal(out["area"].cpu().numpy().astype(np.uint64), a_ref)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W


def test_d8_benchmark_workload_full_size(api):
    """The 4096^2 benchmark workload (beta 2, tilt 0.01, rain U[0,1)): areas
    bit-exact and water within 1e-6 of the full FP64 oracle."""
    n = 4096
    z = inputs.fractal_dem(n, n, beta=2.0, tilt=0.01, seed=1)
    rain = inputs.rain_field(n, n, 1)
    out = api.route_d8(cuda(z), 30.0, cuda(rain), 0, want_w=True, want_area=True, want_dir=True)
    assert api.get_status() == 0
    d_ref, w_ref, _, order = oracle.route_d8(z, 30.0, rain)
    np.testing.assert_array_equal(out["dir"].cpu().numpy(), d_ref)
    _, a_ref = oracle.accumulate_d8(d_ref, order, None)
    np.testing.assert_array_equal(out["area"].cpu().numpy().astype(np.uint64), a_ref)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W


@pytest.mark.parametrize("shape", [(777, 1333), (1024, 1536)])
def test_route_mfd_walker_without_trailing_words(api, shape):
    """Grids of many extended tiles, so some cells are finished by the walker
    kernel, which then reads the trailing words the tiles keep in the
    workspace (none are requested by the caller)."""
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, beta=2.2, tilt=0.0, seed=ny + 7)
    rain = inputs.rain_field(ny, nx, 5)
    out = api.route_mfd(cuda(z), 30.0, 1.1, cuda(rain), 0)
    assert api.get_status() == 0
    _, _, w_ref, _ = oracle.route_mfd(z, 30.0, 1.1, rain)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W
    # unit rain as well
    out = api.route_mfd(cuda(z), 30.0, 1.1, None, 0)
    _, _, w_ref, _ = oracle.route_mfd(z, 30.0, 1.1, None)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W


@pytest.mark.slow
def test_slope_split_full_size_workload(api):
    """The 8192^2 slope-split workload (beta 2.2, no tilt, unit rain, p = 1.1),
    generated on the device as the benchmark does: masks bit-exact and water
    within 1e-6 of the full FP64 oracle, per cell."""
    n = 8192
    zt = inputs.fractal_dem_torch(n, n, beta=2.2, tilt=0.0, seed=3, device="cuda")
    out = api.route_mfd(zt, 30.0, 1.1, None, 0, want_mask=True)
    assert api.get_status() == 0
    z = zt.cpu().numpy()
    m_ref, _, w_ref, _ = oracle.route_mfd(z, 30.0, 1.1, None)
    np.testing.assert_array_equal(out["mask"].cpu().numpy(), m_ref)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W


def _adjoint_fd_check(api, zt, count, seed):
    """dL/dz and dL/drain of the GPU adjoint (L = sum over sinks of w^2, unit
    rain, MFD p = 1.1) against central finite differences of the FP64 oracle,
    taken exactly and incrementally (oracle.MfdLossDelta) at `count` random
    interior cells whose elevation gaps to all neighbours exceed 1 mm."""
    ny, nx = zt.shape
    m = api.receivers_mfd(zt, 30.0, 1.1)
    R = api.routing_mfd(m, zt, 30.0, 1.1)
    fwd = api.accumulate(R, None, want_w=True, want_lo=True)
    dLdr, dLdz = api.adjoint(R, fwd["w"], fwd["w_lo"], want_dz=True)
    assert api.get_status() == 0
    dLdr, dLdz, z = dLdr.cpu().numpy(), dLdz.cpu().numpy(), zt.cpu().numpy()
    del m, R, fwd
    torch.cuda.empty_cache()
    m_ref, f_ref, w_ref, _ = oracle.route_mfd(z, 30.0, 1.1, None)
    D = oracle.MfdLossDelta(z, 30.0, 1.1, m_ref, f_ref, w_ref)
    z64 = z.astype(np.float64)
    rng = np.random.default_rng(seed)
    got_z, fd_z, got_r, fd_r = [], [], [], []
    while len(fd_z) < count:
        y, x = int(rng.integers(1, ny - 1)), int(rng.integers(1, nx - 1))
        gap = min(abs(z64[y, x] - z64[y + oracle.OFFY[k], x + oracle.OFFX[k]]) for k in range(8))
        if gap < 1e-3:
            continue
        fz = D.central(y * nx + x, 1e-3 * gap, 0)
        if np.isnan(fz):
            continue
        fd_z.append(fz)
        got_z.append(dLdz[y, x])
        fd_r.append(D.central(y * nx + x, 1e-3, 1))
        got_r.append(dLdr[y, x])
    fd_z, got_z, fd_r, got_r = map(np.asarray, (fd_z, got_z, fd_r, got_r))
    scale = np.abs(fd_z).max()
    assert np.all(np.abs(got_z - fd_z) <= 1e-4 * np.abs(fd_z) + 1e-6 * scale), \
        np.max(np.abs(got_z - fd_z) / np.maximum(np.abs(fd_z), 1e-30))
    assert np.all(np.abs(got_r - fd_r) <= 1e-4 * np.abs(fd_r)), \
        np.max(np.abs(got_r - fd_r) / np.abs(fd_r))


def test_mfd_adjoint_finite_differences(api):
    """Adjoint against finite differences on a 1024^2 slope-split DEM."""
    zt = inputs.fractal_dem_torch(1024, 1024, beta=2.2, tilt=0.0, seed=21, device="cuda")
    _adjoint_fd_check(api, zt, 64, seed=21)


@pytest.mark.slow
def test_mfd_adjoint_finite_differences_full_size(api):
    """The 16384^2 slope-split adjoint workload (the benchmark's DEM, loss =
    sum over sinks of w^2): dL/dz and dL/drain at 64 random cells against
    central finite differences of the FP64 oracle, to 1e-4 relative."""
    zt = inputs.fractal_dem_torch(16384, 16384, beta=2.2, tilt=0.0, seed=5, device="cuda")
    _adjoint_fd_check(api, zt, 64, seed=64)


def _crossings(order, deps, nx, tx=64, ty=32):
    """C = the largest number of 64x32-tile boundaries a dependency path
    crosses (cells in high-to-low order; deps[c] = cells c receives from)."""
    cross = np.zeros(len(order), np.int64)
    tile = lambda c: ((c % nx) // tx, (c // nx) // ty)
    for c in order:
        for j in deps.get(int(c), ()):
            cross[c] = max(cross[c], cross[j] + (tile(j) != tile(int(c))))
    return int(cross.max()) if len(cross) else 0


def _donor_lists(recv_of, n):
    deps = {}
    for j in range(n):
        for t in recv_of(j):
            deps.setdefault(t, []).append(j)
    return deps


@pytest.mark.parametrize("shape", [(32, 64), (20, 45), (33, 65), (97, 131), (256, 300)])
def test_richardson_d8_exact_after_c_plus_one(api, shape):
    """Richardson I+X on 64x32 tiles: the result of the exact solve, after
    exactly C + 1 iterations (C = most tile crossings of any stream).  A grid
    of one tile (one "process": D^-1 = A^-1) is exact after one iteration."""
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, beta=2.0, tilt=0.01, seed=nx)
    d = api.receivers_d8(cuda(z), 30.0)
    R = api.routing_d8(d)
    out, iters = api.accumulate_richardson(R, None)
    d_ref, w_ref, _, order = oracle.route_d8(z, 30.0, None)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W
    dr = d_ref.ravel()
    recv = lambda j: () if dr[j] == oracle.SINK else (j + oracle.OFFY[dr[j]] * nx + oracle.OFFX[dr[j]],)
    C = _crossings(order, _donor_lists(recv, nx * ny), nx)
    assert iters == C + 1
    # (I-X)(I+X): two applications per iteration, half the iterations
    out2, iters2 = api.accumulate_richardson(R, None, order=2)
    assert iters2 == (C + 2) // 2
    np.testing.assert_array_equal(out2["w"].cpu().numpy(), out["w"].cpu().numpy())
    rain = inputs.rain_field(ny, nx, 2)
    out, _ = api.accumulate_richardson(R, cuda(rain))
    _, w_ref, _, _ = oracle.route_d8(z, 30.0, rain)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W


@pytest.mark.parametrize("shape", [(70, 90), (200, 257)])
def test_richardson_mfd_exact_after_c_plus_one(api, shape):
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, beta=2.2, tilt=0.0, seed=ny)
    zt = cuda(z)
    m = api.receivers_mfd(zt, 30.0, 1.1)
    R = api.routing_mfd(m, zt, 30.0, 1.1)
    out, iters = api.accumulate_richardson(R, None)
    m_ref, _, w_ref, order = oracle.route_mfd(z, 30.0, 1.1, None)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W
    mr = m_ref.ravel()
    recv = lambda j: tuple(j + oracle.OFFY[k] * nx + oracle.OFFX[k] for k in range(8) if (mr[j] >> k) & 1)
    assert iters == _crossings(order, _donor_lists(recv, nx * ny), nx) + 1
    # the same water as the two-phase exact solve
    w2 = api.accumulate(R, None, want_w=True)["w"]
    assert relerr(out["w"].cpu().numpy(), w2.cpu().numpy().astype(np.float64)) <= 1e-6


def test_richardson_stops_at_the_iteration_limit(api):
    z = inputs.planar_dem(40, 300, 0.01, 30.0)  # rows are chains across 5 tiles
    d = api.receivers_d8(cuda(z), 30.0, oracle.EDGE_ROUTE)
    R = api.routing_d8(d)
    with pytest.raises(Exception):
        api.accumulate_richardson(R, None, max_iterations=2)
    out, iters = api.accumulate_richardson(R, None, max_iterations=50)
    assert iters == 5  # C = 4 crossings along a 300-cell row
    assert api.accumulate_richardson(R, None, order=2)[1] == 3
    assert api.accumulate_richardson(R, None, order=5)[1] == 1
    np.testing.assert_allclose(out["w"].cpu().numpy()[5, :], np.arange(1, 301), rtol=0)


def _batch_specs():
    return [(17, 23, 2.0), (64, 64, 1.8), (31, 200, 2.4), (130, 97, 2.1), (300, 257, 2.0),
            (5, 5, 2.2), (1, 40, 2.0), (90, 1, 2.0), (256, 300, 1.9), (128, 64, 2.3)]


@pytest.mark.parametrize("autotune", [False, True])
def test_route_batch_d8(api, autotune):
    specs = _batch_specs()
    dems = [inputs.fractal_dem(ny, nx, beta=b, tilt=0.0, seed=i) for i, (ny, nx, b) in enumerate(specs)]
    rains = [inputs.rain_field(z.shape[0], z.shape[1], i) for i, z in enumerate(dems)]
    outs = api.route_batch([cuda(z) for z in dems], [cuda(r) for r in rains], "d8",
                           want_w=True, want_area=True, autotune=autotune)
    assert api.batch_status(outs) == 0
    for z, r, o in zip(dems, rains, outs):
        d_ref, w_ref, _, order = oracle.route_d8(z, 30.0, r)
        _, a_ref = oracle.accumulate_d8(d_ref, order, None)
        np.testing.assert_array_equal(o["route"].cpu().numpy(), d_ref)
        np.testing.assert_array_equal(o["area"].cpu().numpy().astype(np.uint64), a_ref)
        assert relerr(o["w"].cpu().numpy(), w_ref) <= RTOL_W


def test_route_batch_mfd(api):
    specs = _batch_specs()
    dems = [inputs.fractal_dem(ny, nx, beta=b, tilt=0.0, seed=10 + i) for i, (ny, nx, b) in enumerate(specs)]
    rains = [inputs.rain_field(z.shape[0], z.shape[1], i) for i, z in enumerate(dems)]
    outs = api.route_batch([cuda(z) for z in dems], [cuda(r) for r in rains], "mfd", p=1.1,
                           want_w=True, want_lo=True)
    assert api.batch_status(outs) == 0
    for z, r, o in zip(dems, rains, outs):
        m_ref, f_ref, w_ref, _ = oracle.route_mfd(z, 30.0, 1.1, r)
        np.testing.assert_array_equal(o["route"].cpu().numpy(), m_ref)
        assert relerr(o["w"].cpu().numpy(), w_ref) <= RTOL_W


def test_dinf_batch_adjoint_and_large_route(api):
    """D-infinity through every MFD path: a 1024x1536 route (walkers), the
    batched route, and the adjoint dL/drain; dL/dz is refused."""
    ny, nx = 1024, 1536
    z = inputs.fractal_dem(ny, nx, beta=2.2, tilt=0.0, seed=77)
    rain = inputs.rain_field(ny, nx, 77)
    out = api.route_mfd(cuda(z), 30.0, 1.1, cuda(rain), oracle.DINF, want_lo=True, want_mask=True)
    assert api.get_status() == 0
    m_ref, f_ref, w_ref, order = oracle.route_mfd(z, 30.0, 1.1, rain, oracle.DINF)
    np.testing.assert_array_equal(out["mask"].cpu().numpy(), m_ref)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W
    zt = cuda(z)
    R = api.routing_mfd(out["mask"].cuda(), zt, 30.0, 1.1, oracle.DINF)
    wd, wl = out["w"].cuda(), out["w_lo"].cuda()
    dLdr, _ = api.adjoint(R, wd, wl)
    g_ref = oracle.adjoint(order, w_ref, frac=f_ref)
    assert relerr(dLdr.cpu().numpy(), g_ref) <= RTOL_W
    with pytest.raises(Exception):
        api.adjoint(R, wd, wl, want_dz=True)
    specs = _batch_specs()
    dems = [inputs.fractal_dem(a, b, beta=c, tilt=0.0, seed=30 + i) for i, (a, b, c) in enumerate(specs)]
    rains = [inputs.rain_field(d.shape[0], d.shape[1], i) for i, d in enumerate(dems)]
    outs = api.route_batch([cuda(d) for d in dems], [cuda(r) for r in rains], "mfd", p=1.1,
                           flags=oracle.DINF, want_w=True)
    assert api.batch_status(outs) == 0
    for d, r, o in zip(dems, rains, outs):
        m_ref, _, w_ref, _ = oracle.route_mfd(d, 30.0, 1.1, r, oracle.DINF)
        np.testing.assert_array_equal(o["route"].cpu().numpy(), m_ref)
        assert relerr(o["w"].cpu().numpy(), w_ref) <= RTOL_W


@pytest.mark.parametrize("shape", [(33, 65), (300, 517)])
def test_adjoint_mfd_kept_weights(api, shape):
    """With FR_WEIGHTS_IN_WORKSPACE the adjoint and a second accumulation read
    the fractions the forward left in the caller's workspace: results equal
    bit for bit those that recompute them."""
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, beta=2.2, tilt=0.0, seed=nx + 7)
    rain = inputs.rain_field(ny, nx, 3)
    zt, rt = cuda(z), cuda(rain)
    ws = torch.empty(api.workspace_size(nx, ny, mfd=True), dtype=torch.uint8, device="cuda")
    fused = api.route_mfd(zt, 30.0, 1.1, rt, want_lo=True, want_mask=True, ws=ws)
    Rk = api.routing_mfd(fused["mask"], zt, 30.0, 1.1, _lib.FR_WEIGHTS_IN_WORKSPACE)
    kept = api.adjoint(Rk, fused["w"], fused["w_lo"], want_dz=True, ws=ws)
    R = api.routing_mfd(fused["mask"], zt, 30.0, 1.1)
    ref = api.adjoint(R, fused["w"], fused["w_lo"], want_dz=True)
    assert torch.equal(kept[0], ref[0]) and torch.equal(kept[1], ref[1])
    # the adjoint left the fractions in place: an accumulation may reuse them
    again = api.accumulate(Rk, rt, want_w=True, want_lo=True, ws=ws)
    assert torch.equal(again["w"], fused["w"]) and torch.equal(again["w_lo"], fused["w_lo"])
    assert api.get_status(ws=ws) == 0 and api.get_status() == 0


def test_autograd_route_mfd_keep_weights(api):
    """RouteMFD with the forward's fractions kept gives the gradients of the
    default (recomputing) backward bit for bit."""
    ny, nx = 70, 90
    z = inputs.fractal_dem(ny, nx, beta=2.2, tilt=0.0, seed=11)
    rain = inputs.rain_field(ny, nx, 11)
    gbar = cuda(np.random.default_rng(4).random((ny, nx)).astype(np.float32))
    grads = []
    for keep in (False, True):
        zt = cuda(z).requires_grad_(True)
        rt = cuda(rain).requires_grad_(True)
        w = api.RouteMFD.apply(zt, rt, 30.0, 1.1, 0, keep)
        (w * gbar).sum().backward()
        grads.append((zt.grad, rt.grad))
    assert torch.equal(grads[0][0], grads[1][0]) and torch.equal(grads[0][1], grads[1][1])


def test_autograd_route_mfd(api):
    """RouteMFD backward equals the adjoint of the FP64 oracle."""
    ny, nx = 48, 40
    z = inputs.fractal_dem(ny, nx, beta=2.2, tilt=0.0, seed=5)
    rain = inputs.rain_field(ny, nx, 5)
    zt = cuda(z).requires_grad_(True)
    rt = cuda(rain).requires_grad_(True)
    w = api.RouteMFD.apply(zt, rt, 30.0, 1.1, 0)
    gbar = np.random.default_rng(3).random((ny, nx)).astype(np.float32)
    (w * cuda(gbar)).sum().backward()
    m_ref, f_ref, w_ref, order = oracle.route_mfd(z, 30.0, 1.1, rain)
    g_ref = oracle.adjoint(order, w_ref, frac=f_ref, gbar=gbar.astype(np.float64))
    dz_ref = oracle.mfd_grad_z(z, 30.0, 1.1, f_ref, w_ref, g_ref)
    assert relerr(rt.grad.cpu().numpy(), g_ref) <= RTOL_W
    dz = zt.grad.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(dz - dz_ref)) <= 1e-4 * np.abs(dz_ref).max()


# ------------------------------------------------------------------ depression filling
@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (2, 7), (3, 3), (33, 65), (64, 32), (97, 131),
                                   (300, 517)])
def test_fill_parity(api, shape):
    """fr_fill against the priority-flood oracle, bit for bit: a fractal
    surface and an integer-valued one (wide flats and many equal neighbours)."""
    rng = np.random.default_rng(shape[0] * 1000 + shape[1])
    for z in (inputs.fractal_dem(*shape, beta=2.0, tilt=0.0, seed=11),
              rng.integers(0, 6, size=shape).astype(np.float32)):
        F, sweeps = api.fill(cuda(z))
        np.testing.assert_array_equal(F.cpu().numpy(), oracle.fill(z))
        assert sweeps >= 1


def test_fill_large_basins_drain_to_edge(api):
    """A 1024x1536 surface with wide closed basins (beta 2.2, no tilt): the fill
    matches the oracle bit for bit, D8 routing on it has sinks only on the
    edge, and a call allowed one sweep reports FR_ERR_NO_PROGRESS."""
    z = inputs.fractal_dem(1024, 1536, beta=2.2, tilt=0.0, seed=12)
    F, sweeps = api.fill(cuda(z))
    np.testing.assert_array_equal(F.cpu().numpy(), oracle.fill(z))
    d = api.receivers_d8(F, 30.0).cpu().numpy()
    assert (d[1:-1, 1:-1] != oracle.SINK).all()
    assert sweeps > 1
    with pytest.raises(Exception):
        api.fill(cuda(z), max_sweeps=1)


def test_fill_full_size_workload(api):
    """The 4096^2 D8 benchmark DEM, filled, against the full oracle."""
    n = 4096
    z = inputs.fractal_dem(n, n, beta=2.0, tilt=0.01, seed=1)
    F, _ = api.fill(cuda(z))
    np.testing.assert_array_equal(F.cpu().numpy(), oracle.fill(z))
