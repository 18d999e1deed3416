"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: the worked 3x3 example
the paper prints (Fig. 1, Sec. 2.1-2.2), dense LU solves of the linear system of
Sec. 2.2 (a different method than the high-to-low sweep), closed forms on planar
DEMs, hand-computed MFD fractions, mass conservation (Sec. 4), upstream BFS
basin sizes, a second valid processing order (Sec. 3.2), and central finite
differences for the elevation gradient.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_12800_gb300 import inputs

OFFX = (1, 0, -1, 0, 1, -1, -1, 1)
OFFY = (0, -1, 0, 1, -1, -1, 1, 1)


def _dem(ny, nx, seed, beta=2.0, tilt=0.01):
    return inputs.fractal_dem(ny, nx, beta=beta, tilt=tilt, seed=seed)


def _dense_A_d8(dir_):
    """A = I - W assembled from a direction grid (Eq. linear-system)."""
    ny, nx = dir_.shape
    n = nx * ny
    A = np.eye(n)
    for y in range(ny):
        for x in range(nx):
            d = dir_[y, x]
            if d == oracle.SINK:
                continue
            A[(y + OFFY[d]) * nx + x + OFFX[d], y * nx + x] -= 1.0
    return A


def _dense_A_mfd(frac):
    ny, nx = frac.shape[:2]
    n = nx * ny
    A = np.eye(n)
    for y in range(ny):
        for x in range(nx):
            for k in range(8):
                f = frac[y, x, k]
                if f != 0.0:
                    A[(y + OFFY[k]) * nx + x + OFFX[k], y * nx + x] -= f
    return A


# ---------------------------------------------------------------- Fig. 1 ----

@pytest.mark.parametrize("rule", [oracle.D8_STEEPEST, oracle.D8_LOWEST])
def test_fig1_routing_list(fig1, rule):
    d = oracle.receivers_d8(fig1["z"], 1.0, oracle.EDGE_ROUTE | rule)
    for src, dst in fig1["list"].items():
        i = src - 1
        y, x = divmod(i, 3)
        code = d[y, x]
        if dst == 0:
            assert code == oracle.SINK
        else:
            assert code != oracle.SINK
            assert (y + OFFY[code]) * 3 + x + OFFX[code] == dst - 1


def test_fig1_order_and_water(fig1):
    z = fig1["z"]
    assert list(oracle.high_to_low_order(z) + 1) == fig1["order"]
    d, w, a, _ = oracle.route_d8(z, 1.0, flags=oracle.EDGE_ROUTE)
    np.testing.assert_array_equal(w.ravel(), fig1["w"])
    np.testing.assert_array_equal(a.ravel(), fig1["w"].astype(np.uint64))


def test_fig1_apply_A_columns(fig1):
    """apply_A(e_j) is column j of the printed matrix A (Eq. linear-system)."""
    d = oracle.receivers_d8(fig1["z"], 1.0, oracle.EDGE_ROUTE)
    for j in range(9):
        e = np.zeros((3, 3))
        e.flat[j] = 1.0
        col = oracle.apply_A(e, dir_=d).ravel()
        np.testing.assert_array_equal(col, fig1["A"][:, j])
    # and the printed A times the printed w gives unit rain
    np.testing.assert_array_equal(fig1["A"] @ fig1["w"], np.ones(9))


def test_fig1_edge_sink():
    """Default edge mode: only the interior node 5 routes (to node 3)."""
    z = np.array([[6, 3.5, 1], [8, 5, 3], [9, 7, 4.5]], np.float32)
    d, w, a, _ = oracle.route_d8(z, 1.0)
    assert (d.ravel() == oracle.SINK).sum() == 8
    expect = np.ones(9)
    expect[4], expect[2] = 1, 2
    np.testing.assert_array_equal(w.ravel(), expect)


# ------------------------------------------------------------ D8 receivers --

@pytest.mark.parametrize("shape,seed", [((17, 23), 1), ((32, 32), 2), ((5, 64), 3)])
@pytest.mark.parametrize("edge", [oracle.EDGE_SINK, oracle.EDGE_ROUTE])
def test_d8_receiver_invariants(shape, seed, edge):
    """Receiver is strictly lower and at least as steep (FP64) as every other
    lower neighbour; non-edge sinks have no strictly lower neighbour."""
    ny, nx = shape
    z = _dem(ny, nx, seed)
    d = oracle.receivers_d8(z, 30.0, edge)
    z64 = z.astype(np.float64)
    for y in range(ny):
        for x in range(nx):
            edge_cell = x in (0, nx - 1) or y in (0, ny - 1)
            slopes = {}
            for k in range(8):
                xn, yn = x + OFFX[k], y + OFFY[k]
                if 0 <= xn < nx and 0 <= yn < ny and z64[yn, xn] < z64[y, x]:
                    dist = 30.0 * (1.0 if k < 4 else math.sqrt(2.0))
                    slopes[k] = (z64[y, x] - z64[yn, xn]) / dist
            code = d[y, x]
            if edge == oracle.EDGE_SINK and edge_cell:
                assert code == oracle.SINK
                continue
            if not slopes:
                assert code == oracle.SINK
                continue
            assert code in slopes
            assert slopes[code] >= max(slopes.values()) * (1 - 1e-6)


@pytest.mark.parametrize("rule", [oracle.D8_STEEPEST, oracle.D8_LOWEST])
@pytest.mark.parametrize("shape", [(7, 9), (64, 33), (1, 12), (12, 1)])
def test_planar_closed_form(rule, shape):
    """Plane descending toward +x: area(x, y) = x + 1 with edges routing; with
    edges as sinks, interior rows give max(x, 1) and edge rows 1."""
    ny, nx = shape
    z = inputs.planar_dem(ny, nx, tilt=0.01, dx=30.0)
    xs = np.arange(nx)[None, :].repeat(ny, 0)
    _, _, a, _ = oracle.route_d8(z, 30.0, flags=oracle.EDGE_ROUTE | rule)
    np.testing.assert_array_equal(a, (xs + 1).astype(np.uint64))
    _, _, a, _ = oracle.route_d8(z, 30.0, flags=rule)
    expect = np.maximum(xs, 1)
    expect[0, :] = 1
    expect[-1, :] = 1
    if nx > 0:
        expect[:, 0] = 1
    if ny <= 2 or nx <= 2:
        expect[:] = 1
    else:
        expect[1:-1, -1] = nx - 1
    np.testing.assert_array_equal(a, expect.astype(np.uint64))


# --------------------------------------------------------- accumulation ----

@pytest.mark.parametrize("shape,seed", [((32, 32), 0), ((7, 13), 5), ((1, 30), 6),
                                        ((30, 1), 7), ((2, 2), 8), ((24, 31), 9)])
@pytest.mark.parametrize("edge", [oracle.EDGE_SINK, oracle.EDGE_ROUTE])
def test_d8_dense_solve(shape, seed, edge):
    """High-to-low sweep == LU solve of (I - W) w = r (Sec. 2.2)."""
    ny, nx = shape
    z = _dem(ny, nx, seed)
    rain = inputs.rain_field(ny, nx, seed)
    d = oracle.receivers_d8(z, 30.0, edge)
    order = oracle.high_to_low_order(z)
    w, a = oracle.accumulate_d8(d, order, rain)
    A = _dense_A_d8(d)
    ref = np.linalg.solve(A, rain.astype(np.float64).ravel())
    np.testing.assert_allclose(w.ravel(), ref, rtol=1e-12, atol=0)
    _, a1 = oracle.accumulate_d8(d, order, None)
    ref1 = np.linalg.solve(A, np.ones(nx * ny))
    np.testing.assert_array_equal(a1.ravel(), np.rint(ref1).astype(np.uint64))


@pytest.mark.parametrize("shape,seed,p", [((32, 32), 0, 1.1), ((9, 21), 4, 1.1),
                                          ((16, 16), 2, 2.0), ((1, 17), 3, 1.1)])
@pytest.mark.parametrize("edge", [oracle.EDGE_SINK, oracle.EDGE_ROUTE])
def test_mfd_dense_solve(shape, seed, p, edge):
    ny, nx = shape
    z = _dem(ny, nx, seed, beta=2.2, tilt=0.0)
    rain = inputs.rain_field(ny, nx, seed)
    m, f, w, order = oracle.route_mfd(z, 30.0, p, rain, edge)
    A = _dense_A_mfd(f)
    ref = np.linalg.solve(A, rain.astype(np.float64).ravel())
    np.testing.assert_allclose(w.ravel(), ref, rtol=1e-11, atol=0)


def test_mfd_fractions_by_hand():
    """Centre 10 m, dx = 1: lower neighbours E (s=1), N (s=2), NE (s=1), SE (s=2);
    S is equal (not lower).  p=1: f = s/6; p=2: f = s^2/10."""
    r2 = math.sqrt(2.0)
    z = np.array([[11.0, 8.0, 10.0 - r2],
                  [12.0, 10.0, 9.0],
                  [13.0, 10.0, 10.0 - 2.0 * r2]])
    for p, expect in ((1.0, [1 / 6, 2 / 6, 0, 0, 1 / 6, 0, 0, 2 / 6]),
                      (2.0, [0.1, 0.4, 0, 0, 0.1, 0, 0, 0.4])):
        m, f = oracle.receivers_mfd(z, 1.0, p, oracle.EDGE_SINK)
        np.testing.assert_allclose(f[1, 1], expect, rtol=1e-14, atol=1e-15)
        assert m[1, 1] == 0b10010011
        assert (m.ravel()[[0, 1, 2, 3, 5, 6, 7, 8]] == 0).all()


@pytest.mark.parametrize("edge", [oracle.EDGE_SINK, oracle.EDGE_ROUTE])
def test_mfd_fraction_invariants(edge):
    z = _dem(40, 37, 11, beta=2.2, tilt=0.0)
    p = 1.1
    m, f = oracle.receivers_mfd(z, 30.0, p, edge)
    tot = f.sum(-1)
    nz = m != 0
    np.testing.assert_allclose(tot[nz], 1.0, rtol=1e-14)
    assert (tot[~nz] == 0).all()
    z64 = z.astype(np.float64)
    ny, nx = z.shape
    for y in range(1, ny - 1):
        for x in range(1, nx - 1):
            ks = [k for k in range(8) if (m[y, x] >> k) & 1]
            for k in range(8):
                lower = z64[y + OFFY[k], x + OFFX[k]] < z64[y, x]
                assert bool((m[y, x] >> k) & 1) == lower
            for a in ks:
                for b in ks:
                    sa = (z64[y, x] - z64[y + OFFY[a], x + OFFX[a]]) / (30.0 * (1 if a < 4 else math.sqrt(2)))
                    sb = (z64[y, x] - z64[y + OFFY[b], x + OFFX[b]]) / (30.0 * (1 if b < 4 else math.sqrt(2)))
                    assert f[y, x, a] / f[y, x, b] == pytest.approx((sa / sb) ** p, rel=1e-12)


def test_mfd_single_row_equals_d8():
    """A monotone 1 x N strip has one lower neighbour per cell: MFD == D8."""
    z = np.linspace(100.0, 1.0, 50, dtype=np.float32)[None, :]
    _, f, w, _ = oracle.route_mfd(z, 30.0, 1.1, None, oracle.EDGE_ROUTE)
    _, wd, _, _ = oracle.route_d8(z, 30.0, None, oracle.EDGE_ROUTE)
    np.testing.assert_array_equal(w, wd)
    np.testing.assert_array_equal(w.ravel(), np.arange(1, 51, dtype=np.float64))


@pytest.mark.parametrize("seed", [0, 1])
def test_mass_balance(seed):
    z = _dem(96, 80, seed)
    rain = inputs.rain_field(96, 80, seed)
    d, w, a, _ = oracle.route_d8(z, 30.0, rain)
    s, r = oracle.mass_balance(w, rain, dir_=d)
    assert abs(s - r) <= 1e-12 * r
    sink = d == oracle.SINK
    assert int(a[sink].sum()) == z.size
    m, f, wm, _ = oracle.route_mfd(z, 30.0, 1.1, rain)
    s, r = oracle.mass_balance(wm, rain, mask=m)
    assert abs(s - r) <= 1e-12 * r


def test_bfs_upstream_counts_and_basins():
    z = _dem(128, 96, 3)
    d, _, a, _ = oracle.route_d8(z, 30.0)
    uc = oracle.UpstreamCounter(d)
    rng = np.random.default_rng(0)
    for cell in rng.integers(0, z.size, 200):
        assert uc.count(cell) == a.ravel()[cell]
    for cell in np.flatnonzero(a.ravel() > 20)[:50]:
        assert uc.count(cell) == a.ravel()[cell]
    # every cell drains to exactly one sink; basins partition the grid
    sinks = np.array([uc.sink_of(c) for c in range(z.size)])
    counts = np.bincount(sinks, minlength=z.size)
    np.testing.assert_array_equal(counts[d.ravel() == oracle.SINK],
                                  a.ravel()[d.ravel() == oracle.SINK])
    assert counts.sum() == z.size


def test_order_independence():
    """Sec. 3.2: any order that processes donors first gives the same w."""
    z = _dem(120, 77, 4)
    rain = inputs.rain_field(120, 77, 4)
    d = oracle.receivers_d8(z, 30.0)
    o1 = oracle.high_to_low_order(z)
    o2 = oracle.kahn_order(d, False)
    assert not np.array_equal(o1, o2)
    w1, a1 = oracle.accumulate_d8(d, o1, rain)
    w2, a2 = oracle.accumulate_d8(d, o2, rain)
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_allclose(w1, w2, rtol=1e-13)
    m, f = oracle.receivers_mfd(z, 30.0, 1.1)
    w1 = oracle.accumulate_mfd(f, o1, rain)
    w2 = oracle.accumulate_mfd(f, oracle.kahn_order(m, True), rain)
    np.testing.assert_allclose(w1, w2, rtol=1e-12)


def test_apply_A_residual():
    z = _dem(64, 64, 5)
    rain = inputs.rain_field(64, 64, 5)
    d, w, _, _ = oracle.route_d8(z, 30.0, rain)
    res = rain - oracle.apply_A(w, dir_=d)
    assert np.abs(res).max() <= 1e-12 * np.abs(rain).max()
    m, f, wm, _ = oracle.route_mfd(z, 30.0, 1.1, rain)
    res = rain - oracle.apply_A(wm, frac=f)
    assert np.abs(res).max() <= 1e-11 * np.abs(rain).max()


def test_degenerate_grids():
    for shape in ((1, 1), (1, 2), (2, 1), (3, 3)):
        z = np.full(shape, 5.0, np.float32)            # flat: every cell a sink
        d, w, a, _ = oracle.route_d8(z, 30.0, None, oracle.EDGE_ROUTE)
        assert (d == oracle.SINK).all()
        assert (w == 1).all() and (a == 1).all()
        m, f, wm, _ = oracle.route_mfd(z, 30.0, 1.1, None, oracle.EDGE_ROUTE)
        assert (m == 0).all() and (wm == 1).all()


# ---------------------------------------------------------------- adjoint --

def test_adjoint_d8_closed_form():
    """Loss = sum over sinks of w^2: dL/dr_i = 2 w at the sink i drains to."""
    z = _dem(64, 48, 6)
    rain = inputs.rain_field(64, 48, 6)
    d, w, _, order = oracle.route_d8(z, 30.0, rain)
    g = oracle.adjoint(order, w, dir_=d)
    uc = oracle.UpstreamCounter(d)
    sinks = np.array([uc.sink_of(c) for c in range(z.size)])
    np.testing.assert_allclose(g.ravel(), 2.0 * w.ravel()[sinks], rtol=1e-14)


@pytest.mark.parametrize("kind", ["d8", "mfd"])
def test_adjoint_dense_transpose(kind):
    """g solves A^T g = gbar (dense LU) for an arbitrary gbar."""
    z = _dem(24, 29, 7, beta=2.2)
    rain = inputs.rain_field(24, 29, 7)
    gbar = np.random.default_rng(1).standard_normal(z.shape)
    if kind == "d8":
        d, w, _, order = oracle.route_d8(z, 30.0, rain)
        g = oracle.adjoint(order, w, dir_=d, gbar=gbar)
        A = _dense_A_d8(d)
    else:
        m, f, w, order = oracle.route_mfd(z, 30.0, 1.1, rain)
        g = oracle.adjoint(order, w, frac=f, gbar=gbar)
        A = _dense_A_mfd(f)
    ref = np.linalg.solve(A.T, gbar.ravel())
    np.testing.assert_allclose(g.ravel(), ref, rtol=1e-10, atol=1e-12)


def _loss_mfd(z64, rain, p, flags=0):
    m, f = oracle.receivers_mfd(z64, 30.0, p, flags)
    order = oracle.high_to_low_order(z64)
    w = oracle.accumulate_mfd(f, order, rain)
    return float((w[m == 0] ** 2).sum())


@pytest.mark.parametrize("p", [1.1, 1.5])
def test_mfd_grad_z_finite_differences(p):
    """dL/dz (adjoint formula) vs central differences of the full FP64 solve."""
    ny, nx = 20, 18
    z = _dem(ny, nx, 8, beta=2.2, tilt=0.0).astype(np.float64)
    rain = inputs.rain_field(ny, nx, 8)
    m, f, w, order = oracle.route_mfd(z, 30.0, p, rain)
    g = oracle.adjoint(order, w, frac=f)
    dz = oracle.mfd_grad_z(z, 30.0, p, f, w, g)
    rng = np.random.default_rng(2)
    checked = 0
    for cell in rng.permutation(z.size):
        y, x = divmod(int(cell), nx)
        # step well below the smallest elevation gap around the cell so that
        # no lower set changes under the perturbation
        gaps = [abs(z[y, x] - z[y + OFFY[k], x + OFFX[k]]) for k in range(8)
                if 0 <= y + OFFY[k] < ny and 0 <= x + OFFX[k] < nx]
        h = 1e-4 * min(gaps)
        if h < 1e-7:
            continue
        zp = z.copy(); zp[y, x] += h
        zm = z.copy(); zm[y, x] -= h
        fd = (_loss_mfd(zp, rain, p) - _loss_mfd(zm, rain, p)) / (2 * h)
        assert dz[y, x] == pytest.approx(fd, rel=1e-5, abs=1e-6 * max(1.0, abs(fd)))
        checked += 1
        if checked == 40:
            break
    assert checked == 40


def _dense_loss_mfd(z, rain, p):
    """L = sum over sinks of w^2 with w from a dense solve of (I - W) w = r
    (fractions of the pinned receiver rule; no oracle accumulation)."""
    m, f = oracle.receivers_mfd(z, 30.0, p)
    A = _dense_A_mfd(f)
    r = np.ones(z.size) if rain is None else rain.astype(np.float64).ravel()
    w = np.linalg.solve(A, r).reshape(z.shape)
    return float((w[m == 0] ** 2).sum())


@pytest.mark.parametrize("p", [1.1, 1.7])
def test_mfd_delta_loss_matches_dense_finite_differences(p):
    """The incremental loss change (z and rain of one cell) reproduces central
    differences of dense re-solves, and the rain mode the adjoint dL/dr."""
    ny, nx = 18, 21
    z = _dem(ny, nx, 12, beta=2.2, tilt=0.0).astype(np.float64)
    rain = inputs.rain_field(ny, nx, 12)
    m, f, w, order = oracle.route_mfd(z, 30.0, p, rain)
    g = oracle.adjoint(order, w, frac=f)
    D = oracle.MfdLossDelta(z, 30.0, p, m, f, w)
    rng = np.random.default_rng(3)
    checked = 0
    for cell in rng.permutation(z.size):
        y, x = divmod(int(cell), nx)
        gaps = [abs(z[y, x] - z[y + OFFY[k], x + OFFX[k]]) for k in range(8)
                if 0 <= y + OFFY[k] < ny and 0 <= x + OFFX[k] < nx]
        h = 1e-4 * min(gaps)
        if h < 1e-7:
            continue
        zp = z.copy(); zp[y, x] += h
        zm = z.copy(); zm[y, x] -= h
        dense = (_dense_loss_mfd(zp, rain, p) - _dense_loss_mfd(zm, rain, p)) / (2 * h)
        assert D.central(int(cell), h, 0) == pytest.approx(dense, rel=1e-6, abs=1e-9 * max(1.0, abs(dense)))
        # rain: L is quadratic in r, so the central difference is exact
        assert D.central(int(cell), 1e-3, 1) == pytest.approx(g[y, x], rel=1e-10, abs=1e-12)
        checked += 1
        if checked == 12:
            break
    assert checked == 12
    # the scratch arrays come back cleared
    assert not D.dwork.any() and not D.mark.any()


def test_mfd_delta_loss_rejects_mask_changes():
    """A step that reorders two elevations changes a lower set: NaN."""
    ny, nx = 9, 9
    z = _dem(ny, nx, 5, beta=2.2, tilt=0.0).astype(np.float64)
    m, f, w, _ = oracle.route_mfd(z, 30.0, 1.1, None)
    D = oracle.MfdLossDelta(z, 30.0, 1.1, m, f, w)
    c = 4 * nx + 4
    gap = min(abs(z[4, 4] - z[4 + OFFY[k], 4 + OFFX[k]]) for k in range(8))
    assert np.isnan(D.delta(c, 2.0 * gap + 1.0, 0)) or np.isnan(D.delta(c, -(2.0 * gap + 1.0), 0))


# ------------------------------------------------------------------- D4 ----

def test_d4_plane_closed_form():
    """z = 10000 - 2x - y (dx = 1): D8's steepest interior receiver is SE
    (slope 3/sqrt2 > 2), D4's is E; with edge routing the last column of D4
    routes S, so areas are x + 1 along the rows and nx (y + 1) down the last
    column, ending in the corner sink with all nx*ny cells."""
    ny, nx = 7, 9
    y, x = np.mgrid[0:ny, 0:nx]
    z = (10000.0 - 2.0 * x - y).astype(np.float32)
    d8 = oracle.receivers_d8(z, 1.0, oracle.EDGE_ROUTE)
    assert (d8[:-1, :-1] == 7).all()  # SE
    d4 = oracle.receivers_d8(z, 1.0, oracle.EDGE_ROUTE | oracle.D4)
    assert (d4[:, :-1] == 0).all()    # E
    assert (d4[:-1, -1] == 3).all()   # S
    assert d4[-1, -1] == oracle.SINK
    order = oracle.high_to_low_order(z)
    _, area = oracle.accumulate_d8(d4, order, None)
    want = np.where(x < nx - 1, x + 1, nx * (y + 1)).astype(np.uint64)
    np.testing.assert_array_equal(area, want)


@pytest.mark.parametrize("seed", [1, 2])
def test_d4_dense_solve_and_codes(seed):
    ny, nx = 17, 23
    z = _dem(ny, nx, seed)
    rain = inputs.rain_field(ny, nx, seed)
    d = oracle.receivers_d8(z, 30.0, oracle.D4)
    assert set(np.unique(d)) <= {0, 1, 2, 3, oracle.SINK}
    # every D4 receiver is a strictly lower orthogonal neighbour
    for yy in range(ny):
        for xx in range(nx):
            k = d[yy, xx]
            if k != oracle.SINK:
                assert z[yy + OFFY[k], xx + OFFX[k]] < z[yy, xx]
    order = oracle.high_to_low_order(z)
    w, _ = oracle.accumulate_d8(d, order, rain)
    ref = np.linalg.solve(_dense_A_d8(d), rain.astype(np.float64).ravel())
    np.testing.assert_allclose(w.ravel(), ref, rtol=1e-12)


# ------------------------------------------------------------------ D-inf ----

@pytest.mark.parametrize("a,b,want", [
    (4.0, 1.0, {0: np.arctan2(3.0, 5.0) / (np.pi / 4), 7: np.arctan2(1.0, 4.0) / (np.pi / 4)}),
    (2.0, 2.0, {7: 1.0}),     # along the diagonal: all to SE
    (3.0, 0.0, {0: 1.0}),     # along x: all to E (first of the two tied facets)
    (1.0, 4.0, {3: np.arctan2(3.0, 5.0) / (np.pi / 4), 7: np.arctan2(1.0, 4.0) / (np.pi / 4)}),
])
def test_dinf_plane_closed_form(a, b, want):
    """z = 1000 - a x - b y (dx = 1): the steepest facet follows the gradient;
    the water splits between its cardinal and diagonal neighbours in
    proportion to the angle: f_diag = atan(min/max) / (pi/4)."""
    ny, nx = 6, 7
    y, x = np.mgrid[0:ny, 0:nx]
    z = (1000.0 - a * x - b * y).astype(np.float32)
    m, f = oracle.receivers_mfd(z.astype(np.float64), 1.0, 1.1, oracle.DINF)
    for yy in range(1, ny - 1):
        for xx in range(1, nx - 1):
            assert m[yy, xx] == sum(1 << k for k in want)
            for k in range(8):
                assert f[yy, xx, k] == pytest.approx(want.get(k, 0.0), rel=1e-14, abs=1e-15)
    assert (m[0, :] == 0).all() and (m[:, 0] == 0).all()  # edge cells are sinks


@pytest.mark.parametrize("seed", [3, 4])
def test_dinf_invariants_and_dense_solve(seed):
    ny, nx = 19, 22
    z = _dem(ny, nx, seed, beta=2.2, tilt=0.0).astype(np.float64)
    rain = inputs.rain_field(ny, nx, seed)
    m, f = oracle.receivers_mfd(z, 30.0, 1.1, oracle.DINF)
    for yy in range(ny):
        for xx in range(nx):
            bits = [k for k in range(8) if (m[yy, xx] >> k) & 1]
            assert len(bits) <= 2
            if len(bits) == 2:
                kc, kd = bits  # a cardinal and the diagonal next to it
                assert kc < 4 <= kd and kd in (4 + ((kc * 2 - 1) % 8) // 2, 4 + (kc * 2) // 2 % 4)
            for k in bits:
                assert z[yy + OFFY[k], xx + OFFX[k]] < z[yy, xx]
            if bits:
                assert f[yy, xx].sum() == pytest.approx(1.0, abs=1e-14)
            assert all(f[yy, xx, k] == 0.0 for k in range(8) if k not in bits)
    order = oracle.high_to_low_order(z)
    w = oracle.accumulate_mfd(f, order, rain)
    ref = np.linalg.solve(_dense_A_mfd(f), rain.astype(np.float64).ravel())
    np.testing.assert_allclose(w.ravel(), ref, rtol=1e-12)


# ------------------------------------------------------------------ depression filling
def _relax_fill(z):
    """Planchon-Darboux relaxation written independently of the oracle: start
    from +inf inside and lower every interior cell to max(z, min over
    neighbours of the next fp32 value above the neighbour) until nothing moves."""
    z = np.asarray(z, np.float32)
    ny, nx = z.shape
    edge = np.zeros((ny, nx), bool)
    edge[0, :] = edge[-1, :] = edge[:, 0] = edge[:, -1] = True
    F = np.where(edge, z, np.float32(np.inf)).astype(np.float32)
    while True:
        P = np.full((ny + 2, nx + 2), np.inf, np.float32)
        P[1:-1, 1:-1] = F
        m = np.full((ny, nx), np.inf, np.float32)
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dy or dx:
                    m = np.minimum(m, np.nextafter(P[1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx],
                                                   np.float32(np.inf)))
        G = np.where(edge, z, np.maximum(z, np.minimum(F, m))).astype(np.float32)
        if np.array_equal(G, F):
            return F
        F = G


def test_fill_plane_is_unchanged():
    """A plane falling towards the west edge already drains: filling is the identity."""
    yy, xx = np.mgrid[0:9, 0:12]
    z = (0.5 * xx + 0.01 * yy).astype(np.float32)
    np.testing.assert_array_equal(oracle.fill(z), z)


def test_fill_pit_by_hand():
    """A 4x4 basin whose outlet is the corner at 4: the cell next to the outlet
    sits one fp32 step above it, the others one step above that."""
    z = np.array([[5, 5, 5, 5], [5, 1, 2, 5], [5, 3, 0, 5], [5, 5, 5, 4]], np.float32)
    s1 = np.nextafter(np.float32(4), np.float32(np.inf))
    s2 = np.nextafter(s1, np.float32(np.inf))
    want = np.array([[5, 5, 5, 5], [5, s2, s2, 5], [5, s2, s1, 5], [5, 5, 5, 4]], np.float32)
    np.testing.assert_array_equal(oracle.fill(z), want)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (2, 5), (3, 3), (7, 11), (16, 13), (24, 24)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fill_matches_relaxation(shape, seed):
    """Priority-flood against the independent relaxation, bit for bit, on rough
    random surfaces (many pits and flats)."""
    rng = np.random.default_rng(seed)
    z = rng.integers(0, 6, size=shape).astype(np.float32)  # integer heights: many flats
    np.testing.assert_array_equal(oracle.fill(z), _relax_fill(z))
    z = rng.random(shape, dtype=np.float32) * 10
    np.testing.assert_array_equal(oracle.fill(z), _relax_fill(z))


def test_fill_invariants_and_drainage():
    """On a fractal DEM: F >= z, edges unchanged, the defining equation holds at
    every interior cell (so F is the least such surface), and D8 routing on F
    leaves sinks only on the edge."""
    z = inputs.fractal_dem(64, 80, beta=2.0, tilt=0.0, seed=5)
    F = oracle.fill(z)
    assert (F >= z).all()
    np.testing.assert_array_equal(F[0], z[0])
    np.testing.assert_array_equal(F[-1], z[-1])
    np.testing.assert_array_equal(F[:, 0], z[:, 0])
    np.testing.assert_array_equal(F[:, -1], z[:, -1])
    P = np.full((66, 82), np.inf, np.float32)
    P[1:-1, 1:-1] = F
    m = np.full((64, 80), np.inf, np.float32)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy or dx:
                m = np.minimum(m, np.nextafter(P[1 + dy:65 + dy, 1 + dx:81 + dx], np.float32(np.inf)))
    np.testing.assert_array_equal(F[1:-1, 1:-1], np.maximum(z, m)[1:-1, 1:-1])
    d = oracle.receivers_d8(F, 30.0)
    assert (d[1:-1, 1:-1] != oracle.SINK).all()
    assert (oracle.receivers_d8(z, 30.0)[1:-1, 1:-1] == oracle.SINK).any()  # the DEM had pits
