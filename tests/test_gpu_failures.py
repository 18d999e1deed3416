"""Failure detection and the remaining boundary calls on the GPU.

Every failure here is made on the host side of the kernels: a wait limit of
zero that no grid barrier can meet, a DEM holding NaN or Inf, routings with
cycles.  No test faults, traps or hangs the GPU; each call returns and its
status word says what happened, and the same workspace is clean on the next
good call.  Also: a batched route captured in a CUDA graph and replayed on
new inputs, and receiver indices in int32/int64 form, against the oracle.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2606_12800_gb300 import _lib, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL_W = 1e-6
NO_PROGRESS = _lib.FR_ERR_NO_PROGRESS


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


def test_grid_barrier_wait_limit(api):
    """The MFD global phase runs in rounds separated by a grid barrier whose
    wait is bounded.  With the limit set to zero every block that has to
    wait gives up at once: the call returns and reports FR_ERR_NO_PROGRESS.
    With the default restored the same workspace routes correctly."""
    ny, nx = 1024, 1536
    z = inputs.fractal_dem(ny, nx, beta=2.2, tilt=0.0, seed=44)
    zt = cuda(z)
    _, _, w_ref, _ = oracle.route_mfd(z, 30.0, 1.1, None)
    prev = api.set_wait_limit(0)
    try:
        assert prev == 10 * 1000 ** 3
        api.route_mfd(zt, 30.0, 1.1, None, 0)
        assert api.get_status() == NO_PROGRESS
        # the adjoint's rounds use the same barrier
        m = api.receivers_mfd(zt, 30.0, 1.1)
        R = api.routing_mfd(m, zt, 30.0, 1.1)
        o = api.accumulate(R, None, want_w=True, want_lo=True)
        api.get_status()
        api.adjoint(R, o["w"], o["w_lo"])
        assert api.get_status() == NO_PROGRESS
    finally:
        assert api.set_wait_limit(prev) == 0
    out = api.route_mfd(zt, 30.0, 1.1, None, 0)
    assert api.get_status() == 0
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W


def test_nonfinite_dem_is_rejected(api):
    L = _lib.load()
    P = ctypes.c_void_p
    ny, nx = 300, 517
    for bad in (np.nan, np.inf, -np.inf):
        z = inputs.fractal_dem(ny, nx, seed=3)
        z[123, 456] = bad
        zt = cuda(z)
        d = torch.empty((ny, nx), dtype=torch.uint8, device="cuda")
        s = api._stream()
        st = L.fr_receivers_d8(P(zt.data_ptr()), nx, ny, 30.0, _lib.FR_CHECK_FINITE, P(d.data_ptr()),
                               None, s)
        assert st == _lib.FR_ERR_NONFINITE
        st = L.fr_receivers_mfd(P(zt.data_ptr()), nx, ny, 30.0, 1.1, _lib.FR_CHECK_FINITE,
                                P(d.data_ptr()), None, None, s)
        assert st == _lib.FR_ERR_NONFINITE
        ws = api.workspace(nx, ny)
        a = torch.empty((ny, nx), dtype=torch.int64, device="cuda")
        st = L.fr_route_d8(P(zt.data_ptr()), nx, ny, 30.0, _lib.FR_CHECK_FINITE, None, None, None,
                           P(a.data_ptr()), None, P(ws.data_ptr()), ws.numel(), s)
        assert st == _lib.FR_ERR_NONFINITE
        with pytest.raises(_lib.FrError) as e:
            api.fill(zt, flags=_lib.FR_CHECK_FINITE)
        assert e.value.status == _lib.FR_ERR_NONFINITE
    # a finite DEM passes the check and routes as usual
    z = inputs.fractal_dem(ny, nx, seed=3)
    out = api.route_d8(cuda(z), 30.0, None, _lib.FR_CHECK_FINITE, want_w=False, want_area=True)
    assert api.get_status() == 0
    _, _, a_ref, _ = oracle.route_d8(z, 30.0)
    np.testing.assert_array_equal(out["area"].cpu().numpy().astype(np.uint64), a_ref)


def _cyclic_mask(ny, nx):
    """Receiver masks with two-cell cycles: inside one 64x64 tile, across the
    border x = 63 | 64 and across y = 63 | 64, plus a chain feeding one."""
    m = np.zeros((ny, nx), np.uint8)
    E, N, W, S = 1, 2, 4, 8
    m[10, 10], m[10, 11] = E, W
    m[20, 63], m[20, 64] = E, W
    m[63, 100], m[64, 100] = S, N
    m[150, 20:150] = E
    m[150, 150], m[150, 151] = E, W
    return m


def test_mfd_cycles_report_no_progress(api):
    """A cyclic mask routing through the MFD accumulation and the MFD and D8
    adjoints: the cells on the cycles (and below them) are never reached,
    every call returns and reports FR_ERR_NO_PROGRESS."""
    ny, nx = 200, 300
    m = _cyclic_mask(ny, nx)
    z = cuda(inputs.planar_dem(ny, nx, 0.01, 30.0))
    R = api.routing_mfd(cuda(m), z, 30.0, 1.1)
    o = api.accumulate(R, None, want_w=True, want_lo=True)
    assert api.get_status() == NO_PROGRESS
    api.adjoint(R, o["w"], o["w_lo"])
    assert api.get_status() == NO_PROGRESS
    # D8 codes with the same cycles: the adjoint's rounds
    d = np.full((ny, nx), oracle.SINK, np.uint8)
    for (y, x), k in {(10, 10): 0, (10, 11): 2, (20, 63): 0, (20, 64): 2, (63, 100): 3,
                      (64, 100): 1, (150, 150): 0, (150, 151): 2}.items():
        d[y, x] = k
    d[150, 20:150] = 0
    Rd = api.routing_d8(cuda(d))
    w = torch.ones((ny, nx), dtype=torch.float32, device="cuda")
    api.adjoint(Rd, w)
    assert api.get_status() == NO_PROGRESS
    # clean again on a good routing
    zz = inputs.fractal_dem(ny, nx, beta=2.2, tilt=0.0, seed=5)
    out = api.route_mfd(cuda(zz), 30.0, 1.1, None, 0)
    assert api.get_status() == 0
    _, _, w_ref, _ = oracle.route_mfd(zz, 30.0, 1.1, None)
    assert relerr(out["w"].cpu().numpy(), w_ref) <= RTOL_W


@pytest.mark.parametrize("kind", ["d8", "mfd"])
def test_batch_graph_capture_and_replay(api, kind):
    """fr_route_batch captured once in a CUDA graph, then replayed after new
    DEMs and rain were copied into the same input buffers: each replay equals
    the oracle on the new inputs."""
    L = _lib.load()
    P = ctypes.c_void_p
    specs = [(17, 23, 2.0), (64, 64, 1.8), (31, 200, 2.4), (130, 97, 2.1), (300, 257, 2.0),
             (5, 5, 2.2), (1, 40, 2.0), (256, 300, 1.9), (128, 64, 2.3), (700, 650, 2.0)]
    k = _lib.FR_ROUTING_D8 if kind == "d8" else _lib.FR_ROUTING_MFD
    dems = [torch.empty((a, b), dtype=torch.float32, device="cuda") for a, b, _ in specs]
    rains = [torch.empty_like(d) for d in dems]
    route = [torch.empty(d.shape, dtype=torch.uint8, device="cuda") for d in dems]
    w = [torch.empty_like(d) for d in dems]
    area = [torch.empty(d.shape, dtype=torch.int64, device="cuda") for d in dems]
    arr = (_lib.fr_tile * len(specs))()
    for i, (a, b, _) in enumerate(specs):
        t = arr[i]
        t.dem, t.rain, t.w_out, t.w_lo_out = dems[i].data_ptr(), rains[i].data_ptr(), w[i].data_ptr(), None
        t.area_out = area[i].data_ptr() if kind == "d8" else None
        t.route_out, t.nx, t.ny, t.dx = route[i].data_ptr(), b, a, 30.0
    tiles_dev = torch.frombuffer(bytearray(bytes(memoryview(arr).cast("B"))), dtype=torch.uint8).cuda()
    need = int(L.fr_batch_workspace_size(arr, len(specs), k, 0))
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")

    def fill_inputs(seed):
        host = []
        for i, (a, b, beta) in enumerate(specs):
            z = inputs.fractal_dem(a, b, beta=beta, tilt=0.0, seed=seed + i)
            r = inputs.rain_field(a, b, seed + i)
            dems[i].copy_(torch.from_numpy(z))
            rains[i].copy_(torch.from_numpy(r))
            host.append((z, r))
        return host

    def call():
        _lib.check(L.fr_route_batch(arr, P(tiles_dev.data_ptr()), len(specs), k, 1.1, 0,
                                    P(ws.data_ptr()), need, api._stream()), "fr_route_batch")

    fill_inputs(100)
    call()  # warm-up outside the capture (sets the kernels' shared-memory limits)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        call()
    for seed in (200, 300):
        host = fill_inputs(seed)
        g.replay()
        torch.cuda.synchronize()
        assert int(L.fr_get_status(P(ws.data_ptr()), need, api._stream())) == 0
        for i, (z, r) in enumerate(host):
            if kind == "d8":
                d_ref, w_ref, _, order = oracle.route_d8(z, 30.0, r)
                _, a_ref = oracle.accumulate_d8(d_ref, order, None)
                np.testing.assert_array_equal(route[i].cpu().numpy(), d_ref)
                np.testing.assert_array_equal(area[i].cpu().numpy().astype(np.uint64), a_ref)
            else:
                m_ref, _, w_ref, _ = oracle.route_mfd(z, 30.0, 1.1, r)
                np.testing.assert_array_equal(route[i].cpu().numpy(), m_ref)
            assert relerr(w[i].cpu().numpy(), w_ref) <= RTOL_W


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (33, 65), (300, 517)])
@pytest.mark.parametrize("flags", [0, oracle.EDGE_ROUTE])
def test_receiver_index(api, shape, flags):
    ny, nx = shape
    z = inputs.fractal_dem(ny, nx, seed=nx + 2 * ny)
    d_ref = oracle.receivers_d8(z, 30.0, flags)
    yy, xx = np.mgrid[0:ny, 0:nx]
    ox = np.array(oracle.OFFX + (0,) * 248)[d_ref.astype(np.int64)]
    oy = np.array(oracle.OFFY + (0,) * 248)[d_ref.astype(np.int64)]
    ref = np.where(d_ref == oracle.SINK, -1, (yy + oy) * nx + xx + ox)
    d = api.receivers_d8(cuda(z), 30.0, flags)
    for wide in (True, False):
        got = api.receiver_index(d, wide=wide).cpu().numpy()
        assert got.dtype == (np.int64 if wide else np.int32)
        np.testing.assert_array_equal(got.astype(np.int64), ref)
    # codes that point out of the grid read as sinks
    dd = np.full((4, 5), 1, np.uint8)  # N everywhere: row 0 points outside
    got = api.receiver_index(cuda(dd)).cpu().numpy()
    assert (got[0] == -1).all() and (got[1:] == (np.arange(3)[:, None] * 5 + np.arange(5))).all()
