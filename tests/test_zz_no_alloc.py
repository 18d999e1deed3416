"""fr_route_d8_noalloc: the D8 route on the library's own fixed device scratch.

The entry point serves callers that cannot allocate device memory.  It must
return exactly what fr_route_d8 (caller workspace) returns, and what the CPU
oracle computes, on consecutive calls that share the scratch, and reject grids
above its limit.  This file is
collected last so that it also runs after every other test in one process.
"""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest
import torch

import oracle
from paper_2606_12800_gb300 import _lib, inputs

RTOL_W = 1e-6
HEADER = Path(__file__).resolve().parents[1] / "include" / "fr.h"


def test_noalloc_limit_matches_header():
    m = re.search(r"#define\s+FR_NOALLOC_MAX_CELLS\s+\(\(int64_t\)1\s*<<\s*(\d+)\)", HEADER.read_text())
    assert m and (1 << int(m.group(1))) == _lib.FR_NOALLOC_MAX_CELLS


def test_noalloc_rejects_oversized_grids_before_device_work():
    L = _lib.load()
    big = _lib.FR_NOALLOC_MAX_CELLS
    for nx, ny in ((big + 1, 1), (1, big + 1), (1025, 1024), (4096, 4096), (0, 5), (5, 0)):
        st = L.fr_route_d8_noalloc(None, nx, ny, 30.0, 0, None, None, None, None, None, None)
        assert st == _lib.FR_ERR_INVALID_ARG, (nx, ny, st)


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _route(L, fn, z, rain, dx, flags, ws=None):
    ny, nx = z.shape
    dev = z.device
    w = torch.full((ny, nx), float("nan"), dtype=torch.float32, device=dev)
    lo = torch.full((ny, nx), float("nan"), dtype=torch.float32, device=dev)
    a = torch.full((ny, nx), -1, dtype=torch.int64, device=dev)
    d = torch.full((ny, nx), 0xEE, dtype=torch.uint8, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    if fn == "fr_route_d8":
        st = L.fr_route_d8(_p(z), nx, ny, dx, flags, _p(rain), _p(w), _p(lo), _p(a), _p(d),
                           _p(ws), ws.numel(), stream)
    else:
        st = L.fr_route_d8_noalloc(_p(z), nx, ny, dx, flags, _p(rain), _p(w), _p(lo), _p(a),
                                   _p(d), stream)
    assert st == _lib.FR_OK, (fn, st)
    torch.cuda.synchronize(dev)
    return w.cpu().numpy(), lo.cpu().numpy(), a.cpu().numpy(), d.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_matches_route_d8_on_consecutive_calls():
    L = _lib.load()
    dev = torch.device("cuda:0")
    # two calls in a row on the shared scratch: the full limit, then a ragged
    # smaller grid that finds the first call's contents in the scratch
    cases = [((1024, 1024), 7, 30.0, 0, True), ((333, 517), 8, 10.0, _lib.FR_EDGE_ROUTE, False)]
    for (ny, nx), seed, dx, flags, with_rain in cases:
        assert nx * ny <= _lib.FR_NOALLOC_MAX_CELLS
        z = torch.from_numpy(inputs.fractal_dem(ny, nx, seed=seed, dx=dx)).to(dev)
        rain = torch.from_numpy(inputs.rain_field(ny, nx, seed)).to(dev) if with_rain else None
        ws = torch.empty(L.fr_workspace_size(_lib.FR_OP_ROUTE, nx, ny, flags), dtype=torch.uint8,
                         device=dev)
        w0, lo0, a0, d0 = _route(L, "fr_route_d8", z, rain, dx, flags, ws)
        w1, lo1, a1, d1 = _route(L, "fr_route_d8_noalloc", z, rain, dx, flags)
        np.testing.assert_array_equal(d1, d0)
        np.testing.assert_array_equal(a1, a0)
        full0 = w0.astype(np.float64) + lo0
        full1 = w1.astype(np.float64) + lo1
        np.testing.assert_allclose(full1, full0, rtol=RTOL_W, atol=0)
        np.testing.assert_allclose(w1, w0, rtol=RTOL_W, atol=0)
        assert np.isfinite(w1).all() and (a1 >= 1).all()
        # and directly against the oracle (FP64 water, uint64 areas)
        zn = z.cpu().numpy()
        rn = rain.cpu().numpy() if rain is not None else None
        d_ref, w_ref, _, order = oracle.route_d8(zn, dx, rn, flags)
        _, a_ref = oracle.accumulate_d8(d_ref, order, None)
        np.testing.assert_array_equal(d1, d_ref)
        np.testing.assert_array_equal(a1.astype(np.uint64), a_ref)
        assert np.max(np.abs(w1.astype(np.float64) - w_ref) / w_ref) <= RTOL_W
