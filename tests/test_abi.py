"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/fr.h declares, and rejects bad arguments synchronously."""
import ctypes
import os
import re

import pytest

from paper_2606_12800_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_lib.EXPORTS)


def test_status_strings_and_version(lib):
    for code in range(7):
        assert lib.fr_status_string(code)
    assert lib.fr_version() >= 100


def test_workspace_size(lib):
    assert lib.fr_workspace_size(_lib.FR_OP_RECEIVERS, 10, 10, 0) == 0
    n = lib.fr_workspace_size(_lib.FR_OP_ACCUMULATE, 4096, 4096, 0)
    assert n >= 4096 * 4096 * 13
    assert n % 256 == 0
    assert lib.fr_workspace_size(_lib.FR_OP_ACCUMULATE, 0, 10, 0) == 0
    assert lib.fr_workspace_size(_lib.FR_OP_ACCUMULATE, 10, 10, 0x200) == 0  # an unknown flag
    assert lib.fr_workspace_size(_lib.FR_OP_ACCUMULATE, 1 << 21, 1 << 21, 0) == 0  # > 2^40 cells
    # MFD operations keep 8 fp32 fractions per cell on top of the common part
    m = lib.fr_workspace_size(_lib.FR_OP_MFD, 4096, 4096, 0)
    assert m >= n + 4096 * 4096 * 32 and m % 256 == 0
    # fill: a batch of sweep counters plus two change records per 64x32 tile
    f = lib.fr_workspace_size(_lib.FR_OP_FILL, 4096, 4096, 0)
    assert f >= 256 + 2 * (4096 // 64) * (4096 // 32) and f % 256 == 0


def test_argument_validation_is_synchronous(lib):
    P = ctypes.c_void_p
    fake = P(0x1000)
    # null DEM / output, bad sizes, bad dx, unknown flags: rejected before any CUDA call
    assert lib.fr_receivers_d8(None, 4, 4, 1.0, 0, fake, None, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receivers_d8(fake, 0, 4, 1.0, 0, fake, None, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receivers_d8(fake, 4, 4, -1.0, 0, fake, None, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receivers_d8(fake, 4, 4, float("nan"), 0, fake, None, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receivers_d8(fake, 4, 4, 1.0, 0x100, fake, None, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receivers_mfd(fake, 4, 4, 1.0, 0.0, 0, fake, None, None, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receivers_mfd(fake, 4, 4, 1.0, 65.0, 0, fake, None, None, None) == _lib.FR_ERR_INVALID_ARG
    # D4 is a D8-only rule
    assert lib.fr_receivers_mfd(fake, 4, 4, 1.0, 1.1, _lib.FR_D4, fake, None, None, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_workspace_size(_lib.FR_OP_ROUTE, 4, 4, _lib.FR_D4) > 0
    # fill: overlapping input and output, no sweeps, unknown flags, small workspace
    n = ctypes.c_int32(0)
    assert lib.fr_fill(fake, 4, 4, 0, P(0x1010), 10, ctypes.byref(n), fake, 256, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_fill(fake, 4, 4, 0, P(0x100000), 0, None, fake, 256, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_fill(fake, 4, 4, _lib.FR_EDGE_ROUTE, P(0x100000), 5, None, fake, 256, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_fill(fake, 4, 4, 0, P(0x100000), 5, None, fake, 16, None) == _lib.FR_ERR_WORKSPACE
    # D-infinity is an MFD-only split
    assert lib.fr_receivers_d8(fake, 4, 4, 1.0, _lib.FR_DINF, fake, None, None) == _lib.FR_ERR_INVALID_ARG
    # fractions need 16-byte alignment
    assert lib.fr_receivers_mfd(fake, 4, 4, 1.0, 1.1, 0, fake, P(0x1004), None, None) == _lib.FR_ERR_INVALID_ARG
    R = _lib.fr_routing()
    R.kind = 7
    R.nx = R.ny = 4
    assert lib.fr_accumulate(ctypes.byref(R), None, fake, None, None, fake, 1 << 20, None) == _lib.FR_ERR_INVALID_ARG
    R.kind = _lib.FR_ROUTING_D8
    R.dir = 0x1000
    # no output requested
    assert lib.fr_accumulate(ctypes.byref(R), None, None, None, None, fake, 1 << 20, None) == _lib.FR_ERR_INVALID_ARG
    # workspace missing / too small / misaligned
    assert lib.fr_accumulate(ctypes.byref(R), None, fake, None, None, None, 0, None) == _lib.FR_ERR_WORKSPACE
    assert lib.fr_accumulate(ctypes.byref(R), None, fake, None, None, fake, 16, None) == _lib.FR_ERR_WORKSPACE
    assert lib.fr_accumulate(ctypes.byref(R), None, fake, None, None, P(0x1001), 1 << 20, None) == _lib.FR_ERR_WORKSPACE
    # MFD: area output is D8-only; dL/dz is MFD-only
    R.kind = _lib.FR_ROUTING_MFD
    R.mask = 0x1000
    R.dem = 0x1000
    R.dx = 30.0
    R.p = 1.1
    assert lib.fr_accumulate(ctypes.byref(R), None, fake, None, fake, fake, 1 << 20, None) == _lib.FR_ERR_INVALID_ARG
    # an MFD routing needs the larger workspace (fractions)
    small = lib.fr_workspace_size(_lib.FR_OP_ACCUMULATE, 4, 4, 0)
    assert lib.fr_accumulate(ctypes.byref(R), None, fake, None, None, P(0x10000), small, None) == _lib.FR_ERR_WORKSPACE
    R.p = 100.0
    assert lib.fr_accumulate(ctypes.byref(R), None, fake, None, None, P(0x10000), 1 << 20, None) == _lib.FR_ERR_INVALID_ARG
    R.p = 1.1
    R.kind = _lib.FR_ROUTING_D8
    assert lib.fr_route_adjoint(ctypes.byref(R), fake, None, None, fake, fake, fake, 1 << 20, None) == _lib.FR_ERR_INVALID_ARG
    R.reserved = 1
    assert lib.fr_mass_balance(ctypes.byref(R), None, fake, None, None, fake, fake, 1 << 20, None) == _lib.FR_ERR_INVALID_ARG


def test_receiver_index_and_wait_limit_validation(lib):
    P = ctypes.c_void_p
    fake = P(0x1000)
    assert lib.fr_receiver_index(None, 4, 4, 8, fake, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receiver_index(fake, 4, 4, 8, None, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receiver_index(fake, 4, 4, 2, fake, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receiver_index(fake, 0, 4, 4, fake, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receiver_index(fake, 1 << 16, 1 << 16, 4, fake, None) == _lib.FR_ERR_INVALID_ARG
    prev = lib.fr_set_wait_limit(123)
    assert lib.fr_set_wait_limit(prev) == 123


def test_batch_and_global_phase_flags_validation(lib):
    P = ctypes.c_void_p
    tiles = (_lib.fr_tile * 1)()
    t = tiles[0]
    t.dem, t.route_out, t.w_out, t.nx, t.ny, t.dx = 0x1000, 0x2000, 0x3000, 8, 8, 30.0
    assert lib.fr_batch_workspace_size(tiles, 1, _lib.FR_ROUTING_D8, 0) > 0
    assert lib.fr_batch_workspace_size(tiles, 1 << 24, _lib.FR_ROUTING_D8, 0) == 0
    R = _lib.fr_routing()
    R.kind, R.nx, R.ny, R.dir = _lib.FR_ROUTING_D8, 8, 8, 0x1000
    R.flags = _lib.FR_GLOBAL_WALKERS | _lib.FR_GLOBAL_SKELETON
    fake = P(0x1000)
    assert lib.fr_accumulate(ctypes.byref(R), None, None, None, fake, fake, 1 << 20, None) == \
        _lib.FR_ERR_INVALID_ARG


def test_weights_flag_only_for_mfd_routings(lib):
    """FR_WEIGHTS_IN_WORKSPACE describes an MFD routing's workspace: D8
    routings, the receiver calls and the fused routes reject it."""
    fake = ctypes.c_void_p(0x1000)
    W = _lib.FR_WEIGHTS_IN_WORKSPACE
    R = _lib.fr_routing()
    R.kind, R.nx, R.ny, R.dir, R.flags = _lib.FR_ROUTING_D8, 8, 8, 0x1000, W
    assert lib.fr_accumulate(ctypes.byref(R), None, None, None, fake, fake, 1 << 20, None) == \
        _lib.FR_ERR_INVALID_ARG
    assert lib.fr_route_adjoint(ctypes.byref(R), fake, None, None, fake, None, fake, 1 << 20,
                                None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receivers_d8(fake, 8, 8, 30.0, W, fake, None, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receivers_mfd(fake, 8, 8, 30.0, 1.1, W, fake, None, None, None) == \
        _lib.FR_ERR_INVALID_ARG
    assert lib.fr_route_d8(fake, 8, 8, 30.0, W, None, fake, None, None, None, fake, 1 << 20,
                           None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_route_mfd(fake, 8, 8, 30.0, 1.1, W, None, fake, None, None, fake, 1 << 20,
                            None) == _lib.FR_ERR_INVALID_ARG


def test_sink_sums_flag_only_for_d8_routings(lib):
    """FR_SINK_SUMS_IN_WORKSPACE describes a D8 accumulation's workspace: MFD
    routings, the receiver calls and the fused routes reject it, and the
    mass balance with it needs areas and no water."""
    fake = ctypes.c_void_p(0x1000)
    S = _lib.FR_SINK_SUMS_IN_WORKSPACE
    R = _lib.fr_routing()
    R.kind, R.nx, R.ny, R.mask, R.dem, R.dx, R.p, R.flags = \
        _lib.FR_ROUTING_MFD, 8, 8, 0x1000, 0x2000, 30.0, 1.1, S
    ws = 1 << 22
    assert lib.fr_accumulate(ctypes.byref(R), None, fake, None, None, fake, ws, None) == \
        _lib.FR_ERR_INVALID_ARG
    assert lib.fr_mass_balance(ctypes.byref(R), None, None, None, fake, fake, fake, ws, None) == \
        _lib.FR_ERR_INVALID_ARG
    assert lib.fr_receivers_d8(fake, 8, 8, 30.0, S, fake, None, None) == _lib.FR_ERR_INVALID_ARG
    assert lib.fr_route_d8(fake, 8, 8, 30.0, S, None, fake, None, None, None, fake, ws,
                           None) == _lib.FR_ERR_INVALID_ARG
    D = _lib.fr_routing()
    D.kind, D.nx, D.ny, D.dir, D.flags = _lib.FR_ROUTING_D8, 8, 8, 0x1000, S
    assert lib.fr_mass_balance(ctypes.byref(D), None, fake, None, fake, fake, fake, ws, None) == \
        _lib.FR_ERR_INVALID_ARG  # water
    assert lib.fr_mass_balance(ctypes.byref(D), None, None, None, None, fake, fake, ws, None) == \
        _lib.FR_ERR_INVALID_ARG  # no areas
