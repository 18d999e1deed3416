"""CPU oracle for flow routing -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The GPU
product path never imports it and shares no code with it (no kernels, headers,
helpers or constants); the two meet only in the seeded input generators.

The arithmetic lives in ``fr_oracle.c`` (plain C loops, FP64 / uint64, built
with ``-ffp-contract=off``).  This module is argument marshalling over ctypes
plus numpy conveniences.  Each function cites the passage of the paper it
follows (Bangerth, "Massively parallel flow routing and drainage area
determination"):

* ``receivers_d8`` / ``receivers_mfd`` -- local flow routing, Sec. 2.1 and
  App. A.
* ``high_to_low_order`` + ``accumulate_d8`` / ``accumulate_mfd`` -- the
  sequential high-to-low algorithm, Sec. 2.1 (Eq. high-to-low-procedure).
* ``kahn_order`` -- a second valid processing order, Sec. 3.2.
* ``apply_A`` -- the matrix-free product, Sec. 3.1 and App. A.
* ``adjoint`` / ``mfd_grad_z`` -- g = A^{-T} gbar by the reverse sweep; the
  elevation gradient through the MFD weights (A is triangular in high-to-low
  numbering, Sec. 2.4).
* ``mass_balance`` -- outflow at sinks vs total rain, Sec. 4.
* ``upstream_count`` / ``sink_of`` -- per-cell checks for grids too large to
  sort.

Every function here is pinned by ``tests/test_oracle.py`` against values the
paper prints (the 3x3 example of Fig. 1), closed forms, dense linear solves and
invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfr_oracle.so")
_SRC = os.path.join(_HERE, "fr_oracle.c")

SINK = 0xFF
EDGE_SINK = 0
EDGE_ROUTE = 1
D8_STEEPEST = 0
D8_LOWEST = 2
D4 = 8
DINF = 16

OFFX = (1, 0, -1, 0, 1, -1, -1, 1)
OFFY = (0, -1, 0, 1, -1, -1, 1, 1)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, IEEE semantics, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fexcess-precision=standard", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        L.or_receivers_d8.argtypes = [P, I64, I64, ctypes.c_double, ctypes.c_uint32, P]
        L.or_receivers_mfd.argtypes = [P, I64, I64, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint32, P, P]
        L.or_indegree.argtypes = [P, ctypes.c_int, I64, I64, P]
        L.or_high_to_low_order.argtypes = [P, I64, P]
        L.or_high_to_low_order64.argtypes = [P, I64, P]
        L.or_accumulate_d8.argtypes = [P, P, P, I64, I64, P, P]
        L.or_accumulate_mfd.argtypes = [P, P, P, I64, I64, P]
        L.or_kahn_order.argtypes = [P, ctypes.c_int, I64, I64, P]
        L.or_kahn_order.restype = I64
        L.or_apply_A.argtypes = [P, P, I64, I64, P, P]
        L.or_adjoint.argtypes = [P, P, P, I64, I64, P, P, P]
        L.or_mfd_grad_z.argtypes = [P, I64, I64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_uint32, P, P, P, P]
        L.or_mass_balance.argtypes = [P, P, I64, P, P, P]
        L.or_upstream_count.argtypes = [P, I64, I64, I64, P, P]
        L.or_upstream_count.restype = ctypes.c_uint64
        L.or_sink_of.argtypes = [P, I64, I64, I64]
        L.or_mfd_delta_loss.argtypes = [P, I64, I64, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_uint32, P, P, P, I64, ctypes.c_double,
                                        ctypes.c_int, P, P]
        L.or_mfd_delta_loss.restype = ctypes.c_double
        L.or_sink_of.restype = I64
        L.or_fill.argtypes = [P, I64, I64, P]
        L.or_fill.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(z):
    return np.ascontiguousarray(z, dtype=np.float32)


def receivers_d8(z, dx: float, flags: int = 0) -> np.ndarray:
    """D8 direction code per cell (0..7 or SINK), Sec. 2.1."""
    z = _f32(z)
    ny, nx = z.shape
    d = np.empty((ny, nx), np.uint8)
    lib().or_receivers_d8(_p(z), nx, ny, float(dx), int(flags), _p(d))
    return d


def receivers_mfd(z, dx: float, p: float = 1.1, flags: int = 0):
    """MFD receiver mask (bit k) and FP64 fractions (ny, nx, 8), App. A.

    ``z`` may be float32 or float64; it is used in FP64 (float32 converts
    exactly)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    ny, nx = z.shape
    m = np.empty((ny, nx), np.uint8)
    f = np.empty((ny, nx, 8), np.float64)
    lib().or_receivers_mfd(_p(z), nx, ny, float(dx), float(p), int(flags), _p(m), _p(f))
    return m, f


def indegree(routing, is_mask: bool) -> np.ndarray:
    r = np.ascontiguousarray(routing, dtype=np.uint8)
    ny, nx = r.shape
    out = np.empty((ny, nx), np.uint8)
    lib().or_indegree(_p(r), int(bool(is_mask)), nx, ny, _p(out))
    return out


def high_to_low_order(z) -> np.ndarray:
    """Cell indices sorted by (z descending, index ascending), Sec. 2.1.

    float64 input is sorted in FP64, anything else as float32."""
    order = np.empty(np.asarray(z).size, np.int64)
    if np.asarray(z).dtype == np.float64:
        z = np.ascontiguousarray(z)
        lib().or_high_to_low_order64(_p(z), z.size, _p(order))
    else:
        z = _f32(z)
        lib().or_high_to_low_order(_p(z), z.size, _p(order))
    return order


def accumulate_d8(dir_, order, rain=None, want_w: bool = True, want_area: bool = True):
    """High-to-low water passing for D8 (Eq. high-to-low-procedure).

    Returns (w FP64 or None, area uint64 or None); rain None = unit rain."""
    dir_ = np.ascontiguousarray(dir_, dtype=np.uint8)
    ny, nx = dir_.shape
    r = None if rain is None else _f32(rain)
    w = np.empty((ny, nx), np.float64) if want_w else None
    a = np.empty((ny, nx), np.uint64) if want_area else None
    lib().or_accumulate_d8(_p(dir_), _p(np.ascontiguousarray(order, np.int64)), _p(r),
                           nx, ny, _p(w), _p(a))
    return w, a


def accumulate_mfd(frac, order, rain=None) -> np.ndarray:
    """High-to-low water passing with fractions (App. A)."""
    frac = np.ascontiguousarray(frac, dtype=np.float64)
    ny, nx = frac.shape[:2]
    r = None if rain is None else _f32(rain)
    w = np.empty((ny, nx), np.float64)
    lib().or_accumulate_mfd(_p(frac), _p(np.ascontiguousarray(order, np.int64)), _p(r),
                            nx, ny, _p(w))
    return w


def kahn_order(routing, is_mask: bool) -> np.ndarray:
    """Kahn topological order (donors before receivers), Sec. 3.2."""
    r = np.ascontiguousarray(routing, dtype=np.uint8)
    ny, nx = r.shape
    order = np.empty(nx * ny, np.int64)
    got = lib().or_kahn_order(_p(r), int(bool(is_mask)), nx, ny, _p(order))
    if got != nx * ny:
        raise ValueError("routing graph has a cycle")
    return order


def apply_A(x, dir_=None, frac=None) -> np.ndarray:
    """Matrix-free y = A x, Sec. 3.1 (D8) / App. A (fractions)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    ny, nx = x.shape
    y = np.empty_like(x)
    d = None if dir_ is None else np.ascontiguousarray(dir_, np.uint8)
    f = None if frac is None else np.ascontiguousarray(frac, np.float64)
    lib().or_apply_A(_p(d), _p(f), nx, ny, _p(x), _p(y))
    return y


def adjoint(order, w, dir_=None, frac=None, gbar=None) -> np.ndarray:
    """g = A^{-T} gbar (= dL/dr); gbar None = loss sum over sinks of w^2."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    ny, nx = w.shape
    g = np.empty_like(w)
    d = None if dir_ is None else np.ascontiguousarray(dir_, np.uint8)
    f = None if frac is None else np.ascontiguousarray(frac, np.float64)
    gb = None if gbar is None else np.ascontiguousarray(gbar, np.float64)
    lib().or_adjoint(_p(d), _p(f), _p(np.ascontiguousarray(order, np.int64)), nx, ny,
                     _p(w), _p(gb), _p(g))
    return g


def mfd_grad_z(z, dx, p, frac, w, g, flags: int = 0) -> np.ndarray:
    """dL/dz through the MFD fractions, lower sets held fixed."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    ny, nx = z.shape
    out = np.empty((ny, nx), np.float64)
    lib().or_mfd_grad_z(_p(z), nx, ny, float(dx), float(p), int(flags),
                        _p(np.ascontiguousarray(frac, np.float64)),
                        _p(np.ascontiguousarray(w, np.float64)),
                        _p(np.ascontiguousarray(g, np.float64)), _p(out))
    return out


class MfdLossDelta:
    """Exact change of L = sum over sinks of w^2 when z (mode 0) or the rain
    (mode 1) of one cell changes, for finite-difference checks of the adjoint
    (see or_mfd_delta_loss).  Keeps the FP64 routing of one grid."""

    def __init__(self, z, dx, p, mask, frac, w, flags: int = 0):
        self.z = np.ascontiguousarray(z, dtype=np.float64)
        self.ny, self.nx = self.z.shape
        self.dx, self.p, self.flags = float(dx), float(p), int(flags)
        self.mask = np.ascontiguousarray(mask, np.uint8)
        self.frac = np.ascontiguousarray(frac, np.float64)
        self.w = np.ascontiguousarray(w, np.float64)
        self.dwork = np.zeros(self.z.size, np.float64)
        self.mark = np.zeros(self.z.size, np.uint8)

    def delta(self, cell: int, delta: float, mode: int) -> float:
        return float(lib().or_mfd_delta_loss(
            _p(self.z), self.nx, self.ny, self.dx, self.p, self.flags, _p(self.mask),
            _p(self.frac), _p(self.w), int(cell), float(delta), int(mode), _p(self.dwork),
            _p(self.mark)))

    def central(self, cell: int, h: float, mode: int) -> float:
        """(L(x + h) - L(x - h)) / 2h for x = z[cell] (mode 0) or its rain."""
        return (self.delta(cell, h, mode) - self.delta(cell, -h, mode)) / (2.0 * h)


def mass_balance(w, rain=None, dir_=None, mask=None):
    """(sum of w over sinks, sum of rain), Sec. 4."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.empty(2, np.float64)
    d = None if dir_ is None else np.ascontiguousarray(dir_, np.uint8)
    m = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    r = None if rain is None else _f32(rain)
    lib().or_mass_balance(_p(d), _p(m), w.size, _p(r), _p(w), _p(out))
    return float(out[0]), float(out[1])


class UpstreamCounter:
    """Upstream basin size of single cells by BFS over reversed D8 edges."""

    def __init__(self, dir_):
        self.dir = np.ascontiguousarray(dir_, dtype=np.uint8)
        self.ny, self.nx = self.dir.shape
        self._work = np.empty(self.dir.size, np.int64)
        self._seen = np.zeros(self.dir.size, np.uint8)

    def count(self, cell: int) -> int:
        return int(lib().or_upstream_count(_p(self.dir), self.nx, self.ny, int(cell),
                                           _p(self._work), _p(self._seen)))

    def sink_of(self, cell: int) -> int:
        return int(lib().or_sink_of(_p(self.dir), self.nx, self.ny, int(cell)))


def route_d8(z, dx, rain=None, flags: int = 0):
    """Convenience: receivers + high-to-low accumulation (FP64 w, uint64 area)."""
    d = receivers_d8(z, dx, flags)
    order = high_to_low_order(z)
    w, a = accumulate_d8(d, order, rain)
    return d, w, a, order


def route_mfd(z, dx, p=1.1, rain=None, flags: int = 0):
    """Convenience: MFD fractions + high-to-low accumulation (FP64)."""
    m, f = receivers_mfd(z, dx, p, flags)
    order = high_to_low_order(z)
    w = accumulate_mfd(f, order, rain)
    return m, f, w, order


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))


def fill(z) -> np.ndarray:
    """Depression filling (the step before the path, Sec. 4): the least surface
    F >= z, equal to z on the edge, in which every interior cell has a
    neighbour lower by at least one fp32 step (priority-flood)."""
    z = _f32(z)
    ny, nx = z.shape
    out = np.empty_like(z)
    if lib().or_fill(_p(z), nx, ny, _p(out)) != 0:
        raise MemoryError("or_fill: out of memory")
    return out
