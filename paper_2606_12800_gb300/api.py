"""Python API over the C ABI (torch tensors in, torch tensors out).

PyTorch supplies device memory and the current CUDA stream; all arithmetic
runs in libfr.so.  Functions accept CUDA tensors; the ``route_*`` helpers also
accept CPU tensors (pinned memory recommended), in which case the inputs are
copied to the GPU and the results copied back (the end-to-end path).
"""
from __future__ import annotations

import ctypes
from typing import Dict, Optional

import torch

from . import _lib
from ._lib import (FR_ROUTING_D8, FR_ROUTING_MFD, FR_OP_FILL, FR_OP_MFD, FR_OP_ROUTE,
                   FR_WEIGHTS_IN_WORKSPACE, check, fr_routing, load)

# one workspace per (device, stream): calls on different streams may overlap
_ws_cache: Dict[tuple, torch.Tensor] = {}


def _stream() -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_grid(t: torch.Tensor, dtype, name: str):
    if t.dim() != 2:
        raise ValueError("%s must be 2-D (ny, nx)" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s" % (name, dtype))
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


def workspace(nx: int, ny: int, device=None, mfd: bool = False) -> torch.Tensor:
    """A cached workspace large enough for any operation on an nx-by-ny grid
    (with room for the fractions of an MFD routing when ``mfd``)."""
    dev = torch.device(device if device is not None else "cuda")
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    need = workspace_size(nx, ny, mfd)
    key = (idx, torch.cuda.current_stream(torch.device("cuda", idx)).cuda_stream)
    ws = _ws_cache.get(key)
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device=torch.device("cuda", idx))
        _ws_cache[key] = ws
    return ws


def workspace_size(nx: int, ny: int, mfd: bool = False) -> int:
    """Bytes of a workspace for any operation on an nx-by-ny grid (fr_workspace_size)."""
    need = int(load().fr_workspace_size(FR_OP_MFD if mfd else FR_OP_ROUTE, nx, ny, 0))
    if need == 0:
        raise ValueError("invalid grid size %dx%d" % (nx, ny))
    return need


def routing_d8(dir_: torch.Tensor, flags: int = 0) -> fr_routing:
    """D8 routing descriptor; flags: 0, FR_GLOBAL_WALKERS or FR_GLOBAL_SKELETON
    (the global phase of the accumulation, see fr.h)."""
    R = fr_routing()
    R.kind = FR_ROUTING_D8
    R.ny, R.nx = dir_.shape
    R.dir = dir_.data_ptr()
    R.flags = flags
    R._keep = (dir_,)  # the descriptor holds raw pointers: keep the tensors alive
    return R


def routing_mfd(mask: torch.Tensor, dem: torch.Tensor, dx: float, p: float, flags: int = 0) -> fr_routing:
    R = fr_routing()
    R.kind = FR_ROUTING_MFD
    R.ny, R.nx = mask.shape
    R.mask = mask.data_ptr()
    R.dem = dem.data_ptr()
    R.dx = dx
    R.p = p
    R.flags = flags
    R._keep = (mask, dem)
    return R


def receivers_d8(dem: torch.Tensor, dx: float = 30.0, flags: int = 0, indeg: bool = False):
    """D8 receiver codes (uint8; 0..7 or 255), optionally donor counts."""
    _check_grid(dem, torch.float32, "dem")
    ny, nx = dem.shape
    d = torch.empty((ny, nx), dtype=torch.uint8, device=dem.device)
    n = torch.empty_like(d) if indeg else None
    check(load().fr_receivers_d8(_p(dem), nx, ny, dx, flags, _p(d), _p(n), _stream()),
          "fr_receivers_d8")
    return (d, n) if indeg else d


def receivers_mfd(dem: torch.Tensor, dx: float = 30.0, p: float = 1.1, flags: int = 0,
                  frac: bool = False, indeg: bool = False):
    """MFD receiver masks (uint8), optionally fractions (ny, nx, 8) and donor counts."""
    _check_grid(dem, torch.float32, "dem")
    ny, nx = dem.shape
    m = torch.empty((ny, nx), dtype=torch.uint8, device=dem.device)
    f = torch.empty((ny, nx, 8), dtype=torch.float32, device=dem.device) if frac else None
    n = torch.empty_like(m) if indeg else None
    check(load().fr_receivers_mfd(_p(dem), nx, ny, dx, p, flags, _p(m), _p(f), _p(n), _stream()),
          "fr_receivers_mfd")
    out = (m,)
    if frac:
        out += (f,)
    if indeg:
        out += (n,)
    return out if len(out) > 1 else m


def accumulate(R: fr_routing, rain: Optional[torch.Tensor] = None, want_w: bool = True,
               want_lo: bool = False, want_area: bool = False, device=None,
               ws: Optional[torch.Tensor] = None) -> Dict[str, torch.Tensor]:
    """Water per cell for a routing (D8 or MFD); see fr_accumulate.  ws: a
    workspace of the caller's (workspace_size bytes), e.g. to keep the MFD
    fractions for a later adjoint (FR_WEIGHTS_IN_WORKSPACE)."""
    ny, nx = R.ny, R.nx
    dev = device or torch.device("cuda", torch.cuda.current_device())
    if rain is not None:
        _check_grid(rain, torch.float32, "rain")
        dev = rain.device
    out: Dict[str, torch.Tensor] = {}
    w = torch.empty((ny, nx), dtype=torch.float32, device=dev) if want_w else None
    lo = torch.empty((ny, nx), dtype=torch.float32, device=dev) if want_lo else None
    a = torch.empty((ny, nx), dtype=torch.int64, device=dev) if want_area else None
    if ws is None:
        ws = workspace(nx, ny, dev, mfd=R.kind == FR_ROUTING_MFD)
    check(load().fr_accumulate(ctypes.byref(R), _p(rain), _p(w), _p(lo), _p(a), _p(ws),
                               ws.numel(), _stream()), "fr_accumulate")
    if w is not None:
        out["w"] = w
    if lo is not None:
        out["w_lo"] = lo
    if a is not None:
        out["area"] = a
    return out


def _to_cuda(t):
    if t is None or t.is_cuda:
        return t, False
    return t.to("cuda", non_blocking=True), True


def _to_host(out: Dict[str, torch.Tensor]) -> Dict[str, torch.Tensor]:
    """Device results into page-locked host tensors (torch's caching host
    allocator), copied asynchronously, then one synchronisation."""
    res = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()}
    for k, v in out.items():
        res[k].copy_(v, non_blocking=True)
    torch.cuda.current_stream().synchronize()
    return res


def route_d8(dem: torch.Tensor, dx: float = 30.0, rain: Optional[torch.Tensor] = None,
             flags: int = 0, want_w: bool = True, want_lo: bool = False, want_area: bool = True,
             want_dir: bool = False) -> Dict[str, torch.Tensor]:
    """Receivers + accumulation (D8) in one call (fr_route_d8).

    CPU inputs are copied to the GPU and the outputs back to the CPU."""
    dem_d, host = _to_cuda(dem)
    rain_d, _ = _to_cuda(rain)
    _check_grid(dem_d, torch.float32, "dem")
    ny, nx = dem_d.shape
    dev = dem_d.device
    w = torch.empty((ny, nx), dtype=torch.float32, device=dev) if want_w else None
    lo = torch.empty((ny, nx), dtype=torch.float32, device=dev) if want_lo else None
    a = torch.empty((ny, nx), dtype=torch.int64, device=dev) if want_area else None
    d = torch.empty((ny, nx), dtype=torch.uint8, device=dev) if want_dir else None
    ws = workspace(nx, ny, dev)
    check(load().fr_route_d8(_p(dem_d), nx, ny, dx, flags, _p(rain_d), _p(w), _p(lo), _p(a), _p(d),
                             _p(ws), ws.numel(), _stream()), "fr_route_d8")
    out = {k: v for k, v in (("w", w), ("w_lo", lo), ("area", a), ("dir", d)) if v is not None}
    if host:
        out = _to_host(out)
    return out


def route_mfd(dem: torch.Tensor, dx: float = 30.0, p: float = 1.1,
              rain: Optional[torch.Tensor] = None, flags: int = 0, want_lo: bool = False,
              want_mask: bool = False, ws: Optional[torch.Tensor] = None) -> Dict[str, torch.Tensor]:
    """Receivers + accumulation (MFD) in one call (fr_route_mfd).  ws: a
    workspace of the caller's (workspace_size(nx, ny, mfd=True) bytes), which
    then keeps the fractions for a later adjoint (FR_WEIGHTS_IN_WORKSPACE)."""
    dem_d, host = _to_cuda(dem)
    rain_d, _ = _to_cuda(rain)
    _check_grid(dem_d, torch.float32, "dem")
    ny, nx = dem_d.shape
    dev = dem_d.device
    w = torch.empty((ny, nx), dtype=torch.float32, device=dev)
    lo = torch.empty((ny, nx), dtype=torch.float32, device=dev) if want_lo else None
    m = torch.empty((ny, nx), dtype=torch.uint8, device=dev) if want_mask else None
    if ws is None:
        ws = workspace(nx, ny, dev, mfd=True)
    check(load().fr_route_mfd(_p(dem_d), nx, ny, dx, p, flags, _p(rain_d), _p(w), _p(lo), _p(m),
                              _p(ws), ws.numel(), _stream()), "fr_route_mfd")
    out = {k: v for k, v in (("w", w), ("w_lo", lo), ("mask", m)) if v is not None}
    if host:
        out = _to_host(out)
    return out


def accumulate_richardson(R: fr_routing, rain: Optional[torch.Tensor] = None, order: int = 1,
                          max_iterations: int = 10000, want_lo: bool = False, device=None):
    """The paper's Richardson iteration on 64x32 tiles (fr_accumulate_richardson;
    order 1: I+X, order 2: (I-X)(I+X)): ({"w", "w_lo"}, iterations until exact)."""
    ny, nx = R.ny, R.nx
    dev = device or torch.device("cuda", torch.cuda.current_device())
    if rain is not None:
        _check_grid(rain, torch.float32, "rain")
        dev = rain.device
    w = torch.empty((ny, nx), dtype=torch.float32, device=dev)
    lo = torch.empty((ny, nx), dtype=torch.float32, device=dev) if want_lo else None
    ws = workspace(nx, ny, dev, mfd=R.kind == FR_ROUTING_MFD)
    it = ctypes.c_int32(0)
    check(load().fr_accumulate_richardson(ctypes.byref(R), _p(rain), _p(w), _p(lo), int(order),
                                          int(max_iterations), ctypes.byref(it), _p(ws),
                                          ws.numel(), _stream()), "fr_accumulate_richardson")
    out = {"w": w}
    if lo is not None:
        out["w_lo"] = lo
    return out, int(it.value)


def fill(dem: torch.Tensor, max_sweeps: int = 100000, flags: int = 0):
    """Depression filling (fr_fill): (filled DEM, sweeps run)."""
    _check_grid(dem, torch.float32, "dem")
    ny, nx = dem.shape
    out = torch.empty_like(dem)
    ws = torch.empty(int(load().fr_workspace_size(FR_OP_FILL, nx, ny, 0)), dtype=torch.uint8,
                     device=dem.device)
    sweeps = ctypes.c_int32(0)
    check(load().fr_fill(_p(dem), nx, ny, flags, _p(out), int(max_sweeps), ctypes.byref(sweeps),
                         _p(ws), ws.numel(), _stream()), "fr_fill")
    return out, int(sweeps.value)


def adjoint(R: fr_routing, w: torch.Tensor, w_lo: Optional[torch.Tensor] = None,
            dLdw: Optional[torch.Tensor] = None, want_dz: bool = False,
            ws: Optional[torch.Tensor] = None):
    """(dL/dr, dL/dz or None) for L = sum over sinks of w^2, or for the
    incoming gradient dLdw (fr_route_adjoint).  ws: a workspace of the
    caller's; with FR_WEIGHTS_IN_WORKSPACE in R.flags it must hold R's
    fractions from the forward call."""
    ny, nx = R.ny, R.nx
    dev = w.device
    dLdr = torch.empty((ny, nx), dtype=torch.float32, device=dev)
    dLdz = torch.empty((ny, nx), dtype=torch.float32, device=dev) if want_dz else None
    if ws is None:
        ws = workspace(nx, ny, dev, mfd=R.kind == FR_ROUTING_MFD)
    check(load().fr_route_adjoint(ctypes.byref(R), _p(w), _p(w_lo), _p(dLdw), _p(dLdr), _p(dLdz),
                                  _p(ws), ws.numel(), _stream()), "fr_route_adjoint")
    return dLdr, dLdz


def mass_balance(R: fr_routing, rain=None, w=None, w_lo=None, area=None, device=None) -> torch.Tensor:
    """Device tensor [sum over sinks of w, sum of rain, sum over sinks of area]."""
    dev = device or torch.device("cuda", torch.cuda.current_device())
    out = torch.empty(3, dtype=torch.float64, device=dev)
    ws = workspace(R.nx, R.ny, dev)
    check(load().fr_mass_balance(ctypes.byref(R), _p(rain), _p(w), _p(w_lo), _p(area), _p(out),
                                 _p(ws), ws.numel(), _stream()), "fr_mass_balance")
    return out


def get_status(device=None, ws: Optional[torch.Tensor] = None) -> int:
    """Synchronises the current stream and returns (and clears) the device
    status word of the workspace ws, by default the cached one (0 = ok)."""
    if ws is None:
        dev = torch.device(device if device is not None else "cuda")
        idx = dev.index if dev.index is not None else torch.cuda.current_device()
        ws = _ws_cache.get((idx, torch.cuda.current_stream(torch.device("cuda", idx)).cuda_stream))
    if ws is None:
        return 0
    return int(load().fr_get_status(_p(ws), ws.numel(), _stream()))


def receiver_index(dir_: torch.Tensor, wide: bool = True) -> torch.Tensor:
    """Linear receiver index of every cell (-1 for sinks) from D8 codes
    (fr_receiver_index); int64, or int32 with wide=False."""
    _check_grid(dir_, torch.uint8, "dir")
    ny, nx = dir_.shape
    out = torch.empty((ny, nx), dtype=torch.int64 if wide else torch.int32, device=dir_.device)
    check(load().fr_receiver_index(_p(dir_), nx, ny, 8 if wide else 4, _p(out), _stream()),
          "fr_receiver_index")
    return out


def set_wait_limit(ns: int) -> int:
    """Limit of device-side waits in nanoseconds (fr_set_wait_limit); returns
    the previous limit."""
    return int(load().fr_set_wait_limit(int(ns)))


class RouteMFD(torch.autograd.Function):
    """w = route_mfd(dem, rain) with a hand-written adjoint backward
    (gradients with respect to the elevations and the rain).

    keep_weights: keep the forward's workspace, with its 32 B/cell fractions,
    until the backward, which then reads the fractions instead of recomputing
    them from the DEM and the mask (FR_WEIGHTS_IN_WORKSPACE).  By default
    only the DEM, the mask and the two-float water are kept (13 B/cell) and
    the backward recomputes the fractions: the checkpoint of the weights."""

    @staticmethod
    def forward(ctx, dem, rain, dx: float = 30.0, p: float = 1.1, flags: int = 0,
                keep_weights: bool = False):
        mask = receivers_mfd(dem, dx, p, flags)
        R = routing_mfd(mask, dem, dx, p, flags)
        ws = None
        if keep_weights:
            ny, nx = dem.shape
            ws = torch.empty(workspace_size(nx, ny, mfd=True), dtype=torch.uint8, device=dem.device)
        out = accumulate(R, rain, want_w=True, want_lo=True, device=dem.device, ws=ws)
        ctx.save_for_backward(dem, mask, out["w"], out["w_lo"])
        ctx.cfg = (dx, p, flags)
        ctx.ws = ws
        return out["w"]

    @staticmethod
    def backward(ctx, grad_w):
        dem, mask, w, w_lo = ctx.saved_tensors
        dx, p, flags = ctx.cfg
        want_dz = ctx.needs_input_grad[0]
        want_dr = ctx.needs_input_grad[1]
        if not (want_dz or want_dr):
            return None, None, None, None, None, None
        kept = ctx.ws is not None
        R = routing_mfd(mask, dem, dx, p, flags | (FR_WEIGHTS_IN_WORKSPACE if kept else 0))
        dLdr, dLdz = adjoint(R, w, w_lo, dLdw=grad_w.contiguous().float(), want_dz=want_dz, ws=ctx.ws)
        ctx.ws = None
        return (dLdz if want_dz else None), (dLdr if want_dr else None), None, None, None, None


def route_batch(dems, rains=None, kind: str = "d8", dx: float = 30.0, p: float = 1.1,
                flags: int = 0, want_w: bool = True, want_lo: bool = False,
                want_area: bool = False, autotune: bool = False):
    """Routes many independent DEMs (CUDA float32 2-D tensors) with one
    fr_route_batch call.  Returns a list of dicts (route, w, w_lo, area)."""
    from ._lib import fr_tile
    if kind not in ("d8", "mfd"):
        raise ValueError("kind must be 'd8' or 'mfd'")
    k = FR_ROUTING_D8 if kind == "d8" else FR_ROUTING_MFD
    n = len(dems)
    if n == 0:
        return []
    dev = dems[0].device
    outs, arr = [], (fr_tile * n)()
    for i, z in enumerate(dems):
        _check_grid(z, torch.float32, "dem")
        ny, nx = z.shape
        r = None if rains is None else rains[i]
        if r is not None:
            _check_grid(r, torch.float32, "rain")
        o = {"route": torch.empty((ny, nx), dtype=torch.uint8, device=dev)}
        if want_w:
            o["w"] = torch.empty((ny, nx), dtype=torch.float32, device=dev)
        if want_lo:
            o["w_lo"] = torch.empty((ny, nx), dtype=torch.float32, device=dev)
        if want_area:
            o["area"] = torch.empty((ny, nx), dtype=torch.int64, device=dev)
        t = arr[i]
        t.dem, t.rain = z.data_ptr(), (r.data_ptr() if r is not None else None)
        t.w_out = o["w"].data_ptr() if want_w else None
        t.w_lo_out = o["w_lo"].data_ptr() if want_lo else None
        t.area_out = o["area"].data_ptr() if want_area else None
        t.route_out = o["route"].data_ptr()
        t.nx, t.ny, t.dx = nx, ny, dx
        outs.append(o)
    raw = bytes(memoryview(arr).cast("B"))
    tiles_dev = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(dev)
    L = load()
    need = int(L.fr_batch_workspace_size(arr, n, k, flags))
    if need == 0:
        raise ValueError("invalid batch")
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    fn = L.fr_batch_autotune if autotune else L.fr_route_batch
    check(fn(arr, _p(tiles_dev), n, k, p, flags, _p(ws), need, _stream()), "fr_route_batch")
    outs[0]["_ws"] = ws  # keeps the workspace (and its status word) alive
    outs[0]["_tiles"] = tiles_dev
    return outs


def batch_status(outs) -> int:
    """Status word of a route_batch call (synchronises the stream)."""
    ws = outs[0]["_ws"]
    return int(load().fr_get_status(_p(ws), ws.numel(), _stream()))
