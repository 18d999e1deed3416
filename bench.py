#!/usr/bin/env python3
"""Benchmark: cells routed per second on one GB300 (D8 and slope-split).

Headline workload (one step = one pass of the hot path over one synthetic DEM):
  D8 on a 32768 x 32768 float32 fractal DEM (beta 2, tilt 0.005, jitter 1e-4 m,
  dx 30 m) with unit rain: receivers, exact uint64 drainage areas and the
  mass-balance check.  `roofline` is the accumulation call at 9 algorithmic
  bytes per cell (codes in, areas out); `step_roofline` the whole step at 12
  (elevations in, areas out).

Sibling key `slope_split`: the slope-split (MFD, p = 1.1) route on an
8192 x 8192 DEM (beta 2.2, no tilt, unit rain) with the same fields (value,
roofline at 8 bytes per cell, e2e, cpu_baseline, error against the oracle).
Other extra keys report the previous 4096^2 D8 step with rain, long-river
inputs, the batched route, the adjoint, the paper's Richardson iteration and
the depression fill, each timed the same way.

Timing: W untimed warm-up steps, then exactly K timed steps, each bracketed by
CUDA events on the launching stream; the inputs are larger than L2 and L2 is
also flushed (a 512 MiB write) between steps, outside the events; barrier +
synchronize around the timed loop, max over ranks.  With --gpus N > 1
(torchrun) every rank routes its own replica (the path has no exchange step)
and the value is the sum over ranks.

--impl reference times the CPU oracle (the paper's sequential high-to-low
algorithm, FP64/uint64, single thread) on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# headline: D8 32768^2, beta 2, tilt 0.005, unit rain, uint64 areas
N_SIDE = 32768
D8_BETA, D8_TILT, D8_SEED = 2.0, 0.005, 6
# sibling: slope-split 8192^2, beta 2.2, no tilt, unit rain
MFD_SIDE = 8192
MFD_BETA, MFD_P, MFD_SEED = 2.2, 1.1, 3
DX = 30.0
SEED = 1
# CPU oracle samples (crops of the same DEMs)
D8_CROP = 4096
MFD_CROP = 2048

METRIC = "cells routed/sec at 1 GB300 (D8 & slope-split)"

# Sources that define each profiled kernel: a traffic figure from a profile
# summary counts only while these files are unchanged since the capture.
KERNEL_SOURCES = {
    "k_local_d8": ["fr_d8.cu", "fr_engine.cuh", "fr_device.cuh", "fr_internal.h"],
    "k_local_halo_mfd": ["fr_halo.cu", "fr_engine.cuh", "fr_device.cuh", "fr_internal.h"],
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="skip every extra row")
    ap.add_argument("--rows", default="slope_split,d8_4096,long_rivers,batched,adjoint,richardson,fill",
                    help="comma-separated extra rows to run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baselines")
    ap.add_argument("--side", type=int, default=N_SIDE, help="headline grid side (default 32768)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def sources_sha(kernel):
    """sha256 (first 16 hex digits) over the sources that define `kernel`."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2606_12800_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_traffic(kernel, cells):
    """DRAM bytes (read + write) of one launch of `kernel` on `cells` cells,
    from the `traffic-record` line of a committed ncu summary under profiles/:
    scaled by cells from the captured size; None when no summary was taken of
    the kernel as its sources stand now."""
    want = sources_sha(kernel)
    pat = re.compile(r"traffic-record:\s*kernel=(\S+)\s+cells=(\d+)\s+dram_bytes=(\d+)\s+sources=(\w+)")
    found = None
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for m in pat.finditer(f.read()):
                if m.group(1) == kernel:
                    found = (int(m.group(2)), int(m.group(3)), m.group(4), os.path.basename(path))
                    if m.group(4) == want:
                        c, b = found[0], found[1]
                        return b * cells / c, "ncu dram read+write, %s (%d cells, scaled to %d)" % (
                            found[3], c, cells)
    if found:
        return None, "the kernel changed since %s was captured" % found[3]
    return None, "no ncu summary of this kernel"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_init(n, backend="nccl"):
    """One process per GPU (torchrun sets RANK / LOCAL_RANK / WORLD_SIZE /
    MASTER_*); the replicas share nothing but the barrier and the timing."""
    import torch
    if n <= 1:
        return 0, 1
    import torch.distributed as dist
    dist.init_process_group(backend)
    rank = dist.get_rank()
    if backend == "nccl":
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", rank)))
    return rank, dist.get_world_size()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, world):
    """The largest x over all ranks (the slowest replica sets the job time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, cells, total_ms):
    """Whole-job throughput: the cells of every rank's steps over the slowest
    rank's time (weak scaling: each replica routes its own DEM)."""
    return world * steps * cells / (total_ms * 1e-3)


def step_config(n, world):
    """The `config` of the step's JSON line (the same for both arms)."""
    return {"workload": "D8 %dx%d fractal DEM (beta=2, tilt=0.005, jitter 1e-4 m, dx=30 m), "
                        "unit rain: receivers + exact uint64 drainage areas + mass balance" % (n, n),
            "global_batch": world, "cells_per_step": n * n,
            "l2": "inputs larger than L2; also flushed between steps (512 MiB write)",
            "parallelism": "replicas"}


# ----------------------------------------------------------------- reference
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2606_12800_gb300 import inputs
    oracle.build()
    side = 1024  # bounded sample: a 1024^2 DEM of the workload's recipe per step
    z = inputs.fractal_dem(side, side, beta=D8_BETA, tilt=D8_TILT, seed=D8_SEED, dx=DX)

    def one():
        d, w, _, _ = oracle.route_d8(z, DX, None)
        oracle.mass_balance(w, None, dir_=d)
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    value = args.steps * side * side / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "cells/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": step_config(args.side, args.gpus),
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": 1, "kind": "oracle",
                         "sample": "%dx%d DEM of the workload's recipe per step (receivers, "
                                   "unit-rain areas, mass balance; sequential high-to-low, "
                                   "FP64/uint64), scaled to cells/s" % (side, side)},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------- ours
def count_launches(fn):
    """Number of this library's kernels (names in namespace fr) one call of fn
    launches, from the CUDA activity record of the torch profiler."""
    import torch
    from torch.profiler import ProfilerActivity, profile
    try:
        n = None
        for _ in range(2):  # the first profile of a process may miss kernels
            with profile(activities=[ProfilerActivity.CUDA]) as prof:
                fn()
                torch.cuda.synchronize()
            n = sum(e.count for e in prof.key_averages() if "fr::" in e.key)
        return n
    except Exception:  # pragma: no cover
        return None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import ctypes

    import torch
    from paper_2606_12800_gb300 import _lib, api, inputs
    rank, world = dist_init(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    L = _lib.load()
    stream = torch.cuda.current_stream()
    sp = lambda: api._stream()  # noqa: E731
    P = ctypes.c_void_p

    # inputs resident in HBM
    n = args.side
    cells = n * n
    z = inputs.fractal_dem_torch(n, n, beta=D8_BETA, tilt=D8_TILT, seed=D8_SEED, dx=DX, device="cuda")
    dir_ = torch.empty((n, n), dtype=torch.uint8, device=dev)
    area = torch.empty((n, n), dtype=torch.int64, device=dev)
    mb = torch.empty(3, dtype=torch.float64, device=dev)
    ws = api.workspace(n, n, dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    # the mass balance takes its area term from the sums the accumulation
    # formed where it wrote the areas (FR_SINK_SUMS_IN_WORKSPACE)
    R = api.routing_d8(dir_, _lib.FR_SINK_SUMS_IN_WORKSPACE)
    wsp, wsn = P(ws.data_ptr()), ws.numel()

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        _lib.check(L.fr_receivers_d8(P(z.data_ptr()), n, n, DX, 0, P(dir_.data_ptr()), None, sp()),
                   "fr_receivers_d8")
        if evs:
            evs[1].record(stream)
        _lib.check(L.fr_accumulate(ctypes.byref(R), None, None, None, P(area.data_ptr()), wsp, wsn,
                                   sp()), "fr_accumulate")
        if evs:
            evs[2].record(stream)
        _lib.check(L.fr_mass_balance(ctypes.byref(R), None, None, None, P(area.data_ptr()),
                                     P(mb.data_ptr()), wsp, wsn, sp()), "fr_mass_balance")
        if evs:
            evs[3].record(stream)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    status = api.get_status(dev)
    mbv = mb.cpu().numpy()
    assert status == 0, "device status %d" % status
    assert mbv[2] == cells and mbv[1] == cells, mbv
    # the full pass over the stored areas gives the same bits
    full = api.mass_balance(api.routing_d8(dir_), area=area, device=dev).cpu().numpy()
    assert full.tobytes() == mbv.tobytes(), (full, mbv)

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    for i in range(K):
        flush.zero_()
        step(evs[i])
    torch.cuda.synchronize()
    barrier(world)
    step_ms = [e[0].elapsed_time(e[3]) for e in evs]
    recv_ms = [e[0].elapsed_time(e[1]) for e in evs]
    acc_ms = [e[1].elapsed_time(e[2]) for e in evs]
    mb_ms = [e[2].elapsed_time(e[3]) for e in evs]
    total_ms = allmax(sum(step_ms), world)
    clk = clocks.stop()
    if clk is None or clk.get("samples", 0) < 3:
        # timed region shorter than the sampling period: soak the same step
        clocks.start()
        t_end = time.time() + 1.5
        while time.time() < t_end:
            for _ in range(10):
                flush.zero_()
                step()
            torch.cuda.synchronize()
        clk2 = clocks.stop()
        if clk2:
            clk2["window"] = "timed region + 1.5 s soak of the same step"
            clk = clk2
    launches = count_launches(step)
    status = api.get_status(dev)
    assert status == 0, "device status %d" % status

    value = job_value(world, K, cells, total_ms)
    peak, peak_kind = peaks()
    acc_avg = statistics.mean(acc_ms) * 1e-3
    acc_bytes = cells * 9                     # codes 1 in, areas 8 out
    achieved = acc_bytes / acc_avg / 1e9
    step_bytes = cells * 12                   # elevations 4 in, areas 8 out
    traffic, traffic_note = profile_traffic("k_local_d8", cells)

    # parity on a crop of the same DEM (GPU and oracle route the same bytes)
    crop = None
    cpu = None
    if rank == 0 and not args.no_cpu:
        zc = np.ascontiguousarray(z[:D8_CROP, :D8_CROP].cpu().numpy())
        cpu, crop = d8_crop_check(api, zc)

    # end to end through the public API: the DEM from pinned host memory to
    # the device, fr_route_d8 and the mass balance there, the areas, the codes
    # and the mass balance back into pinned host buffers; copies timed
    z_host = z.cpu().pin_memory()
    del z, dir_, area
    torch.cuda.empty_cache()
    area_h = torch.empty((n, n), dtype=torch.int64, pin_memory=True)
    dir_h = torch.empty((n, n), dtype=torch.uint8, pin_memory=True)
    mb_h = torch.empty(3, dtype=torch.float64, pin_memory=True)
    e2e_ms = []
    for i in range(max(3, min(K, 5)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        zd = z_host.to(dev, non_blocking=True)
        out = api.route_d8(zd, DX, None, 0, want_w=False, want_area=True, want_dir=True)
        Rh = api.routing_d8(out["dir"], _lib.FR_SINK_SUMS_IN_WORKSPACE)
        m = api.mass_balance(Rh, area=out["area"], device=dev)
        area_h.copy_(out["area"], non_blocking=True)
        dir_h.copy_(out["dir"], non_blocking=True)
        mb_h.copy_(m, non_blocking=True)
        torch.cuda.synchronize()
        if i >= 1:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        del zd, out, Rh, m
    assert mb_h[2].item() == cells and mb_h[1].item() == cells, mb_h
    e2e = {"value": cells / (statistics.median(e2e_ms) * 1e-3), "unit": "cells/s",
           "h2d_bytes_per_step": cells * 4, "d2h_bytes_per_step": cells * 9 + 24,
           "ms_per_step": statistics.median(e2e_ms),
           "path": "pinned host DEM to the device, api.route_d8 (fr_route_d8) and api.mass_balance "
                   "there, areas + codes + mass balance into pinned host buffers"}
    del z_host, area_h, dir_h, mb_h
    torch.cuda.empty_cache()

    extra = {}
    if not args.no_extra and rank == 0:
        extra = extra_rows(api, L, dev, peak, peak_kind, set(args.rows.split(",")), args.no_cpu)

    line = {
        "metric": METRIC,
        "value": value, "unit": "cells/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": step_config(n, world),
        "phases_ms": {"receivers": statistics.mean(recv_ms), "accumulate": statistics.mean(acc_ms),
                      "mass_balance": statistics.mean(mb_ms)},
        "mass_balance_path": "area term from the sums the accumulation forms where it writes the "
                             "areas, plus the global cells' sinks (FR_SINK_SUMS_IN_WORKSPACE); "
                             "equal bit for bit to the full pass over the stored areas, checked "
                             "before the timed steps",
        "roofline": {"bound": "hbm", "kernel": "fr_accumulate D8 areas (k_local_d8 + global phase)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": traffic, "traffic_note": traffic_note,
                     "algorithmic_bytes_per_cell": 9},
        "step_roofline": {"algorithmic_bytes_per_cell": 12,
                          "achieved": step_bytes / (total_ms / K * 1e-3) / 1e9,
                          "frac": step_bytes / (total_ms / K * 1e-3) / 1e9 / peak},
        "e2e": e2e,
        "gpu_launches": launches * K if launches is not None else None,
        "gpu_launches_per_step": launches,
        "clocks": clk,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if crop:
        line["parity_on_crop"] = crop
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def d8_crop_check(api, zc):
    """The oracle on a crop of the headline DEM, timed on the host cores, and
    the GPU's codes and areas on the same crop compared with it."""
    import torch
    try:
        import oracle
        oracle.build()
        side = zc.shape[0]
        t0 = time.perf_counter()
        d, w, a, _ = oracle.route_d8(zc, DX, None)
        oracle.mass_balance(w, None, dir_=d)
        dt = time.perf_counter() - t0
        cpu = {"value": side * side / dt, "unit": "cells/s", "cores": 1, "kind": "oracle",
               "sample": "%dx%d crop of the headline DEM, one pass (receivers, unit-rain areas, "
                         "mass balance; sequential high-to-low, FP64/uint64), %.1f s" % (side, side, dt),
               "host_cores": os.cpu_count()}
        out = api.route_d8(torch.from_numpy(zc).cuda(), DX, None, 0, want_w=False, want_area=True,
                           want_dir=True)
        gd = out["dir"].cpu().numpy()
        ga = out["area"].cpu().numpy().astype(np.uint64)
        crop = {"cells": side * side, "code_mismatches": int((gd != d).sum()),
                "area_mismatches": int((ga != a).sum()), "max_rel_err": 0.0 if (ga == a).all() else
                float(np.max(np.abs(ga.astype(np.float64) - a) / a))}
        return cpu, crop
    except Exception as e:  # pragma: no cover
        return {"value": None, "unit": "cells/s", "cores": 1, "kind": "oracle",
                "sample": "failed: %s" % e}, None


def extra_rows(api, L, dev, peak, peak_kind, want, no_cpu):
    """The other workloads, each timed with CUDA events."""
    import torch
    rows = {}
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def timed(fn, reps=5):
        for _ in range(2):
            flush.zero_()
            fn()
        ms = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.mean(ms)

    def run(name, fn):
        if name in want:
            rows[name] = fn()
            torch.cuda.empty_cache()

    run("slope_split", lambda: slope_split_row(api, L, dev, peak, peak_kind, timed, no_cpu))
    run("d8_4096", lambda: d8_4096_row(api, L, dev, peak, timed))
    run("long_rivers", lambda: long_rivers_row(api, L, dev, peak, timed))
    run("batched", lambda: batch_rows(api, L, dev))
    run("adjoint", lambda: adjoint_row(api, dev, peak, timed))
    run("richardson", lambda: richardson_row(api, dev, timed))
    run("fill", lambda: fill_row(api, peak, timed))
    return rows


def slope_split_row(api, L, dev, peak, peak_kind, timed, no_cpu):
    """Slope-split route (receivers with fractions + accumulation, unit rain)
    on an 8192^2 DEM (beta 2.2, no tilt): device time, roofline at 8 bytes per
    cell (z in, w out), e2e from pinned host memory, the oracle on a crop, and
    the largest relative error of w against the FP64 oracle on that crop."""
    import ctypes

    import torch
    from paper_2606_12800_gb300 import _lib, inputs
    P = ctypes.c_void_p
    n = MFD_SIDE
    cells = n * n
    zt = inputs.fractal_dem_torch(n, n, beta=MFD_BETA, tilt=0.0, seed=MFD_SEED, dx=DX, device="cuda")
    w = torch.empty((n, n), dtype=torch.float32, device=dev)
    ws = api.workspace(n, n, dev, mfd=True)

    def route():
        _lib.check(L.fr_route_mfd(P(zt.data_ptr()), n, n, DX, MFD_P, 0, None, P(w.data_ptr()), None,
                                  None, P(ws.data_ptr()), ws.numel(), api._stream()), "fr_route_mfd")
    ms = timed(route, reps=10)
    status = api.get_status(dev)
    launches = count_launches(route)
    gbs = cells * 8 / (ms * 1e-3) / 1e9
    row = {"value": cells / (ms * 1e-3), "unit": "cells/s", "ms_per_step": ms, "status": status,
           "workload": "slope-split (MFD p=1.1) route, %dx%d fractal DEM beta=2.2 no tilt, unit "
                       "rain, two-float fp32 w" % (n, n),
           "roofline": {"bound": "hbm", "kernel": "fr_route_mfd (receivers + fractions + "
                                                  "k_local_halo<FwdMfd> + global phase)",
                        "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                        "peak_kind": peak_kind, "algorithmic_bytes_per_cell": 8},
           "gpu_launches_per_step": launches}
    tr, note = profile_traffic("k_local_halo_mfd", cells)
    row["roofline"]["traffic"], row["roofline"]["traffic_note"] = tr, note
    zc = np.ascontiguousarray(zt[:MFD_CROP, :MFD_CROP].cpu().numpy())
    z_host = zt.cpu().pin_memory()
    del zt, w
    torch.cuda.empty_cache()
    e2e_ms = []
    for i in range(4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = api.route_mfd(z_host, DX, MFD_P, None, 0)
        torch.cuda.synchronize()
        if i >= 1:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        del out
    row["e2e"] = {"value": cells / (statistics.median(e2e_ms) * 1e-3), "unit": "cells/s",
                  "h2d_bytes_per_step": cells * 4, "d2h_bytes_per_step": cells * 4,
                  "ms_per_step": statistics.median(e2e_ms),
                  "path": "api.route_mfd (fr_route_mfd) from pinned host DEM; w to host"}
    del z_host
    if not no_cpu:
        try:
            import oracle
            oracle.build()
            t0 = time.perf_counter()
            _, _, w64, _ = oracle.route_mfd(zc, DX, MFD_P, None)
            dt = time.perf_counter() - t0
            row["cpu_baseline"] = {
                "value": MFD_CROP * MFD_CROP / dt, "unit": "cells/s", "cores": 1, "kind": "oracle",
                "sample": "%dx%d crop of the DEM, one pass (receivers, FP64 fractions, "
                          "sequential high-to-low water), %.1f s" % (MFD_CROP, MFD_CROP, dt)}
            g = api.route_mfd(torch.from_numpy(zc).cuda(), DX, MFD_P, None, 0, want_lo=True)
            wg = g["w"].double().cpu().numpy() + g["w_lo"].double().cpu().numpy()
            w1 = g["w"].double().cpu().numpy()
            row["error_vs_oracle"] = {
                "sample": "%dx%d crop of the same DEM" % (MFD_CROP, MFD_CROP),
                "max_rel_err_w": float(np.max(np.abs(w1 - w64) / w64)),
                "max_rel_err_w_plus_lo": float(np.max(np.abs(wg - w64) / w64)),
                "bar": 1e-6}
        except Exception as e:  # pragma: no cover
            row["cpu_baseline"] = {"value": None, "unit": "cells/s", "cores": 1, "kind": "oracle",
                                   "sample": "failed: %s" % e}
    return row


def d8_4096_row(api, L, dev, peak, timed):
    """The D8 step on a 4096^2 DEM (beta 2, tilt 0.01) with rain U[0,1):
    receivers, two-float water and uint64 areas, mass balance."""
    import ctypes

    import torch
    from paper_2606_12800_gb300 import _lib, inputs
    P = ctypes.c_void_p
    n = 4096
    z = torch.from_numpy(inputs.fractal_dem(n, n, beta=2.0, tilt=0.01, seed=SEED, dx=DX)).to(dev)
    rain = torch.from_numpy(inputs.rain_field(n, n, SEED)).to(dev)
    d = torch.empty((n, n), dtype=torch.uint8, device=dev)
    w = torch.empty((n, n), dtype=torch.float32, device=dev)
    area = torch.empty((n, n), dtype=torch.int64, device=dev)
    mb = torch.empty(3, dtype=torch.float64, device=dev)
    ws = api.workspace(n, n, dev)
    R = api.routing_d8(d)
    wsp, wsn = P(ws.data_ptr()), ws.numel()
    ph = {}

    def step():
        _lib.check(L.fr_receivers_d8(P(z.data_ptr()), n, n, DX, 0, P(d.data_ptr()), None,
                                     api._stream()), "fr_receivers_d8")
        _lib.check(L.fr_accumulate(ctypes.byref(R), P(rain.data_ptr()), P(w.data_ptr()), None,
                                   P(area.data_ptr()), wsp, wsn, api._stream()), "fr_accumulate")
        _lib.check(L.fr_mass_balance(ctypes.byref(R), P(rain.data_ptr()), P(w.data_ptr()), None,
                                     P(area.data_ptr()), P(mb.data_ptr()), wsp, wsn, api._stream()),
                   "fr_mass_balance")

    def acc():
        _lib.check(L.fr_accumulate(ctypes.byref(R), P(rain.data_ptr()), P(w.data_ptr()), None,
                                   P(area.data_ptr()), wsp, wsn, api._stream()), "fr_accumulate")
    ms = timed(step, reps=10)
    ph["accumulate"] = timed(acc, reps=10)
    st = api.get_status(dev)
    return {"value": n * n / (ms * 1e-3), "unit": "cells/s", "ms_per_step": ms, "status": st,
            "accumulate_ms": ph["accumulate"],
            "accumulate_frac": n * n * 17 / (ph["accumulate"] * 1e-3) / 1e9 / peak,
            "workload": "D8 4096^2 beta=2 tilt=0.01, rain U[0,1): receivers + two-float w + uint64 "
                        "areas + mass balance (accumulation at 17 B/cell: dir, rain in; w, area out)"}


def long_rivers_row(api, L, dev, peak, timed):
    """D8 unit-rain areas on DEMs with long rivers: the D8 DEMs (4096^2 beta 2
    tilt 0.01; 32768^2 beta 2 tilt 0.005) after depression filling, and a
    32768^2 plane (every row one chain of 32768 cells); the unfilled headline
    DEM for contrast.  Each input is accumulated with both global phases (cell
    walkers, tile skeleton) and with the automatic choice between them (the
    skeleton when the local phase leaves at least 1/512 of the cells); the
    areas of the three runs must agree bit for bit.  Accumulation against the
    roofline at 9 bytes per cell."""
    import ctypes

    import torch
    from paper_2606_12800_gb300 import _lib, inputs
    P = ctypes.c_void_p
    out = {}

    def one(name, z):
        n_y, n_x = z.shape
        d = api.receivers_d8(z, DX)
        ws = api.workspace(n_x, n_y, dev)
        ref = None
        row = {}
        for label, fl in (("auto", 0), ("walkers", _lib.FR_GLOBAL_WALKERS),
                          ("skeleton", _lib.FR_GLOBAL_SKELETON)):
            area = torch.empty((n_y, n_x), dtype=torch.int64, device=dev)
            R = api.routing_d8(d, flags=fl)

            def acc():
                _lib.check(L.fr_accumulate(ctypes.byref(R), None, None, None, P(area.data_ptr()),
                                           P(ws.data_ptr()), ws.numel(), api._stream()), "fr_accumulate")
            ms = timed(acc, reps=3)
            st = api.get_status(dev)
            if ref is None:
                ref = area
                sinks = int(area.view(-1)[d.view(-1) == 0xFF].sum().item())
                g = ws[:128].cpu().numpy().view("u8")
                share = int(g[4]) / (n_x * n_y)
                row.update({"sink_area_sum_equals_cells": sinks == n_x * n_y, "global_cells_frac": share,
                            "chosen": "skeleton" if share >= 1.0 / 512 else "walkers",
                            "max_area": int(area.max().item())})
                row.update({"accumulate_ms": ms, "cells_per_s": n_x * n_y / (ms * 1e-3),
                            "frac": n_x * n_y * 9 / (ms * 1e-3) / 1e9 / peak, "status": st})
            else:
                row[label + "_ms"] = ms
                row[label + "_status"] = st
                row[label + "_areas_equal"] = bool(torch.equal(area, ref))
                del area
        del d, ref
        out[name] = row

    z = inputs.fractal_dem_torch(4096, 4096, beta=2.0, tilt=0.01, seed=SEED, dx=DX, device="cuda")
    F, _ = api.fill(z)
    one("filled_4096", F)
    del z, F
    z = torch.from_numpy(np.ascontiguousarray(inputs.planar_dem(N_SIDE, N_SIDE, tilt=0.005, dx=DX))).to(dev)
    one("planar_32768", z)
    del z
    torch.cuda.empty_cache()
    z = inputs.fractal_dem_torch(N_SIDE, N_SIDE, beta=D8_BETA, tilt=D8_TILT, seed=D8_SEED, dx=DX,
                                 device="cuda")
    one("rough_32768", z)
    t0 = time.perf_counter()
    F, sweeps = api.fill(z)
    torch.cuda.synchronize()
    fill_s = time.perf_counter() - t0
    del z
    torch.cuda.empty_cache()
    one("filled_32768", F)
    out["filled_32768"]["fill_s"] = fill_s
    out["filled_32768"]["fill_sweeps"] = sweeps
    del F
    return out


def adjoint_row(api, dev, peak, timed):
    """Slope-split on 16384^2 (beta 2.2, no tilt, unit rain): the adjoint of
    L = sum over sinks of w^2 giving dL/drain and dL/dz, timed alone (the
    forward route runs once, untimed, before it)."""
    from paper_2606_12800_gb300 import inputs
    n = 16384
    zt = inputs.fractal_dem_torch(n, n, beta=2.2, tilt=0.0, seed=SEED + 4, device="cuda")
    m = api.receivers_mfd(zt, DX, 1.1)
    R = api.routing_mfd(m, zt, DX, 1.1)
    fwd = api.accumulate(R, None, want_w=True, want_lo=True, device=dev)

    def adj():
        return api.adjoint(R, fwd["w"], fwd["w_lo"], want_dz=True)
    ms = timed(adj, reps=3)
    status = api.get_status(dev)
    # the same adjoint reading the fractions the forward left in a workspace
    # of its own (FR_WEIGHTS_IN_WORKSPACE) instead of recomputing them
    import torch
    from paper_2606_12800_gb300 import _lib
    ws = torch.empty(api.workspace_size(n, n, mfd=True), dtype=torch.uint8, device=dev)
    fwd = api.accumulate(R, None, want_w=True, want_lo=True, device=dev, ws=ws)
    Rk = api.routing_mfd(m, zt, DX, 1.1, _lib.FR_WEIGHTS_IN_WORKSPACE)

    def adj_kept():
        return api.adjoint(Rk, fwd["w"], fwd["w_lo"], want_dz=True, ws=ws)
    ms_kept = timed(adj_kept, reps=3)
    status |= api.get_status(dev, ws=ws)
    del zt, m, fwd, ws
    # algorithmic bytes: z 4 + w 4 in, dL/dr 4 + dL/dz 4 out
    return {"ms": ms, "kept_weights_ms": ms_kept, "value": n * n / (ms * 1e-3), "unit": "cells/s",
            "status": status,
            "workload": "MFD p=1.1 adjoint alone (dL/drain and dL/dz) of L = sum over sinks of "
                        "w^2, %dx%d fractal DEM beta=2.2" % (n, n),
            "hbm_frac": (n * n * 16) / (ms * 1e-3) / 1e9 / peak, "algorithmic_bytes_per_cell": 16}


def fill_row(api, peak, timed):
    """Depression filling (fr_fill) of the 4096^2 D8 DEM (beta 2, tilt 0.01)
    and of the slope-split DEM (8192^2, beta 2.2, no tilt: wide closed
    basins): sweeps to the exact fill and device time, against the roofline at
    8 algorithmic bytes per cell (z in, F out)."""
    from paper_2606_12800_gb300 import inputs
    out = {}
    for name, n, beta, tilt, seed in (("d8_4096", 4096, 2.0, 0.01, SEED),
                                      ("mfd_8192", MFD_SIDE, MFD_BETA, 0.0, MFD_SEED)):
        z = inputs.fractal_dem_torch(n, n, beta=beta, tilt=tilt, seed=seed, device="cuda")
        res = {}

        def run():
            res["F"], res["sweeps"] = api.fill(z)
        ms = timed(run, reps=3)
        gbs = n * n * 8 / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "sweeps": res["sweeps"], "cells_per_s": n * n / (ms * 1e-3),
                     "raised_frac": float((res["F"] != z).float().mean().item()),
                     "hbm_frac": gbs / peak}
        del z, res
    return out


def richardson_row(api, dev, timed):
    """The paper's Richardson I+X iteration on 64x32 tiles (one GPU) against
    the exact solve, on the 4096^2 D8 DEM with rain and the slope-split DEM
    (8192^2, unit rain): iterations and device time."""
    import torch
    from paper_2606_12800_gb300 import inputs
    out = {}
    n = 4096
    z = torch.from_numpy(inputs.fractal_dem(n, n, beta=2.0, tilt=0.01, seed=SEED, dx=DX)).to(dev)
    rain = torch.from_numpy(inputs.rain_field(n, n, SEED)).to(dev)
    R = api.routing_d8(api.receivers_d8(z, DX))
    it = {}

    def rich_d8(order):
        it[order] = api.accumulate_richardson(R, rain, order=order)[1]
    ms_r1 = timed(lambda: rich_d8(1), reps=3)
    ms_r2 = timed(lambda: rich_d8(2), reps=3)
    ms_x = timed(lambda: api.accumulate(R, rain, want_w=True), reps=3)
    out["d8_4096"] = {"i_plus_x": {"iterations": it[1], "ms": ms_r1},
                      "i_minus_x_i_plus_x": {"iterations": it[2], "ms": ms_r2},
                      "exact_ms": ms_x}
    del z, rain, R
    n = MFD_SIDE
    zt = inputs.fractal_dem_torch(n, n, beta=MFD_BETA, tilt=0.0, seed=MFD_SEED, device="cuda")
    m = api.receivers_mfd(zt, DX, MFD_P)
    Rm = api.routing_mfd(m, zt, DX, MFD_P)

    def rich_mfd(order):
        it[order] = api.accumulate_richardson(Rm, None, order=order)[1]
    ms_r1 = timed(lambda: rich_mfd(1), reps=2)
    ms_r2 = timed(lambda: rich_mfd(2), reps=2)
    ms_x = timed(lambda: api.accumulate(Rm, None, want_w=True, device=dev), reps=2)
    out["mfd_8192"] = {"i_plus_x": {"iterations": it[1], "ms": ms_r1},
                       "i_minus_x_i_plus_x": {"iterations": it[2], "ms": ms_r2},
                       "exact_ms": ms_x}
    return out


def batch_rows(api, L, dev):
    """512 independent tiles (sides log-uniform in [64, 2048], beta in [1.8, 2.4],
    rain U[0,1)): one fr_route_batch call replayed from a CUDA graph, against a
    loop of per-tile fr_route_d8 / fr_route_mfd calls, for D8 and slope-split."""
    import ctypes

    import torch
    from paper_2606_12800_gb300 import _lib, inputs
    P = ctypes.c_void_p
    specs = inputs.batch_specs(512, seed=SEED)
    dems = [inputs.fractal_dem_torch(t.n_y, t.n_x, beta=t.beta, tilt=0.0, seed=t.seed, device="cuda")
            for t in specs]
    rains = [inputs.rain_field_torch(t.n_y, t.n_x, t.seed, device="cuda") for t in specs]
    cells = sum(t.n_x * t.n_y for t in specs)
    stream = torch.cuda.current_stream()
    out = {"tiles": len(specs), "cells": cells,
           "workload": "512 tiles, sides log-uniform in [64, 2048], beta U[1.8, 2.4], rain U[0,1), w out"}

    def ev_time(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    for kind in ("d8", "mfd"):
        k = _lib.FR_ROUTING_D8 if kind == "d8" else _lib.FR_ROUTING_MFD
        route = [torch.empty((t.n_y, t.n_x), dtype=torch.uint8, device=dev) for t in specs]
        w = [torch.empty((t.n_y, t.n_x), dtype=torch.float32, device=dev) for t in specs]
        arr = (_lib.fr_tile * len(specs))()
        for i, t in enumerate(specs):
            a = arr[i]
            a.dem, a.rain, a.w_out, a.w_lo_out, a.area_out = (dems[i].data_ptr(), rains[i].data_ptr(),
                                                             w[i].data_ptr(), None, None)
            a.route_out, a.nx, a.ny, a.dx = route[i].data_ptr(), t.n_x, t.n_y, DX
        tiles_dev = torch.frombuffer(bytearray(bytes(memoryview(arr).cast("B"))),
                                     dtype=torch.uint8).to(dev)
        need = int(L.fr_batch_workspace_size(arr, len(specs), k, 0))
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
        wsp = P(ws.data_ptr())

        def batched():
            _lib.check(L.fr_route_batch(arr, P(tiles_dev.data_ptr()), len(specs), k, 1.1, 0, wsp, need,
                                        api._stream()), "fr_route_batch")
        _lib.check(L.fr_batch_autotune(arr, P(tiles_dev.data_ptr()), len(specs), k, 1.1, 0, wsp, need,
                                       api._stream()), "fr_batch_autotune")
        torch.cuda.synchronize()
        row = {}
        row["batched_ms"] = ev_time(batched, 5)
        try:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                batched()
            row["batched_graph_ms"] = ev_time(g.replay, 5)
            del g
        except Exception as e:  # pragma: no cover
            row["batched_graph_ms"] = None
            row["graph_error"] = str(e)[:200]
        st = int(L.fr_get_status(wsp, need, api._stream()))
        row["status"] = st
        tws = api.workspace(2048, 2048, dev, mfd=(kind == "mfd"))
        twsp, twsn = P(tws.data_ptr()), tws.numel()

        def per_tile():
            s = api._stream()
            for i, t in enumerate(specs):
                if kind == "d8":
                    L.fr_route_d8(P(dems[i].data_ptr()), t.n_x, t.n_y, DX, 0, P(rains[i].data_ptr()),
                                  P(w[i].data_ptr()), None, None, P(route[i].data_ptr()), twsp, twsn, s)
                else:
                    L.fr_route_mfd(P(dems[i].data_ptr()), t.n_x, t.n_y, DX, 1.1, 0, P(rains[i].data_ptr()),
                                   P(w[i].data_ptr()), None, P(route[i].data_ptr()), twsp, twsn, s)
        row["per_tile_ms"] = ev_time(per_tile, 3)
        best = row["batched_graph_ms"] or row["batched_ms"]
        row["cells_per_s"] = cells / (best * 1e-3)
        row["per_tile_cells_per_s"] = cells / (row["per_tile_ms"] * 1e-3)
        row["speedup_vs_per_tile"] = row["per_tile_ms"] / best
        out[kind] = row
        del route, w, ws, tiles_dev
    return out


if __name__ == "__main__":
    main()
