#!/usr/bin/env python3
"""Benchmark: cells routed per second on one GB300 (D8 and slope-split).

Workload (one step = one pass of the hot path over one synthetic DEM):
  D8 on a 4096 x 4096 float32 fractal DEM (beta 2, tilt 0.01, jitter 1e-4 m,
  dx 30 m) with rain U[0,1): receivers, exact accumulation of the rain
  (two-float fp32) and of unit rain (uint64 drainage areas), and the
  mass-balance check.  Extra keys report the slope-split (MFD, p = 1.1) route
  on an 8192 x 8192 DEM (beta 2.2, no tilt), the batched route and the
  adjoint, each timed the same way.

Timing: W untimed warm-up steps, then exactly K timed steps, each bracketed by
CUDA events on the launching stream; L2 is flushed (a 512 MiB write) between
steps, outside the events; barrier + synchronize around the timed loop, max
over ranks.  With --gpus N > 1 (torchrun) every rank routes its own replica
(the path has no exchange step) and the value is the sum over ranks.

--impl reference times the CPU oracle (the paper's sequential high-to-low
algorithm, FP64/uint64, single thread) on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 4096
MFD_SIDE = 8192
DX = 30.0
SEED = 1
# DRAM bytes (read + write) of one k_local_d8 launch on the 4096^2 workload, from
# an ncu capture of this kernel as it stands (profiles/k_local_d8_4096.md);
# None whenever the kernel changes until it is captured again.
TRAFFIC_K_LOCAL_D8 = 88.336640e6 + 147.438336e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extra", action="store_true", help="skip the MFD/batch/adjoint rows")
    ap.add_argument("--rows", default="slope_split,batched,adjoint,d8_32768,richardson,fill",
                    help="comma-separated extra rows to run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


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


# ----------------------------------------------------------------- reference
METRIC = "cells routed/sec at 1 GB300 (D8 & slope-split)"


def step_config(n, world, cells):
    """The `config` of the step's JSON line (the same for both arms)."""
    return {"workload": "D8 %dx%d fractal DEM (beta=2, tilt=0.01, jitter 1e-4 m, dx=30 m), "
                        "rain U[0,1): receivers + two-float rain accumulation + uint64 "
                        "unit-rain areas + mass balance" % (n, n),
            "global_batch": world, "cells_per_step": cells,
            "l2": "flushed between steps (512 MiB write)", "parallelism": "replicas"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2606_12800_gb300 import inputs
    oracle.build()
    side = 1024  # bounded sample: a 1024^2 DEM of the same recipe per step
    z = inputs.fractal_dem(side, side, beta=2.0, tilt=0.01, seed=SEED, dx=DX)
    rain = inputs.rain_field(side, side, SEED)
    for _ in range(args.warmup):
        oracle.route_d8(z, DX, rain)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        d, w, a, order = oracle.route_d8(z, DX, rain)
        _, a = oracle.accumulate_d8(d, order, None, want_w=False)
        oracle.mass_balance(w, rain, dir_=d)
    dt = time.perf_counter() - t0
    value = args.steps * side * side / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "cells/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": step_config(N_SIDE, args.gpus, N_SIDE * N_SIDE),
        "cpu_baseline": {"value": value, "unit": "cells/s", "cores": 1, "kind": "oracle",
                         "sample": "%dx%d crop of the workload's recipe per step (receivers, "
                                   "water, areas, mass balance; sequential high-to-low, "
                                   "FP64/uint64), scaled to cells/s" % (side, side)},
        "e2e": {"value": value, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------- ours
def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    from paper_2606_12800_gb300 import _lib, api, inputs
    rank, world = dist_init(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    L = _lib.load()
    stream = torch.cuda.current_stream()
    sp = lambda: api._stream()  # noqa: E731

    # inputs resident in HBM
    n = N_SIDE
    z_np = inputs.fractal_dem(n, n, beta=2.0, tilt=0.01, seed=SEED, dx=DX)
    r_np = inputs.rain_field(n, n, SEED)
    z = torch.from_numpy(z_np).to(dev)
    rain = torch.from_numpy(r_np).to(dev)
    dir_ = torch.empty((n, n), dtype=torch.uint8, device=dev)
    w = torch.empty((n, n), dtype=torch.float32, device=dev)
    area = torch.empty((n, n), dtype=torch.int64, device=dev)
    mb = torch.empty(3, dtype=torch.float64, device=dev)
    ws = api.workspace(n, n, dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    R = api.routing_d8(dir_)
    import ctypes
    P = ctypes.c_void_p
    wsp, wsn = P(ws.data_ptr()), ws.numel()

    def step(evs=None):
        if evs:
            evs[0].record(stream)
        _lib.check(L.fr_receivers_d8(P(z.data_ptr()), n, n, DX, 0, P(dir_.data_ptr()), None, sp()),
                   "fr_receivers_d8")
        if evs:
            evs[1].record(stream)
        _lib.check(L.fr_accumulate(ctypes.byref(R), P(rain.data_ptr()), P(w.data_ptr()), None,
                                   P(area.data_ptr()), wsp, wsn, sp()), "fr_accumulate")
        if evs:
            evs[2].record(stream)
        _lib.check(L.fr_mass_balance(ctypes.byref(R), P(rain.data_ptr()), P(w.data_ptr()), None,
                                     P(area.data_ptr()), P(mb.data_ptr()), wsp, wsn, sp()),
                   "fr_mass_balance")
        if evs:
            evs[3].record(stream)

    for _ in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    status = api.get_status(dev)
    mbv = mb.cpu().numpy()
    assert status == 0, "device status %d" % status
    assert mbv[2] == n * n and abs(mbv[0] - mbv[1]) <= 1e-9 * mbv[1], mbv

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
            for _ in range(50):
                flush.zero_()
                step()
            torch.cuda.synchronize()
        clk2 = clocks.stop()
        if clk2:
            clk2["window"] = "timed region + 1.5 s soak of the same step"
            clk = clk2

    cells = n * n
    value = job_value(world, K, cells, total_ms)
    peak, peak_kind = peaks()
    acc_bytes = cells * (1 + 4 + 4 + 8)     # dir + rain in, w + area out
    acc_avg = statistics.mean(acc_ms) * 1e-3
    achieved = acc_bytes / acc_avg / 1e9
    step_bytes = cells * (4 + 4 + 4 + 8)     # algorithmic: z + rain in, w + area out

    # end to end through the public API: pinned host buffers, copies timed
    zh = torch.from_numpy(z_np).pin_memory()
    rh = torch.from_numpy(r_np).pin_memory()
    e2e_ms = []
    for i in range(max(3, min(K, 10)) + 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = api.route_d8(zh, DX, rh, 0, want_w=True, want_area=True)
        torch.cuda.synchronize()
        if i >= 2:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        del out
    e2e = {"value": cells / (statistics.median(e2e_ms) * 1e-3), "unit": "cells/s",
           "h2d_bytes_per_step": cells * 8, "d2h_bytes_per_step": cells * 12,
           "ms_per_step": statistics.median(e2e_ms)}

    extra = {}
    if not args.no_extra and rank == 0:
        extra = extra_rows(api, L, dev, peak, set(args.rows.split(",")))

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(z_np, r_np)

    line = {
        "metric": METRIC,
        "value": value, "unit": "cells/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": step_config(n, world, cells),
        "phases_ms": {"receivers": statistics.mean(recv_ms), "accumulate": statistics.mean(acc_ms),
                      "mass_balance": statistics.mean(mb_ms)},
        "roofline": {"bound": "hbm", "kernel": "fr_accumulate D8 (k_local_d8 + k_global)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": TRAFFIC_K_LOCAL_D8,
                     "traffic_note": "ncu dram read+write of k_local_d8, one launch at this size",
                     "algorithmic_bytes_per_cell": 17,
                     "step_frac": step_bytes / (total_ms / K * 1e-3) / 1e9 / peak},
        "e2e": e2e,
        "gpu_launches": K * 5,
        "clocks": clk,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def cpu_baseline(z_np, r_np):
    """The oracle as it stands on the host cores, on a 2048^2 crop."""
    try:
        import oracle
        oracle.build()
        side = 2048
        z = np.ascontiguousarray(z_np[:side, :side])
        r = np.ascontiguousarray(r_np[:side, :side])
        t0 = time.perf_counter()
        d, w, a, order = oracle.route_d8(z, DX, r)
        oracle.accumulate_d8(d, order, None, want_w=False)
        oracle.mass_balance(w, r, dir_=d)
        dt = time.perf_counter() - t0
        return {"value": side * side / dt, "unit": "cells/s", "cores": 1, "kind": "oracle",
                "sample": "%dx%d crop of the workload DEM, one pass (sequential high-to-low, "
                          "FP64/uint64), %.1f s" % (side, side, dt),
                "host_cores": os.cpu_count()}
    except Exception as e:  # pragma: no cover
        return {"value": None, "unit": "cells/s", "cores": 1, "kind": "oracle",
                "sample": "failed: %s" % e}


def extra_rows(api, L, dev, peak, want):
    """The other workloads, each timed with CUDA events: slope-split route
    (8192^2), the batched route, the MFD adjoint (16384^2) and D8 on 32768^2."""
    import torch
    from paper_2606_12800_gb300 import inputs
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

    if "slope_split" in want:
        n = MFD_SIDE
        zt = inputs.fractal_dem_torch(n, n, beta=2.2, tilt=0.0, seed=SEED + 2, device="cuda")

        def mfd():
            m = api.receivers_mfd(zt, DX, 1.1)
            Rm = api.routing_mfd(m, zt, DX, 1.1)
            return api.accumulate(Rm, None, want_w=True, device=dev)
        ms = timed(mfd)
        rows["slope_split"] = {"value": n * n / (ms * 1e-3), "unit": "cells/s", "ms": ms,
                               "workload": "MFD p=1.1, %dx%d fractal DEM beta=2.2 no tilt, unit rain" % (n, n),
                               "hbm_frac": (n * n * 8) / (ms * 1e-3) / 1e9 / peak}
        del zt
        torch.cuda.empty_cache()
    if "batched" in want:
        rows["batched"] = batch_rows(api, L, dev)
        torch.cuda.empty_cache()
    if "adjoint" in want:
        rows["adjoint"] = adjoint_row(api, dev, peak, timed)
        torch.cuda.empty_cache()
    if "d8_32768" in want:
        rows["d8_32768"] = d8_large_row(api, L, dev, peak, timed)
        torch.cuda.empty_cache()
    if "richardson" in want:
        rows["richardson"] = richardson_row(api, dev, timed)
    if "fill" in want:
        rows["fill"] = fill_row(api, peak, timed)
        torch.cuda.empty_cache()
    return rows


def adjoint_row(api, dev, peak, timed):
    """Slope-split on 16384^2 (beta 2.2, no tilt, unit rain): forward, then the
    adjoint of L = sum over sinks of w^2 giving dL/drain and dL/dz."""
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
    del zt, m, fwd
    # algorithmic bytes: z 4 + w 8 (two words) in, dL/dr 4 + dL/dz 4 out
    return {"ms": ms, "value": n * n / (ms * 1e-3), "unit": "cells/s", "status": status,
            "workload": "MFD p=1.1 adjoint of L = sum over sinks of w^2, %dx%d fractal DEM "
                        "beta=2.2, dL/drain and dL/dz" % (n, n),
            "hbm_frac": (n * n * 20) / (ms * 1e-3) / 1e9 / peak}


def d8_large_row(api, L, dev, peak, timed):
    """D8 on 32768^2 (beta 2, tilt 0.005, unit rain): receivers + exact uint64
    areas; the accumulation alone against the roofline (dir 1 B in, area 8 B
    out per cell)."""
    import ctypes
    import torch
    from paper_2606_12800_gb300 import _lib, inputs
    n = 32768
    P = ctypes.c_void_p
    zt = inputs.fractal_dem_torch(n, n, beta=2.0, tilt=0.005, seed=SEED + 5, device="cuda")
    d = torch.empty((n, n), dtype=torch.uint8, device=dev)
    area = torch.empty((n, n), dtype=torch.int64, device=dev)
    ws = api.workspace(n, n, dev)
    R = api.routing_d8(d)

    def recv():
        _lib.check(L.fr_receivers_d8(P(zt.data_ptr()), n, n, DX, 0, P(d.data_ptr()), None,
                                     api._stream()), "fr_receivers_d8")

    def acc():
        _lib.check(L.fr_accumulate(ctypes.byref(R), None, None, None, P(area.data_ptr()),
                                   P(ws.data_ptr()), ws.numel(), api._stream()), "fr_accumulate")
    recv()
    ms_recv = timed(recv, reps=3)
    ms_acc = timed(acc, reps=3)
    status = api.get_status(dev)
    total = int(area.view(-1)[d.view(-1) == 0xFF].sum().item())
    cells = n * n
    del zt, d, area
    return {"ms_receivers": ms_recv, "ms_accumulate": ms_acc,
            "value": cells / ((ms_recv + ms_acc) * 1e-3), "unit": "cells/s", "status": status,
            "sink_area_sum_equals_cells": total == cells,
            "workload": "D8 %dx%d fractal DEM beta=2 tilt=0.005, unit rain, uint64 areas" % (n, n),
            "accumulate_roofline": {"bound": "hbm", "algorithmic_bytes_per_cell": 9,
                                    "achieved_gbs": cells * 9 / (ms_acc * 1e-3) / 1e9, "peak": peak,
                                    "frac": cells * 9 / (ms_acc * 1e-3) / 1e9 / peak}}


def fill_row(api, peak, timed):
    """Depression filling (fr_fill) of the D8 step's DEM (4096^2, beta 2, tilt
    0.01) and of the slope-split DEM (8192^2, beta 2.2, no tilt: wide closed
    basins): sweeps to the exact fill and device time, against the roofline at
    8 algorithmic bytes per cell (z in, F out)."""
    from paper_2606_12800_gb300 import inputs
    out = {}
    for name, n, beta, tilt, seed in (("d8_4096", N_SIDE, 2.0, 0.01, SEED),
                                      ("mfd_8192", MFD_SIDE, 2.2, 0.0, SEED + 2)):
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
    the two-launch exact solve, on the D8 step's DEM (4096^2, rain) and the
    slope-split DEM (8192^2, unit rain): iterations and device time."""
    import torch
    from paper_2606_12800_gb300 import inputs
    out = {}
    n = N_SIDE
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
                      "exact_two_phase_ms": ms_x}
    del z, rain, R
    n = MFD_SIDE
    zt = inputs.fractal_dem_torch(n, n, beta=2.2, tilt=0.0, seed=SEED + 2, device="cuda")
    m = api.receivers_mfd(zt, DX, 1.1)
    Rm = api.routing_mfd(m, zt, DX, 1.1)

    def rich_mfd(order):
        it[order] = api.accumulate_richardson(Rm, None, order=order)[1]
    ms_r1 = timed(lambda: rich_mfd(1), reps=2)
    ms_r2 = timed(lambda: rich_mfd(2), reps=2)
    ms_x = timed(lambda: api.accumulate(Rm, None, want_w=True, device=dev), reps=2)
    out["mfd_8192"] = {"i_plus_x": {"iterations": it[1], "ms": ms_r1},
                       "i_minus_x_i_plus_x": {"iterations": it[2], "ms": ms_r2},
                       "exact_two_phase_ms": ms_x}
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
