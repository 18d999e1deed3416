"""Named workloads run through the public API, for profiling one kernel at a
chosen size (``ncu -k ...  python -m paper_2606_12800_gb300.cases mfd --n 4096``).

Cases (all on seeded synthetic fractal DEMs, inputs resident on the device):
  d8        receivers + D8 accumulation with rain U[0,1) (two-float w, uint64 areas)
  d8_area   receivers + D8 unit-rain areas only
  d8_step   receivers + D8 unit-rain areas + the mass balance as a full pass over
            the stored areas (the benchmark step takes the mass balance's area term
            from the accumulation's sink sums instead)
  mfd       slope-split route (p = 1.1), unit rain
  adjoint   slope-split route, then the adjoint of L = sum over sinks of w^2
            (dL/drain and dL/dz)
  fill      depression filling of the D8 DEM (beta 2, tilt 0.01)
  d8_plane  D8 unit-rain areas on a plane falling towards +x (every row one
            river of n cells): the global cells go to the tile-skeleton solve
  d8_filled D8 unit-rain areas on the D8 DEM (beta 2, tilt 0.005) after
            depression filling: long rivers, the tile-skeleton solve
Each case runs ``--reps`` times and prints the device status word.
"""
import argparse

import numpy as np
import torch

from . import api, inputs


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("case", choices=["d8", "d8_area", "d8_step", "mfd", "adjoint", "fill", "d8_plane",
                                     "d8_filled"])
    ap.add_argument("--n", type=int, default=4096, help="grid side (n x n)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=1)
    a = ap.parse_args(argv)
    n, dev = a.n, torch.device("cuda", torch.cuda.current_device())
    if a.case == "fill":
        z = inputs.fractal_dem_torch(n, n, beta=2.0, tilt=0.01, seed=a.seed, device="cuda")
        for _ in range(a.reps):
            api.fill(z)
    elif a.case in ("d8_plane", "d8_filled"):
        if a.case == "d8_plane":
            z = torch.from_numpy(np.ascontiguousarray(inputs.planar_dem(n, n, tilt=0.005, dx=30.0))).to(dev)
        else:
            z = inputs.fractal_dem_torch(n, n, beta=2.0, tilt=0.005, seed=a.seed, dx=30.0, device="cuda")
            z, _ = api.fill(z)
        R = api.routing_d8(api.receivers_d8(z, 30.0))
        for _ in range(a.reps):
            api.accumulate(R, None, want_w=False, want_area=True, device=dev)
    elif a.case.startswith("d8"):
        z = inputs.fractal_dem_torch(n, n, beta=2.0, tilt=0.01, seed=a.seed, device="cuda")
        rain = None if a.case in ("d8_area", "d8_step") else inputs.rain_field_torch(n, n, a.seed, device="cuda")
        d = api.receivers_d8(z, 30.0)
        R = api.routing_d8(d)
        for _ in range(a.reps):
            api.receivers_d8(z, 30.0)
            out = api.accumulate(R, rain, want_w=rain is not None, want_area=True, device=dev)
            if a.case == "d8_step":
                api.mass_balance(R, area=out["area"], device=dev)
    else:
        z = inputs.fractal_dem_torch(n, n, beta=2.2, tilt=0.0, seed=a.seed, device="cuda")
        for _ in range(a.reps):
            out = api.route_mfd(z, 30.0, 1.1, None, 0, want_lo=True, want_mask=True)
            if a.case == "adjoint":
                R = api.routing_mfd(out["mask"], z, 30.0, 1.1)
                api.adjoint(R, out["w"], out["w_lo"], want_dz=True)
    torch.cuda.synchronize()
    st = api.get_status(dev)
    print("case %s n=%d reps=%d status %d" % (a.case, n, a.reps, st))
    return 0 if st == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
