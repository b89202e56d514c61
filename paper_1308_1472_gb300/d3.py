"""Throughput of the three-dimensional path on one GPU.

Scalar advection (Eq. (1) of Sec. 5 in three dimensions) of a smooth
Gaussian on the periodic unit cube, octree of m^3 patches, diagonal constant
velocity.  Two workloads:
  * uniform: every patch at one level (level 5, m = 8: 32^3 patches,
    16.8 M cells; the state, two buffers, is larger than the 129 MB L2 in
    FP64 and about its size in FP32);
  * amr: levels lmin..lmax refined around the Gaussian (max - min tagging),
    regridded every 8 steps (regrids timed separately), one global dt;
  * amr-sub: the same with sub-cycling (level l takes 2^(l - lmin) substeps).
`python bench.py --d3` times the same workloads with the CPU oracle beside.
Steps are timed with CUDA events on the context's stream after warm-up;
cell-updates are interior cells advanced by one step.  The update's
algorithmic traffic is one read and one write of q per cell-update (2 S
bytes, S = 4 or 8), reported against the measured HBM copy bandwidth.

    python -m paper_1308_1472_gb300.d3 [--workload uniform|amr|amr-sub] [--precision f32|f64] [--steps 40]
"""
from __future__ import annotations

import argparse
import json
import os
import time

from . import fc
from . import fc3

GAUSS = [0.1, 1.0, 0.5, 0.5, 0.5, 0.12]
VEL = (0.8, 0.6, -0.7)


def hbm_peak():
    p = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return float(json.load(fh).get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def run(workload="uniform", precision="f32", steps=40, warmup=5, level=5, m=8, lmin=3, lmax=5, threshold=0.01):
    """cell-updates / s of one workload; under sub-cycling a step is a coarse
    step and a leaf of level l counts 2^(l - lmin) cell-updates per cell"""
    import torch
    prec = fc.FC_FP32 if precision == "f32" else fc.FC_FP64
    S = 4 if precision == "f32" else 8
    stream = torch.cuda.current_stream()
    kw = dict(m=m, precision=prec, u=VEL[0], v=VEL[1], w=VEL[2], tag_threshold=threshold, device=0,
              stream=stream.cuda_stream)
    if workload == "uniform":
        ctx = fc3.Context3(min_level=level, max_level=level, **kw)
        ctx.set_initial(fc3.FC3_INIT_GAUSS, GAUSS)
    else:
        ctx = fc3.Context3(min_level=lmin, max_level=lmax, subcycle=1 if workload == "amr-sub" else 0, **kw)
        ctx.init_refine(fc3.FC3_INIT_GAUSS, GAUSS)
    n = ctx.n
    lv = ctx.forest_get_leaves()[0]
    dt = ctx.stats()["next_dt"]
    ctx.advance(warmup, dt)
    s0 = ctx.conservation_sum()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    regrid_s, done, cu = 0.0, 0, 0.0
    total_ms = 0.0
    adaptive = workload != "uniform"
    while done < steps:
        k = min(8, steps - done) if adaptive else steps
        c0 = ctx.stats()["cell_updates"]
        ev[0].record(stream)
        ctx.advance(k, dt)
        ev[1].record(stream)
        torch.cuda.synchronize()
        total_ms += ev[0].elapsed_time(ev[1])
        cu += ctx.stats()["cell_updates"] - c0
        done += k
        if adaptive and done < steps:
            t0 = time.perf_counter()
            ctx.regrid(ctx.tag())
            regrid_s += time.perf_counter() - t0
            dt = ctx.stats()["next_dt"]
    drift = (ctx.conservation_sum() - s0) / s0
    peak, src = hbm_peak()
    rate = cu / (total_ms * 1e-3)
    gbs = rate * 2 * S / 1e9
    out = {"workload": workload, "precision": precision, "m": m, "leaves": int(n), "levels": sorted(set(lv.tolist())),
           "steps": steps, "ms_per_step": total_ms / steps, "cell_updates_per_s": rate,
           "hbm": {"achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak, "peak_source": src,
                   "bytes_per_cell_update": 2 * S},
           "mass_drift": drift, "regrid_s": regrid_s}
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["uniform", "amr", "amr-sub", "all"], default="all")
    ap.add_argument("--precision", choices=["f32", "f64", "both"], default="both")
    ap.add_argument("--steps", type=int, default=40)
    a = ap.parse_args()
    rows = []
    for w in (["uniform", "amr", "amr-sub"] if a.workload == "all" else [a.workload]):
        for p in (["f32", "f64"] if a.precision == "both" else [a.precision]):
            rows.append(run(w, p, a.steps))
            print(json.dumps(rows[-1]))


if __name__ == "__main__":
    main()
