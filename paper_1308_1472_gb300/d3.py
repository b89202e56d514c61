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
    python -m paper_1308_1472_gb300.d3 --table     # uniform vs adaptive to a fixed time, error vs exact
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

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


def exact_gauss(lv, x, y, z, m, t):
    """the initial Gaussian carried by the velocity for time t on the periodic
    cube, at the cell centres of every leaf (nearest periodic image)"""
    out = np.empty((len(lv), m, m, m))
    c = np.array(GAUSS[2:5]) + np.array(VEL) * t
    for k in range(len(lv)):
        dx = 1.0 / (m << int(lv[k]))
        cc = (np.arange(m) + 0.5) * dx
        pos = [x[k] * m * dx + cc, y[k] * m * dx + cc, z[k] * m * dx + cc]
        d = [(p - c[a] + 0.5) % 1.0 - 0.5 for a, p in enumerate(pos)]
        r2 = d[2][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[0][None, None, :] ** 2
        out[k] = GAUSS[0] + GAUSS[1] * np.exp(-r2 / GAUSS[5] ** 2)
    return out


def table(lmin=3, lmax=5, T=0.25, precision="f64", m=8, every=4, threshold=0.01):
    """the paper's Table 1 comparison in three dimensions: a uniform mesh at
    the finest level against adaptive meshes with one global dt and with
    sub-cycling, regridded every `every` coarse steps, to the same time T;
    whole-run wall time (steps and regrids) and L1 error against the exact
    solution"""
    import torch
    prec = fc.FC_FP32 if precision == "f32" else fc.FC_FP64
    rows = []
    for name, lo, sub in (("uniform", lmax, 0), ("AMR, global dt", lmin, 0), ("AMR, sub-cycled", lmin, 1)):
        ctx = fc3.Context3(m=m, min_level=lo, max_level=lmax, precision=prec, subcycle=sub, u=VEL[0], v=VEL[1],
                           w=VEL[2], tag_threshold=threshold, device=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if lo == lmax:
            ctx.set_initial(fc3.FC3_INIT_GAUSS, GAUSS)
        else:
            ctx.init_refine(fc3.FC3_INIT_GAUSS, GAUSS)
        t, steps, regrids, leaves_max = 0.0, 0, 0, ctx.n
        while t < T * (1 - 1e-12):
            dt = ctx.stats()["next_dt"]
            t, _ = ctx.advance(1, min(dt, T - t))
            steps += 1
            if lo < lmax and steps % every == 0 and t < T * (1 - 1e-12):
                ctx.regrid(ctx.tag())
                regrids += 1
                leaves_max = max(leaves_max, ctx.n)
        ctx.sync()
        wall = time.perf_counter() - t0
        lv, x, y, z = ctx.forest_get_leaves()
        q = ctx.read_fields().astype(np.float64)
        ex = exact_gauss(lv, x, y, z, m, t)
        vol = (1.0 / (m << lv.astype(np.int64))) ** 3
        err = float((np.abs(q - ex).reshape(len(lv), -1).sum(axis=1) * vol).sum())
        rows.append({"mesh": name, "wall_s": wall, "coarse_steps": steps, "regrids": regrids,
                     "cell_updates": ctx.stats()["cell_updates"], "leaves_max": int(leaves_max),
                     "l1_error": err})
        ctx.close()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", choices=["uniform", "amr", "amr-sub", "all"], default="all")
    ap.add_argument("--precision", choices=["f32", "f64", "both"], default="both")
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--table", action="store_true", help="uniform vs adaptive (global dt, sub-cycled) to a fixed time")
    a = ap.parse_args()
    if a.table:
        rows = table(precision="f64" if a.precision in ("f64", "all", "both") else a.precision)
        print("| mesh, time step | wall s | coarse steps | regrids | cell-updates | leaves (max) | L1 error |")
        print("|---|---|---|---|---|---|---|")
        for r in rows:
            print(f"| {r['mesh']} | {r['wall_s']:.3f} | {r['coarse_steps']} | {r['regrids']} | {r['cell_updates']:.3e} | "
                  f"{r['leaves_max']} | {r['l1_error']:.3e} |")
        print(json.dumps(rows))
        return
    rows = []
    for w in (["uniform", "amr", "amr-sub"] if a.workload == "all" else [a.workload]):
        for p in (["f32", "f64"] if a.precision == "both" else [a.precision]):
            rows.append(run(w, p, a.steps))
            print(json.dumps(rows[-1]))


if __name__ == "__main__":
    main()
