"""Dam-break runs through the C ABI only (Sec. 5 style experiments with the
shallow-water equations): the single-level 32 x 32 run and the adaptive run
with tagging and regridding every few steps, in FP64 and FP32.

Each reports the time, step and regrid wall-clock times, cell-updates/s, the
leaf counts it went through and the drift of the FP64 mass sum; the adaptive
run also reports the relative L1 difference of FP32 from FP64 at the end.

    python -m paper_1308_1472_gb300.runs single      # level 2, m = 8, FP64, 50 steps
    python -m paper_1308_1472_gb300.runs adaptive    # levels 3-6, m = 16, 400 steps, regrid every 4
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import fc

DAMBREAK = [0.5, 0.5, 0.04, 2.0, 1.0]      # centre (0.5, 0.5), r^2 = 0.04, h 2 inside, 1 outside


def single(steps=50, device=0):
    ctx = fc.Context(m=8, min_level=2, max_level=2, precision=fc.FC_FP64, cfl=0.9, device=device)
    ctx.set_initial(fc.FC_INIT_DAMBREAK, DAMBREAK)
    s0 = ctx.conservation_sums()
    ctx.advance(1)
    a = time.perf_counter()
    t, _ = ctx.advance(steps - 1)
    el = time.perf_counter() - a
    st = ctx.stats()
    out = {"run": "dam break, one level", "levels": "2", "m": 8, "precision": "f64", "steps": steps, "time": t,
           "leaves": int(st["num_leaves"]), "cell_updates": int(st["cell_updates"]),
           "cell_updates_per_s": (steps - 1) * 16 * 64 / el, "step_seconds": round(el, 5),
           "mass_drift": float((ctx.conservation_sums()[0] - s0[0]) / s0[0])}
    ctx.close()
    return out


def adaptive(precision, steps=400, regrid_every=4, lmin=3, lmax=6, m=16, threshold=0.05, subcycle=0,
             device=0):
    ctx = fc.Context(m=m, min_level=lmin, max_level=lmax, precision=precision, subcycle=subcycle,
                     tag_threshold=threshold, cfl=0.9, device=device)
    ctx.init_refine(fc.FC_INIT_DAMBREAK, DAMBREAK)
    s0 = ctx.conservation_sums()[0]
    ctx.autotune()
    t_step = t_regrid = 0.0
    done = regrids = 0
    leaves = [ctx.n]
    while done < steps:
        k = min(regrid_every, steps - done)
        a = time.perf_counter()
        t, _ = ctx.advance(k)
        t_step += time.perf_counter() - a
        done += k
        if done < steps:
            a = time.perf_counter()
            ctx.regrid(ctx.tag())
            t_regrid += time.perf_counter() - a
            regrids += 1
            leaves.append(ctx.n)
    st = ctx.stats()
    out = {"run": "dam break, adaptive", "levels": f"{lmin}-{lmax}", "m": m,
           "precision": "f32" if precision == fc.FC_FP32 else "f64", "subcycle": bool(subcycle),
           "steps": steps, "time": t, "regrids": regrids, "retries": int(st["retries"]),
           "leaves_min": int(min(leaves)), "leaves_max": int(max(leaves)), "cell_updates": int(st["cell_updates"]),
           "step_seconds": round(t_step, 4), "regrid_seconds": round(t_regrid, 4),
           "cell_updates_per_s": st["cell_updates"] / t_step,
           "cell_updates_per_s_with_regrid": st["cell_updates"] / (t_step + t_regrid),
           "mass_drift": float((ctx.conservation_sums()[0] - s0) / s0)}
    leaves_final = ctx.forest_get_leaves()
    h = ctx.read_fields(0).astype(np.float64)
    ctx.close()
    return out, leaves_final, h


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["single", "adaptive"])
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--subcycle", type=int, default=0)
    args = ap.parse_args(argv)
    if args.which == "single":
        print(json.dumps(single(args.steps or 50)))
        return 0
    steps = args.steps or 400
    r64, l64, h64 = adaptive(fc.FC_FP64, steps, subcycle=args.subcycle)
    print(json.dumps(r64), flush=True)
    r32, l32, h32 = adaptive(fc.FC_FP32, steps, subcycle=args.subcycle)
    same_forest = all(np.array_equal(a, b) for a, b in zip(l32, l64))
    r32["same_final_forest_as_f64"] = bool(same_forest)
    if same_forest:
        r32["rel_l1_vs_f64"] = float(np.abs(h32 - h64).sum() / np.abs(h64).sum())
    print(json.dumps(r32), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
