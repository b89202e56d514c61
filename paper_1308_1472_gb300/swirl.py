"""The paper's Example 1 and Table 1 on one GPU.

Scalar advection (Eq. 1) of a concentration that is 0 on the left half of
the unit square and 1 on the right half, in the swirl velocity field
(stream function sin^2(pi x) sin^2(pi y) / pi; the paper prescribes a
distorting flow without giving it), patches of m = 8 cells, tagging by the
max - min criterion of Sec. 5.  Table 1 compares, for a fixed maximum level
8 and minimum level 3, a uniform level-8 mesh with adaptive meshes under one
global dt or sub-cycled levels, regridded after every coarse step or every
4; this runner times each strategy's whole run (initialisation, steps,
regrids) with every kernel on the GPU and reports the cell-updates and the
L1 difference of the final field to the uniform run.  Count and weight
partitions (the table's third column) have no counterpart on one GPU.

    python -m paper_1308_1472_gb300.swirl [--levels 3-8] [--t 0.5] [--precision f64]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import fc

BOX = [0.5, 1.0, 0.0, 1.0, 1.0, 0.0]     # q = 1 on the right half, 0 elsewhere


def run(strategy, lmin, lmax, T, m=8, precision=fc.FC_FP64, threshold=0.05, device=0):
    """one strategy: ("uniform", 0, 0) or ("amr", subcycle, regrid_every)"""
    import torch
    kind, subcycle, every = strategy
    lo = lmax if kind == "uniform" else lmin
    ctx = fc.Context(equation=fc.FC_EQ_ADV, m=m, min_level=lo, max_level=lmax, precision=precision,
                     subcycle=subcycle, tag_crit=fc.FC_TAG_MAXMIN, tag_threshold=threshold, adv_u=1.0,
                     velocity=fc.FC_VEL_SWIRL, device=device)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    if kind == "uniform":
        ctx.set_initial(fc.FC_INIT_ADV_BOX, BOX)
    else:
        ctx.init_refine(fc.FC_INIT_ADV_BOX, BOX)
    steps = regrids = 0
    leaves_max = 0
    while True:
        st = ctx.stats()
        t = st["time"]
        if t >= T * (1 - 1e-12):
            break
        dt = st["next_dt"]
        if t + dt > T:
            ctx.advance(1, T - t)
        else:
            ctx.advance(1)
        steps += 1
        if kind != "uniform" and steps % every == 0:
            ctx.regrid(ctx.tag())
            regrids += 1
        leaves_max = max(leaves_max, ctx.stats()["num_leaves"])
    ctx.sync()
    torch.cuda.synchronize(device)
    wall = time.perf_counter() - t0
    st = ctx.stats()
    q = ctx.read_fields(0).astype(np.float64)
    _, lv, xs, ys = ctx.forest_get_leaves()
    N = (1 << lmax) * m
    G = np.zeros((N, N))
    for k in range(len(lv)):
        r = 1 << (lmax - lv[k])
        G[ys[k] * m * r:(ys[k] + 1) * m * r, xs[k] * m * r:(xs[k] + 1) * m * r] = np.kron(q[k], np.ones((r, r)))
    out = {"wall_s": wall, "coarse_steps": steps, "regrids": regrids, "cell_updates": int(st["cell_updates"]),
           "final_leaves": int(st["num_leaves"]), "max_leaves": int(leaves_max), "time": st["time"],
           "mass": float(ctx.conservation_sums()[0])}
    ctx.close()
    return out, G


STRATEGIES = [
    ("uniform, none, global", ("uniform", 0, 1)),
    ("AMR, every step, global", ("amr", 0, 1)),
    ("AMR, every 4, global", ("amr", 0, 4)),
    ("AMR, every step, subcycle", ("amr", 1, 1)),
    ("AMR, every 4, subcycle", ("amr", 1, 4)),
]


def table1(lmin=3, lmax=8, T=0.5, precision=fc.FC_FP64, warm=True):
    if warm:       # compile / first-touch costs out of the timings
        run(("amr", 1, 4), 2, 4, 0.05, precision=precision)
    rows, ref = [], None
    for name, strat in STRATEGIES:
        r, G = run(strat, lmin, lmax, T, precision=precision)
        if ref is None:
            ref = G
        dx = 1.0 / ref.shape[0]
        r["l1_vs_uniform"] = float(np.abs(G - ref).sum() * dx * dx)
        r["strategy"] = name
        rows.append(r)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--levels", default="3-8")
    ap.add_argument("--t", type=float, default=0.5)
    ap.add_argument("--precision", choices=["f32", "f64"], default="f64")
    a = ap.parse_args()
    lmin, lmax = (int(v) for v in a.levels.split("-"))
    prec = fc.FC_FP32 if a.precision == "f32" else fc.FC_FP64
    rows = table1(lmin, lmax, a.t, prec)
    print("| mesh, remesh, time step | wall s | coarse steps | regrids | cell-updates | leaves (max) | "
          "L1 vs uniform |")
    print("|---|---|---|---|---|---|---|")
    for r in rows:
        print(f"| {r['strategy']} | {r['wall_s']:.3f} | {r['coarse_steps']} | {r['regrids']} | "
              f"{r['cell_updates']:.3e} | {r['max_leaves']} | {r['l1_vs_uniform']:.2e} |")
    print(json.dumps(rows))


if __name__ == "__main__":
    main()
