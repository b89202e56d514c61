"""Solid-body rotation on a sphere (Sec. 5 Eq. (1) of the paper, capacity
form): a Gaussian hill on the cubed sphere (Fig. 1 right), or Example 2's
field that is 1 on one half of the sphere and 0 on the other on the two-tree
sphere (--pillow, max-min tagging); one full revolution with tagging and
regridding every few coarse steps, through the C ABI only.

Reports throughput (cell-updates/s over the stepping, regrids timed apart),
the relative L1 error against the exact solution after one revolution (the
initial hill, sampled on the final forest by fc_set_initial and weighted by
cell area through fc_conservation_sums), the drift of the FP64 mass sum, and
the error for a sequence of finest levels.

    python -m paper_1308_1472_gb300.sphere            # levels 3-7, m = 32, FP32
    python -m paper_1308_1472_gb300.sphere --levels 3-5 --m 16 --precision 64
    python -m paper_1308_1472_gb300.sphere --pillow --levels 2-6 --m 16   # Example 2
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

from . import fc

OMEGA = 2.0 * math.pi          # one revolution per unit time
TILT = math.pi / 4             # rotation axis 45 degrees from +z toward +x


def equator_point(alpha=0.3, tilt=TILT):
    """(lon, lat) of a point on the rotation's equator, alpha radians from +y"""
    e1 = np.array([0.0, 1.0, 0.0])
    e2 = np.array([math.cos(tilt), 0.0, -math.sin(tilt)])
    p = math.cos(alpha) * e1 + math.sin(alpha) * e2
    return math.atan2(p[1], p[0]), math.asin(p[2])


def l1_error(ctx, params, kind, init):
    """relative area-weighted L1 difference of ctx's field to the exact
    solution after whole revolutions (the initial state) on ctx's forest"""
    ex = fc.Context(conn=params["conn"], equation=fc.FC_EQ_ADV, m=params["m"], min_level=params["lmin"],
                    max_level=params["lmax"], precision=fc.FC_FP64, omega=OMEGA, omega_axis_tilt=TILT,
                    device=params["device"])
    ex.forest_set_leaves(*ctx.forest_get_leaves())
    ex.set_initial(kind, init)
    qe = ex.read_fields()
    q = ctx.read_fields().astype(np.float64)
    ex.write_fields(np.abs(q - qe))
    num = ex.conservation_sums()[0]
    ex.write_fields(np.abs(qe))
    den = ex.conservation_sums()[0]
    ex.close()
    return float(num / den)


def run(lmin=3, lmax=7, m=32, precision=fc.FC_FP32, regrid_every=8, width=0.1, threshold=0.002, subcycle=1,
        revolutions=1.0, device=0, autotune=True, pillow=False):
    lon0, lat0 = equator_point()
    if pillow:    # Example 2: the half facing (lon, lat) holds 1; its border crosses both trees
        conn, kind, init, crit = fc.FC_CONN_PILLOW, fc.FC_INIT_HALF, [0.4, 0.5], fc.FC_TAG_MAXMIN
    else:
        conn, kind, init, crit = fc.FC_CONN_SPHERE, fc.FC_INIT_HILL, [lon0, lat0, width], fc.FC_TAG_GRAD
    ctx = fc.Context(conn=conn, equation=fc.FC_EQ_ADV, m=m, min_level=lmin, max_level=lmax,
                     precision=precision, subcycle=subcycle, tag_threshold=threshold, tag_crit=crit, cfl=0.9,
                     omega=OMEGA, omega_axis_tilt=TILT, device=device)
    ctx.init_refine(kind, init)
    s0 = ctx.conservation_sums()[0]
    if autotune:
        ctx.autotune()
    T = revolutions * 2.0 * math.pi / OMEGA
    t_step = t_regrid = 0.0
    steps = regrids = 0
    leaves_max = ctx.n
    t = 0.0
    while t < T * (1 - 1e-14):
        nd = ctx.stats()["next_dt"]
        rem = T - t
        k = regrid_every
        if nd <= 0 or k * nd >= rem:          # land exactly on T
            k = max(1, math.ceil(rem / nd)) if nd > 0 else 1
            k = min(k, regrid_every)
            dt = rem / k if k * nd >= rem else 0.0
        else:
            dt = 0.0
        a = time.perf_counter()
        t, _ = ctx.advance(k, dt)
        t_step += time.perf_counter() - a
        steps += k
        if t < T * (1 - 1e-14):
            a = time.perf_counter()
            ctx.regrid(ctx.tag())
            t_regrid += time.perf_counter() - a
            regrids += 1
            leaves_max = max(leaves_max, ctx.n)
    st = ctx.stats()
    params = dict(m=m, lmin=lmin, lmax=lmax, device=device, conn=conn)
    err = l1_error(ctx, params, kind, init)
    drift = float((ctx.conservation_sums()[0] - s0) / s0)
    out = {"sphere": "two-tree" if pillow else "cubed", "levels": f"{lmin}-{lmax}", "m": m, "precision": "f32" if precision == fc.FC_FP32 else "f64",
           "time": t, "coarse_steps": steps, "regrids": regrids, "retries": int(st["retries"]),
           "leaves_final": int(st["num_leaves"]), "leaves_max": int(leaves_max),
           "cell_updates": int(st["cell_updates"]), "step_seconds": round(t_step, 4),
           "regrid_seconds": round(t_regrid, 4),
           "cell_updates_per_s": st["cell_updates"] / t_step if t_step > 0 else None,
           "l1_error_vs_exact": err, "mass_drift": drift, "init": init}
    ctx.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--levels", default="3-7")
    ap.add_argument("--m", type=int, default=32)
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--regrid-every", type=int, default=8)
    ap.add_argument("--width", type=float, default=0.1)
    ap.add_argument("--threshold", type=float, default=None,
                    help="tagging threshold (default 0.002 for the hill's gradient, 0.05 for Example 2's max-min)")
    ap.add_argument("--pillow", action="store_true", help="Example 2 on the two-tree sphere")
    ap.add_argument("--sweep", action="store_true", help="also run every finest level from lmin + 1 up")
    args = ap.parse_args(argv)
    lmin, lmax = (int(v) for v in args.levels.split("-"))
    prec = fc.FC_FP32 if args.precision == 32 else fc.FC_FP64
    tops = range(lmin + 1, lmax + 1) if args.sweep else [lmax]
    for top in tops:
        thr = args.threshold if args.threshold is not None else (0.05 if args.pillow else 0.002)
        r = run(lmin, top, args.m, prec, args.regrid_every, args.width, thr, pillow=args.pillow)
        print(json.dumps(r), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
