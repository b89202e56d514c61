"""Learned refinement tagger: training data from the solver's own runs,
training with the library's CNN kernels (fc_cnn_loss_grad / fc_cnn_adam), use
through fc_set_tagger + fc_tag(..., FC_TAGGER_LEARNED), and the comparison
against the plain criterion.

The paper has no learned component.  The network replaces nothing: it adds a
prediction of the plain criterion's flags `horizon` steps ahead, combined with
the plain flags at tag time (see fc_set_tagger), so that regridding can run
less often while refined regions still cover where features are going.

PyTorch provides device memory only; every step runs in libfc kernels.

    python -m paper_1308_1472_gb300.tagger   # train + evaluate, prints JSON
"""
from __future__ import annotations

import ctypes
import json
import sys
import time

import numpy as np

from . import fc

S_DEFAULT = 20


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the learned tagger runs on the GPU")
    return torch


def collect(seeds, lmin=4, lmax=6, m=16, threshold=0.002, horizon=8, snapshots=6, n_humps=64, device=0):
    """Tiles (raw h, hu, hv with base depth removed later) at time t and the
    plain criterion's flags at t + horizon on the same forest, over runs of the
    hump problem with the given seeds."""
    from fc_inputs import humps_params
    torch = _torch()
    xs, ts = [], []
    for seed in seeds:
        ctx = fc.Context(m=m, min_level=lmin, max_level=lmax, precision=fc.FC_FP32, subcycle=1,
                         tag_threshold=threshold, device=device)
        ctx.init_refine(fc.FC_INIT_HUMPS, humps_params(n_humps, seed))
        for snap in range(snapshots):
            n, S = ctx.n, m + 4
            x = torch.empty((n, 3, S, S), dtype=torch.float32, device=f"cuda:{device}")
            ctx.export_tiles_device(x.data_ptr(), x.numel(), [0.0, 1.0, 1.0, 1.0])
            ctx.advance(horizon)
            f = ctx.tag()
            t = np.stack([f == 1, f == -1], axis=1).astype(np.float32)
            xs.append(x)
            ts.append(torch.from_numpy(t).to(x.device))
            ctx.regrid(f)
        ctx.close()
    return torch.cat(xs), torch.cat(ts)


def input_transform(x):
    """xform = (mean depth, 1/sd(h), 1/sd(hu), 1/sd(hv)) of the training data
    x [n][3][S][S] (device), from the library's FP64 channel statistics"""
    n, _, S, _ = x.shape
    st = np.zeros(6)
    fc.check(fc.lib().fc_cnn_input_stats(n, S, x.data_ptr(), st.ctypes.data_as(fc._dp), None), "fc_cnn_input_stats")
    return [float(st[0])] + [1.0 / max(float(v), 1e-12) for v in st[3:]]


def apply_transform(x, xf):
    """x normalised in place by the library (the transform of fc_export_tiles); returns x"""
    n, _, S, _ = x.shape
    a = np.ascontiguousarray(xf, np.float64)
    fc.check(fc.lib().fc_cnn_normalize(n, S, x.data_ptr(), a.ctypes.data_as(fc._dp), None), "fc_cnn_normalize")
    return x


def init_weights(seed=0):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.normal(size=432) * np.sqrt(2 / 27), np.zeros(16),
                           rng.normal(size=2304) * np.sqrt(2 / 144), np.zeros(16),
                           rng.normal(size=288) * np.sqrt(2 / 144), np.zeros(2)]).astype(np.float32)


def train(x, t, epochs=12, batch=4096, lr=2e-3, bf16=1, seed=0, pos_weight=True):
    """Adam on mean binary cross-entropy, mini-batches; returns (w, losses)."""
    torch = _torch()
    L = fc.lib()
    n, _, S, _ = x.shape
    w = torch.from_numpy(init_weights(seed)).to(x.device)
    m1 = torch.zeros_like(w)
    m2 = torch.zeros_like(w)
    g = torch.zeros_like(w)
    loss = ctypes.c_float()
    gen = torch.Generator(device="cpu").manual_seed(seed)
    losses, step = [], 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen).to(x.device)
        tot, nb = 0.0, 0
        for b0 in range(0, n - batch + 1 if n >= batch else 1, batch):
            idx = perm[b0:b0 + batch]
            xb = x[idx].contiguous()
            tb = t[idx].contiguous()
            step += 1
            fc.check(L.fc_cnn_loss_grad(len(idx), S, w.data_ptr(), xb.data_ptr(), tb.data_ptr(), g.data_ptr(),
                                        ctypes.byref(loss), bf16, None), "fc_cnn_loss_grad")
            fc.check(L.fc_cnn_adam(w.data_ptr(), g.data_ptr(), m1.data_ptr(), m2.data_ptr(), step,
                                   ctypes.c_float(lr), None), "fc_cnn_adam")
            tot += loss.value
            nb += 1
        losses.append(tot / max(nb, 1))
    return w.cpu().numpy(), losses


def predict(w, x, bf16=1):
    torch = _torch()
    L = fc.lib()
    n, _, S, _ = x.shape
    dw = torch.from_numpy(np.ascontiguousarray(w, np.float32)).to(x.device)
    out = torch.empty((n, 2), dtype=torch.float32, device=x.device)
    fc.check(L.fc_cnn_forward(n, S, dw.data_ptr(), x.contiguous().data_ptr(), out.data_ptr(), bf16, None),
             "fc_cnn_forward")
    return out


def accuracy(logits, t):
    p = (logits > 0).float()
    return [float((p[:, k] == t[:, k]).float().mean()) for k in range(2)]


def reference_projection(ref_q, ref_m, ref_level, leaves, m):
    """average a uniform fine solution (level ref_level, patches of ref_m cells,
    array [Nf][Nf] of h) onto the cells of an adaptive forest's leaves"""
    tr, lv, xs, ys = leaves
    out = np.zeros((len(lv), m, m))
    for k in range(len(lv)):
        r = 1 << (ref_level - lv[k])
        x0, y0 = xs[k] * m * r, ys[k] * m * r
        blk = ref_q[y0:y0 + m * r, x0:x0 + m * r]
        out[k] = blk.reshape(m, r, m, r).mean(axis=(1, 3))
    return out


def run_amr(tagger, w, xf, seed, steps, regrid_every, dt_coarse, lmin, lmax, m, threshold, n_humps, device=0):
    from fc_inputs import humps_params
    ctx = fc.Context(m=m, min_level=lmin, max_level=lmax, precision=fc.FC_FP32, subcycle=1,
                     tag_threshold=threshold, device=device)
    ctx.init_refine(fc.FC_INIT_HUMPS, humps_params(n_humps, seed))
    if tagger == fc.FC_TAGGER_LEARNED:
        ctx.set_tagger(w, xf, bf16=1)
    done = 0
    while done < steps:
        k = min(regrid_every, steps - done)
        ctx.advance(k, dt_coarse)
        done += k
        if done < steps:
            ctx.regrid(ctx.tag(tagger))
    st = ctx.stats()
    h = ctx.read_fields()[:, 0].astype(np.float64)
    leaves = ctx.forest_get_leaves()
    ctx.close()
    return h, leaves, st


def uniform_reference(seed, steps, dt_coarse, lmin, lmax, m, n_humps, device=0):
    """the same problem on the uniform finest level, dt_coarse / 2^(lmax - lmin) per step"""
    from fc_inputs import humps_params
    ctx = fc.Context(m=m, min_level=lmax, max_level=lmax, precision=fc.FC_FP32, device=device)
    ctx.set_initial(fc.FC_INIT_HUMPS, humps_params(n_humps, seed))
    r = 1 << (lmax - lmin)
    ctx.advance(steps * r, dt_coarse / r)
    q = ctx.read_fields()[:, 0].astype(np.float64)
    tr, lv, xs, ys = ctx.forest_get_leaves()
    N = (1 << lmax) * m
    H = np.zeros((N, N))
    for k in range(len(lv)):
        H[ys[k] * m:(ys[k] + 1) * m, xs[k] * m:(xs[k] + 1) * m] = q[k]
    ctx.close()
    return H


def l1_error(h, leaves, H, lmax, m):
    proj = reference_projection(H, m, lmax, leaves, m)
    tr, lv, _, _ = leaves
    area = np.array([(1.0 / ((1 << l) * m)) ** 2 for l in lv])
    return float((np.abs(h - proj).sum(axis=(1, 2)) * area).sum())


def evaluate(w, xf, seed=999, steps=32, lmin=4, lmax=6, m=16, threshold=0.002, n_humps=64, device=0):
    """L1 error against the uniform finest-level run and cell-updates for the
    plain criterion (regrid every 4 and every 8 steps) and the learned tagger
    (regrid every 8 steps)."""
    dx_c = 1.0 / ((1 << lmin) * m)
    dt_c = 0.9 * dx_c / 2.0          # speeds stay below 2 for these humps (depth <= ~2)
    H = uniform_reference(seed, steps, dt_c, lmin, lmax, m, n_humps, device)
    out = {}
    for name, tagger, every in (("plain_every4", fc.FC_TAGGER_PLAIN, 4), ("plain_every8", fc.FC_TAGGER_PLAIN, 8),
                                ("learned_every8", fc.FC_TAGGER_LEARNED, 8)):
        h, leaves, st = run_amr(tagger, w, xf, seed, steps, every, dt_c, lmin, lmax, m, threshold, n_humps, device)
        out[name] = {"l1_error": l1_error(h, leaves, H, lmax, m), "cell_updates": int(st["cell_updates"]),
                     "regrids": int(st["regrids"]), "leaves_final": int(st["num_leaves"])}
    return out


def _interp(xs, ys, x, logy):
    """piecewise-linear interpolation of y(x) between sorted points (in log y
    if logy), None outside the points' range"""
    for k in range(len(xs) - 1):
        a, b = xs[k], xs[k + 1]
        if min(a, b) <= x <= max(a, b) and a != b:
            u = (x - a) / (b - a)
            if logy:
                return float(np.exp(np.log(ys[k]) + u * (np.log(ys[k + 1]) - np.log(ys[k]))))
            return float(ys[k] + u * (ys[k + 1] - ys[k]))
    return None


def pareto(w, xf, thresholds=(0.003, 0.002, 0.0015, 0.001, 0.0007), every=8, seed=999, steps=32, lmin=4, lmax=6,
           m=16, n_humps=64, device=0):
    """L1 error in h (against the uniform finest-level run) and cell-updates of
    the plain criterion and of the learned tagger at each tag threshold, both
    regridding every `every` coarse steps; for each learned point, the plain
    curve's error at the same cell-updates (interpolated linearly in cell-
    updates and logarithmically in error between plain points) and the plain
    curve's cell-updates at the same error"""
    dx_c = 1.0 / ((1 << lmin) * m)
    dt_c = 0.9 * dx_c / 2.0          # speeds stay below 2 for these humps (depth <= ~2)
    H = uniform_reference(seed, steps, dt_c, lmin, lmax, m, n_humps, device)
    curves = {}
    for name, tg in (("plain", fc.FC_TAGGER_PLAIN), ("learned", fc.FC_TAGGER_LEARNED)):
        pts = []
        for thr in thresholds:
            h, leaves, st = run_amr(tg, w, xf, seed, steps, every, dt_c, lmin, lmax, m, thr, n_humps, device)
            pts.append({"threshold": thr, "l1_error": l1_error(h, leaves, H, lmax, m),
                        "cell_updates": int(st["cell_updates"]), "regrids": int(st["regrids"])})
        curves[name] = sorted(pts, key=lambda d: d["cell_updates"])
    pc = [d["cell_updates"] for d in curves["plain"]]
    pe = [d["l1_error"] for d in curves["plain"]]
    comp = []
    for d in curves["learned"]:
        comp.append({"threshold": d["threshold"], "l1_error": d["l1_error"], "cell_updates": d["cell_updates"],
                     "plain_error_at_same_cell_updates": _interp(pc, pe, d["cell_updates"], True),
                     "plain_cell_updates_at_same_error": _interp(pe, pc, d["l1_error"], False)})
    return {"regrid_every": every, "plain": curves["plain"], "learned": curves["learned"], "comparison": comp}


def cnn_throughput(w, x, reps=5):
    """patches per second and TFLOP/s of the forward pass (1.57 MFLOP per
    20 x 20 patch) on the device data x, event-timed"""
    torch = _torch()
    n = x.shape[0]
    predict(w, x)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        predict(w, x)
    b.record()
    torch.cuda.synchronize()
    s = a.elapsed_time(b) / 1000.0 / reps
    S = x.shape[2]
    flops = 2 * ((S - 2) ** 2 * 16 * 27 + (S - 4) ** 2 * 16 * 144 + (S - 6) ** 2 * 2 * 144)
    return {"patches_per_s": n / s, "tflops": n * flops / s / 1e12, "patches": int(n)}


def main():
    t0 = time.time()
    x, t = collect(seeds=range(1, 9))
    xf = input_transform(x)
    xt = apply_transform(x, xf)
    n = x.shape[0]
    ntr = int(0.85 * n)
    w, losses = train(xt[:ntr], t[:ntr])
    acc = accuracy(predict(w, xt[ntr:]), t[ntr:])
    ev = evaluate(w, xf)
    pa = pareto(w, xf)
    print(json.dumps({"samples": int(n), "train_losses": [round(v, 4) for v in losses],
                      "holdout_accuracy_refine_coarsen": acc, "xform": xf, "evaluation": ev, "pareto": pa,
                      "cnn_forward": cnn_throughput(w, xt), "seconds": round(time.time() - t0, 1)}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
