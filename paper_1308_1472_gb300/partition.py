"""Partition of a forest's leaves over ranks and the ghost exchange of one
step (Sec. 4 of the paper: leaves are split into contiguous ranges of the
space-filling-curve order, either by count or weighted by the work a leaf
does per coarse step; a rank receives the fields of the remote leaves its
own leaves read; the time step is a maximum over ranks and the conserved
totals a sum over ranks).  Under sub-cycling the same layer, of both time
levels, is exchanged before every substep's ghost fill; after a regrid the
leaves are repartitioned and their fields migrated (see below).

Host logic only (numpy and torch.distributed).  Every run of this library
uses one GPU, so no GPU code uses this module; it states the multi-rank plan
and is exercised by CPU ranks.  The inputs are the leaf levels in SFC order
and the neighbour table int32[n][8][4] {kind, id0, id1, orient} of
``fc_forest_get_neighbors`` (directions -x, +x, -y, +y, then the corners
(-x,-y), (+x,-y), (-x,+y), (+x,+y)).
"""
from __future__ import annotations

import numpy as np

NB_NONE, NB_SAME, NB_COARSER, NB_FINER = 0, 1, 2, 3


def leaf_weights(levels: np.ndarray, min_level: int, subcycle: bool) -> np.ndarray:
    """work of each leaf per coarse step: 1, or 2^(level - min_level)
    substeps when levels are sub-cycled (the weighted partition of Table 1)"""
    levels = np.asarray(levels, np.int64)
    if not subcycle:
        return np.ones(len(levels), np.int64)
    return np.left_shift(np.int64(1), levels - min_level)


def partition_offsets(weights: np.ndarray, nranks: int) -> np.ndarray:
    """contiguous ranges of the SFC order: rank r owns leaves
    offsets[r] .. offsets[r+1]-1.  Leaf k goes to the rank whose share
    [r W / R, (r+1) W / R) of the total weight W holds the weight before it
    (integer arithmetic, so every rank computes the same split)."""
    if nranks < 1:
        raise ValueError("nranks must be positive")
    w = np.asarray(weights, np.int64)
    if np.any(w < 0):
        raise ValueError("weights must be non-negative")
    before = np.concatenate(([0], np.cumsum(w)[:-1])) if len(w) else np.zeros(0, np.int64)
    total = int(w.sum())
    rank = (before * nranks) // max(total, 1)
    off = np.searchsorted(rank, np.arange(nranks + 1), side="left").astype(np.int64)
    off[-1] = len(w)
    return off


def owners(offsets: np.ndarray, n: int) -> np.ndarray:
    """rank of every leaf"""
    return (np.searchsorted(offsets, np.arange(n), side="right") - 1).astype(np.int64)


def _neighbours(nbr: np.ndarray, p: int, directions=range(8)):
    out = []
    for d in directions:
        kind, a, b = int(nbr[p, d, 0]), int(nbr[p, d, 1]), int(nbr[p, d, 2])
        if kind == NB_NONE:
            continue
        out.append((kind, d, a))
        if kind == NB_FINER and b >= 0:
            out.append((kind, d, b))
    return out


def step_sources(nbr: np.ndarray) -> list:
    """for every leaf, the leaves whose fields one global-dt step of it
    reads: itself and its face and corner neighbours (both leaves of a finer
    face).  That is enough under face-and-corner 2:1 balance with m >= 8:
    the ghost ring (2 cells), the coarse cells and limited slopes that
    coarse-to-fine interpolation reads (2 coarse cells = 4 fine cells from
    the face) and the fine-side fluxes that correct the leaf's boundary cells
    (3 fine cells of stencil) all lie inside the leaf's face and corner
    neighbours, which are at least m/2 >= 4 of its cells wide; a coarser
    neighbour's ghost cells in that strip come from leaves of its own level
    or finer, which are again among these neighbours."""
    n = nbr.shape[0]
    out = []
    for p in range(n):
        s = {p}
        for _, _, q in _neighbours(nbr, p):
            s.add(q)
        out.append(np.array(sorted(s), np.int64))
    return out


def ghost_layers(nbr: np.ndarray, offsets: np.ndarray) -> list:
    """per rank, the sorted remote leaves whose fields it receives before a
    step"""
    n = nbr.shape[0]
    own = owners(offsets, n)
    src = step_sources(nbr)
    layers = []
    for r in range(len(offsets) - 1):
        need = set()
        for p in range(int(offsets[r]), int(offsets[r + 1])):
            need.update(int(q) for q in src[p] if own[q] != r)
        layers.append(np.array(sorted(need), np.int64))
    return layers


def send_lists(nbr: np.ndarray, offsets: np.ndarray) -> dict:
    """(source rank, destination rank) -> sorted leaves the source sends"""
    n = nbr.shape[0]
    own = owners(offsets, n)
    out = {}
    for dst, layer in enumerate(ghost_layers(nbr, offsets)):
        for src in np.unique(own[layer]) if len(layer) else []:
            out[(int(src), dst)] = layer[own[layer] == src]
    return out


def exchange_ghosts(q: np.ndarray, offsets: np.ndarray, sends: dict, rank: int, group=None) -> None:
    """torch.distributed point-to-point exchange of the fields q[n][F][m][m]
    (this rank's own leaves valid) so that afterwards this rank's ghost
    leaves hold their owners' values.  Every rank calls it with the same
    plan."""
    import torch
    import torch.distributed as dist
    reqs, bufs = [], []
    for (src, dst), ids in sorted(sends.items()):
        if src == rank:
            t = torch.from_numpy(np.ascontiguousarray(q[ids]))
            reqs.append(dist.isend(t, dst, group=group))
            bufs.append(t)
    recv = []
    for (src, dst), ids in sorted(sends.items()):
        if dst == rank:
            t = torch.empty((len(ids),) + q.shape[1:], dtype=torch.from_numpy(q[:0]).dtype)
            reqs.append(dist.irecv(t, src, group=group))
            recv.append((ids, t))
    for r in reqs:
        r.wait()
    for ids, t in recv:
        q[ids] = t.numpy()


def max_cell_speed(q: np.ndarray, leaves: np.ndarray, g: float) -> float:
    """largest max(|u| + c, |v| + c) over the given leaves' cells (shallow
    water; the rate that sets dt after initialisation or a regrid)"""
    if len(leaves) == 0:
        return 0.0
    h, hu, hv = q[leaves, 0], q[leaves, 1], q[leaves, 2]
    c = np.sqrt(g * h)
    return float(np.maximum(np.abs(hu / h) + c, np.abs(hv / h) + c).max())


def allreduce_step_rate(q: np.ndarray, offsets: np.ndarray, rank: int, g: float, group=None) -> float:
    """global maximum wave speed: local maximum over the own leaves, then a
    maximum over ranks"""
    import torch
    import torch.distributed as dist
    t = torch.tensor([max_cell_speed(q, np.arange(offsets[rank], offsets[rank + 1]), g)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def allreduce_sums(partial: np.ndarray, group=None) -> np.ndarray:
    """global conservation sums from per-rank partial sums"""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(partial, np.float64)).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy()


# ---- repartition after a regrid ---------------------------------------------
# A regrid (Sec. 3: tag, refine or coarsen, balance, transfer) changes the
# leaves, and the weights of the new forest give new SFC ranges.  Every rank
# knows the whole forest (tree, level, x, y of each leaf) and the global
# flags, so each derives the new forest and the new ranges by itself; only
# fields move.  A new leaf's fields are built from old leaves: a kept leaf is
# copied, a refined leaf is interpolated from its old ancestor's tile with its
# ghost ring (limited linear slopes reach one cell beyond the ancestor), and a
# coarsened leaf averages its four old children.

KEPT, REFINED, COARSENED = 0, 1, 2


def regrid_origin(old, new) -> np.ndarray:
    """int64[n_new][3] = {kind, old leaf, levels} for every leaf of the new
    forest: KEPT (the old leaf with the same tree, level and position),
    REFINED (the old ancestor, `levels` levels coarser) or COARSENED (the
    first of the four old children, which are consecutive in SFC order).
    `old` and `new` are (tree, level, x, y) arrays in SFC order."""
    ot, ol, ox, oy = (np.asarray(a, np.int64) for a in old)
    index = {(int(ot[k]), int(ol[k]), int(ox[k]), int(oy[k])): k for k in range(len(ot))}
    nt, nl, nx, ny = (np.asarray(a, np.int64) for a in new)
    out = np.zeros((len(nt), 3), np.int64)
    for k in range(len(nt)):
        t, lev, x, y = int(nt[k]), int(nl[k]), int(nx[k]), int(ny[k])
        o = index.get((t, lev, x, y))
        if o is not None:
            out[k] = (KEPT, o, 0)
            continue
        for dl in range(1, lev + 1):
            o = index.get((t, lev - dl, x >> dl, y >> dl))
            if o is not None:
                out[k] = (REFINED, o, dl)
                break
        else:
            kids = [index.get((t, lev + 1, 2 * x + a, 2 * y + b)) for b in (0, 1) for a in (0, 1)]
            if any(c is None for c in kids) or kids != list(range(kids[0], kids[0] + 4)):
                raise ValueError(f"new leaf {k} has no origin in the old forest")
            out[k] = (COARSENED, kids[0], 1)
    return out


def regrid_sources(origin: np.ndarray, nbr_old: np.ndarray) -> list:
    """for every new leaf, the sorted old leaves whose fields its transfer
    reads (the old neighbour table gives a refined leaf's ghost ring)"""
    step = None
    out = []
    for kind, o, _ in np.asarray(origin, np.int64):
        if kind == KEPT:
            out.append(np.array([o], np.int64))
        elif kind == COARSENED:
            out.append(np.arange(o, o + 4, dtype=np.int64))
        else:
            if step is None:
                step = step_sources(nbr_old)
            out.append(step[int(o)])
    return out


def regrid_needs(origin: np.ndarray, nbr_old: np.ndarray, offsets_new: np.ndarray) -> list:
    """per rank of the new partition, the sorted old leaves it needs"""
    src = regrid_sources(origin, nbr_old)
    out = []
    for r in range(len(offsets_new) - 1):
        need = set()
        for k in range(int(offsets_new[r]), int(offsets_new[r + 1])):
            need.update(int(q) for q in src[k])
        out.append(np.array(sorted(need), np.int64))
    return out


def migration_lists(origin: np.ndarray, nbr_old: np.ndarray, offsets_old: np.ndarray,
                    offsets_new: np.ndarray) -> dict:
    """(old owner, new owner) -> sorted old leaves the old owner sends so
    that every rank holds what its new leaves are built from; the plan has
    the form of `send_lists`, so `exchange_ghosts` carries it out on the
    fields of the old forest"""
    n_old = nbr_old.shape[0]
    own = owners(offsets_old, n_old)
    out = {}
    for dst, need in enumerate(regrid_needs(origin, nbr_old, offsets_new)):
        remote = need[own[need] != dst] if len(need) else need
        for src in np.unique(own[remote]) if len(remote) else []:
            out[(int(src), dst)] = remote[own[remote] == src]
    return out
