"""Partition of the leaves over ranks (Sec. 4: contiguous SFC ranges by count
or by work weight) and the ghost exchange of a step, checked on CPU ranks:
gloo processes each step the oracle on their own leaves after receiving
their ghost layer, with every other leaf replaced by an unrelated state, and
their own leaves must equal the unpartitioned run bit for bit (the paper's
partition-independence of the results)."""
import os
import socket
import sys

import numpy as np
import pytest

from fc_inputs import dambreak_params, humps_params
from oracle import fco
from oracle.fco import Oracle, OracleParams
from paper_1308_1472_gb300 import partition as pt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_offsets_cover_in_order_and_balance():
    rng = np.random.default_rng(5)
    for nranks in (1, 2, 3, 7):
        for n in (1, 5, 100):
            w = rng.integers(1, 9, n)
            off = pt.partition_offsets(w, nranks)
            assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 0)
            # rank r holds exactly the leaves whose preceding weight lies in its share
            before = np.concatenate(([0], np.cumsum(w)[:-1]))
            own = pt.owners(off, n)
            assert np.array_equal(own, (before * nranks) // w.sum())
            # so no rank exceeds its share by more than one leaf's weight
            share = w.sum() / nranks
            for r in range(nranks):
                assert w[off[r]:off[r + 1]].sum() <= share + w.max()


def test_weights_follow_substeps():
    lv = np.array([3, 4, 4, 5, 3])
    assert np.array_equal(pt.leaf_weights(lv, 3, False), [1, 1, 1, 1, 1])
    assert np.array_equal(pt.leaf_weights(lv, 3, True), [1, 2, 2, 4, 1])
    # weighted partition of a forest whose fine leaves sit at the end
    w = pt.leaf_weights(np.array([2] * 12 + [4] * 4), 2, True)
    off = pt.partition_offsets(w, 2)
    # weight before leaf 12 is 12 (rank 0's share is [0, 14)), before leaf 13 it is 16
    assert off[1] == 13


def _forest(m=8, lmin=2, lmax=4, init="dam"):
    o = Oracle(OracleParams(m=m, min_level=lmin, max_level=lmax, subcycle=0))
    if init == "dam":
        o.init_refine(fco.INIT_DAMBREAK, dambreak_params())
    else:
        o.init_refine(fco.INIT_HUMPS, humps_params(12, 7))
    return o


def test_ghost_layer_is_the_remote_face_and_corner_neighbours():
    o = _forest()
    nbr = o.neighbors()
    _, lv, _, _ = o.leaves()
    assert len(np.unique(lv)) > 1
    off = pt.partition_offsets(np.ones(o.n, np.int64), 3)
    own = pt.owners(off, o.n)
    layers = pt.ghost_layers(nbr, off)
    for r, layer in enumerate(layers):
        brute = set()
        for p in range(off[r], off[r + 1]):
            for d in range(8):
                kind, a, b = nbr[p, d, :3]
                for q in (a, b):
                    if kind != pt.NB_NONE and q >= 0 and own[q] != r:
                        brute.add(int(q))
        assert layer.tolist() == sorted(brute)
    # the send lists are the layers seen from the owners
    sends = pt.send_lists(nbr, off)
    for (src, dst), ids in sends.items():
        assert np.all(own[ids] == src) and np.all(np.isin(ids, layers[dst]))


def _emulated_ranks_agree(o_init, layers, off, dt):
    """every rank's own leaves after one step from its own leaves plus the
    given layer (everything else an unrelated lake at rest), compared with
    the unpartitioned step; ranks emulated in one process"""
    ref = _forest(init=o_init)
    q0 = ref.fields()
    ref.advance(1, dt)
    full = ref.fields()
    out = []
    for r, layer in enumerate(layers):
        keep = np.zeros(ref.n, bool)
        keep[off[r]:off[r + 1]] = True
        keep[layer] = True
        q = q0.copy()
        q[~keep] = 0.0
        q[~keep, 0] = 0.7
        loc = _forest(init=o_init)
        loc.set_fields(q)
        loc.advance(1, dt)
        out.append(np.array_equal(loc.fields()[off[r]:off[r + 1]], full[off[r]:off[r + 1]]))
    return out


@pytest.mark.parametrize("nranks", [2, 3])
def test_corner_neighbours_are_needed(nranks):
    """the bit-exact comparison sees a layer without the corner neighbours
    (transverse terms and corner ghost cells read them): the plan's layer
    passes, a faces-only layer fails on every rank"""
    o = _forest(init="humps")
    nbr = o.neighbors()
    off = pt.partition_offsets(np.ones(o.n, np.int64), nranks)
    own = pt.owners(off, o.n)
    dt = 0.5 * o.next_dt
    assert all(_emulated_ranks_agree("humps", pt.ghost_layers(nbr, off), off, dt))
    faces = []
    for r in range(nranks):
        s = set()
        for p in range(off[r], off[r + 1]):
            for d in range(4):
                kind, a, b = nbr[p, d, :3]
                s.update(int(q) for q in (a, b) if kind != pt.NB_NONE and q >= 0 and own[q] != r)
        faces.append(np.array(sorted(s), np.int64))
    assert not any(_emulated_ranks_agree("humps", faces, off, dt))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, init, weighted, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle.fco import Oracle as Ora  # noqa: F811
    from paper_1308_1472_gb300 import partition as P
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ref = _forest(init=init)
    loc = _forest(init=init)
    nbr = ref.neighbors()
    _, lv, _, _ = ref.leaves()
    w = P.leaf_weights(lv, int(lv.min()), weighted)
    off = P.partition_offsets(w, world)
    sends = P.send_lists(nbr, off)
    mine = np.arange(off[rank], off[rank + 1])
    layer = P.ghost_layers(nbr, off)[rank]
    keep = np.zeros(ref.n, bool)
    keep[mine] = True
    keep[layer] = True
    q = ref.fields()
    q[~keep] = 0.0                      # nothing but the own leaves is known ...
    q[~np.isin(np.arange(ref.n), mine)] = 0.0
    dt = 0.5 * ref.next_dt
    ok = True
    for step in range(3):
        P.exchange_ghosts(q, off, sends, rank)
        # ... and after the exchange the leaves outside the ghost layer hold
        # an unrelated state (lake at rest, lower depth)
        q[~keep] = 0.0
        q[~keep, 0] = 0.7
        loc.set_fields(q)
        loc.advance(1, dt)
        ref.advance(1, dt)
        qn = loc.fields()
        q[mine] = qn[mine]
        ok = ok and np.array_equal(q[mine], ref.fields()[mine])
        rate = P.allreduce_step_rate(q, off, rank, 1.0)
        full = ref.fields()
        ok = ok and rate == P.max_cell_speed(full, np.arange(ref.n), 1.0)
        area = (1.0 / ((1 << lv[mine]) * 8.0)) ** 2
        part = (q[mine].sum(axis=(2, 3)) * area[:, None]).sum(axis=0)
        sums = P.allreduce_sums(part)
        ok = ok and np.allclose(sums, ref.sums(), rtol=1e-13, atol=1e-15)
    out[rank] = ok
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,init,weighted", [(2, "dam", False), (3, "humps", True)])
def test_partitioned_steps_equal_unpartitioned(world, init, weighted):
    torch = pytest.importorskip("torch")
    fco.oracle_lib()                       # built before the ranks start
    mp = torch.multiprocessing.get_context("spawn")
    manager = mp.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, world, port, init, weighted, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    assert all(out[r] for r in range(world))


def _sphere(conn):
    """an adapted forest on one of the spheres (Sec. 5, Eq. (1) in capacity
    form): Example 2's half-sphere field on the two trees, the hill on the
    cube's six"""
    o = Oracle(OracleParams(conn=conn, equation=fco.EQ_ADV, m=8, min_level=1, max_level=3,
                            omega=2 * np.pi, omega_axis_tilt=np.pi / 4, tag_threshold=0.05,
                            tag_crit=fco.TAG_MAXMIN))
    if conn == fco.CONN_PILLOW:
        o.init_refine(fco.INIT_HALF, [0.4, 0.5])
    else:
        o.init_refine(fco.INIT_HILL, [0.3, 0.2, 0.35])
    return o


def _sphere_ranks_agree(conn, layers, off, q0, dt, full):
    out = []
    for r, layer in enumerate(layers):
        keep = np.zeros(len(q0), bool)
        keep[off[r]:off[r + 1]] = True
        keep[layer] = True
        q = q0.copy()
        q[~keep] = 0.3
        loc = _sphere(conn)
        loc.set_fields(q)
        loc.advance(1, dt)
        out.append(np.array_equal(loc.fields()[off[r]:off[r + 1]], full[off[r]:off[r + 1]]))
    return out


@pytest.mark.parametrize("conn,nranks", [(fco.CONN_PILLOW, 2), (fco.CONN_PILLOW, 3), (fco.CONN_SPHERE, 3)])
def test_sphere_partition_is_exact(conn, nranks):
    """on the spheres the layer crosses tree borders with their orientation
    maps (and on the two-tree sphere a corner leaf is its own diagonal
    neighbour): each emulated rank's own leaves after one step from its own
    leaves and its layer, every other leaf holding an unrelated constant,
    equal the unpartitioned step bit for bit; a layer of face neighbours
    only does not"""
    ref = _sphere(conn)
    nbr = ref.neighbors()
    _, lv, _, _ = ref.leaves()
    assert len(np.unique(lv)) > 1
    if conn == fco.CONN_PILLOW:
        self_diag = [p for p in range(ref.n) for d in range(4, 8) if nbr[p, d, 0] == pt.NB_SAME and nbr[p, d, 1] == p]
        assert self_diag                                  # the singular corners are in the forest
    off = pt.partition_offsets(np.ones(ref.n, np.int64), nranks)
    own = pt.owners(off, ref.n)
    layers = pt.ghost_layers(nbr, off)
    for r, layer in enumerate(layers):
        assert not np.any((layer >= off[r]) & (layer < off[r + 1]))
    q0 = ref.fields()
    dt = 0.5 * ref.next_dt
    ref.advance(1, dt)
    full = ref.fields()
    assert all(_sphere_ranks_agree(conn, layers, off, q0, dt, full))
    if conn == fco.CONN_PILLOW and nranks == 2:
        return    # one tree per rank: here every remote diagonal neighbour is also a remote face neighbour
    faces = []
    for r in range(nranks):
        s = set()
        for p in range(off[r], off[r + 1]):
            for d in range(4):
                kind, a, b = nbr[p, d, :3]
                s.update(int(x) for x in (a, b) if kind != pt.NB_NONE and x >= 0 and own[x] != r)
        faces.append(np.array(sorted(s), np.int64))
    assert not all(_sphere_ranks_agree(conn, faces, off, q0, dt, full))
