"""The oracle's table-driven connectivity (Sec. 2: each tree a reference
square, the trees' connectivity given from outside) against what fixes it:
tables written from the definitions of the four built-in connectivities
(walls, the periodic square, the two-tree sphere's continued x borders and
half-turned y borders, the cubed sphere's face frames) reproduce the oracle's
point maps bit for bit, corners included (four cells meeting, two cells
meeting at the two-tree sphere's equator points, no image where three cube
faces meet); and a 2 x 2 brick of trees maps every point as one square one
level finer does."""
import ctypes as C

import numpy as np
import pytest

from oracle import fco

N = 1 << 30


def _table(entries, ntrees):
    tab = np.full((ntrees, 4, 3), -1, np.int32)
    for (t, s), (t2, s2, flip) in entries.items():
        tab[t, s] = (t2, s2, flip)
    return np.ascontiguousarray(tab)


def table_square():
    return _table({}, 1)


def table_periodic():
    return _table({(0, 0): (0, 1, 0), (0, 1): (0, 0, 0), (0, 2): (0, 3, 0), (0, 3): (0, 2, 0)}, 1)


def table_pillow():
    """x borders continue into the other tree; a y border meets the same y
    border of the other tree with x reversed"""
    e = {}
    for t in (0, 1):
        e[(t, 1)] = (1 - t, 0, 0)
        e[(t, 0)] = (1 - t, 1, 0)
        e[(t, 2)] = (1 - t, 2, 1)
        e[(t, 3)] = (1 - t, 3, 1)
    return _table(e, 2)


FRAMES = [((0, 1, 0), (0, 0, 1)), ((-1, 0, 0), (0, 0, 1)), ((0, -1, 0), (0, 0, 1)),
          ((1, 0, 0), (0, 0, 1)), ((0, 1, 0), (-1, 0, 0)), ((0, 1, 0), (1, 0, 0))]


def table_cube():
    """from the face frames alone: tree t on the face with normal a_t x b_t;
    across side +x lies the face whose normal is a_t (side -x: -a_t, +y: b_t,
    -y: -b_t); the neighbour's side facing t is the one whose outward
    direction is n_t; the coordinate along the shared edge runs along b (x
    sides) or a (y sides) in each tree, reversed if those directions differ"""
    a = [np.array(f[0]) for f in FRAMES]
    b = [np.array(f[1]) for f in FRAMES]
    n = [np.cross(a[t], b[t]) for t in range(6)]
    out_dir = lambda t, s: [-a[t], a[t], -b[t], b[t]][s]          # noqa: E731
    along = lambda t, s: b[t] if s < 2 else a[t]                  # noqa: E731
    e = {}
    for t in range(6):
        for s in range(4):
            t2 = next(u for u in range(6) if np.array_equal(n[u], out_dir(t, s)))
            s2 = next(k for k in range(4) if np.array_equal(out_dir(t2, k), n[t]))
            flip = int(not np.array_equal(along(t, s), along(t2, s2)))
            e[(t, s)] = (t2, s2, flip)
    return _table(e, 6)


def _tmap(lib, tab, t, X, Y):
    xo, yo = C.c_longlong(), C.c_longlong()
    r = lib.fco_table_map_point(tab.ctypes.data_as(C.POINTER(C.c_int32)), t, X, Y, C.byref(xo), C.byref(yo))
    return (r, xo.value, yo.value) if r >= 0 else (-1, 0, 0)


def _omap(lib, conn, t, X, Y):
    xo, yo = C.c_longlong(), C.c_longlong()
    r = lib.fco_map_point(conn, t, X, Y, C.byref(xo), C.byref(yo))
    return (r, xo.value, yo.value) if r >= 0 else (-1, 0, 0)


def _points(rng, k):
    """points inside and in a band of half a tree around it, with the
    corners and the cells next to the borders oversampled"""
    X = rng.integers(-N // 2, N + N // 2, k)
    Y = rng.integers(-N // 2, N + N // 2, k)
    edge = np.array([-2, -1, 0, 1, N - 2, N - 1, N, N + 1], np.int64)
    X[: k // 4] = rng.choice(edge, k // 4)
    Y[k // 8: k // 4 + k // 8] = rng.choice(edge, k // 4)
    return X, Y


@pytest.mark.parametrize("conn,table,ntrees", [(fco.CONN_SQUARE, table_square, 1),
                                               (fco.CONN_PERIODIC, table_periodic, 1),
                                               (fco.CONN_PILLOW, table_pillow, 2),
                                               (fco.CONN_SPHERE, table_cube, 6)])
def test_tables_reproduce_the_built_in_maps(conn, table, ntrees):
    lib = fco.oracle_lib()
    tab = table()
    rng = np.random.default_rng(7 + conn)
    kinds = {"inside": 0, "side": 0, "corner image": 0, "corner none": 0}
    for t in range(ntrees):
        X, Y = _points(rng, 4000)
        for x, y in zip(X.tolist(), Y.tolist()):
            got, want = _tmap(lib, tab, t, x, y), _omap(lib, conn, t, x, y)
            assert got == want, (t, x, y, got, want)
            out = (x < 0 or x >= N) + (y < 0 or y >= N)
            key = ["inside", "side", "corner image" if got[0] >= 0 else "corner none"][out]
            kinds[key] += 1
    assert kinds["inside"] and kinds["side"]
    if conn == fco.CONN_SQUARE:
        assert kinds["corner image"] == 0
    elif conn == fco.CONN_SPHERE:
        assert kinds["corner image"] == 0 and kinds["corner none"] > 0     # three faces meet
    else:
        assert kinds["corner none"] == 0 and kinds["corner image"] > 0


def test_pillow_corner_is_the_reflected_own_corner():
    lib = fco.oracle_lib()
    tab = table_pillow()
    for t in (0, 1):
        for dx, dy in ((1, 1), (3, 7), (N // 4, 5)):
            assert _tmap(lib, tab, t, N - 1 + dx, N - 1 + dy) == (t, N - dx, N - dy)
            assert _tmap(lib, tab, t, -dx, -dy) == (t, dx - 1, dy - 1)


def test_two_by_two_brick_is_one_square_a_level_finer():
    """four trees (tree = 2 ty + tx, Morton order of the quadrants), walls
    outside: a point of tree t maps as the point (tx N + X, ty N + Y) of a
    square twice as wide does, interior corner (four trees) included"""
    lib = fco.oracle_lib()
    e = {}
    for ty in (0, 1):
        for tx in (0, 1):
            t = 2 * ty + tx
            if tx == 0: e[(t, 1)] = (t + 1, 0, 0)
            if tx == 1: e[(t, 0)] = (t - 1, 1, 0)
            if ty == 0: e[(t, 3)] = (t + 2, 2, 0)
            if ty == 1: e[(t, 2)] = (t - 2, 3, 0)
    tab = _table(e, 4)
    rng = np.random.default_rng(3)
    seen_diag = 0
    for t in range(4):
        tx, ty = t % 2, t // 2
        X, Y = _points(rng, 3000)
        for x, y in zip(X.tolist(), Y.tolist()):
            gx, gy = tx * N + x, ty * N + y
            if 0 <= gx < 2 * N and 0 <= gy < 2 * N:
                want = (2 * (gy // N) + gx // N, gx % N, gy % N)
            else:
                want = (-1, 0, 0)
            got = _tmap(lib, tab, t, x, y)
            assert got == want, (t, x, y, got, want)
            if got[0] >= 0 and (x < 0 or x >= N) and (y < 0 or y >= N):
                seen_diag += 1
    assert seen_diag > 0


# ---------------------------------------------------------------- forests
def table_brick():
    """a 2 x 2 brick of trees t = tx + 2 ty, walls around it"""
    e = {}
    for ty in range(2):
        for tx in range(2):
            t = tx + 2 * ty
            if tx == 0:
                e[(t, 1)] = (t + 1, 0, 0)
            else:
                e[(t, 0)] = (t - 1, 1, 0)
            if ty == 0:
                e[(t, 3)] = (t + 2, 2, 0)
            else:
                e[(t, 2)] = (t - 2, 3, 0)
    return _table(e, 4)


def _oracle(conn, lmin=0, lmax=6, table=None):
    from oracle.fco import Oracle, OracleParams
    o = Oracle(OracleParams(conn=conn, equation=fco.EQ_ADV, m=8, min_level=lmin, max_level=lmax))
    if table is not None:
        o.set_connectivity(table)
    return o


def _refine_some(o, seed, rounds=2):
    """random refinement flags, then 2:1 balance"""
    rng = np.random.default_rng(seed)
    for _ in range(rounds):
        o.adapt_topology((rng.random(o.n) < 0.3).astype(np.int8))
    o.balance()


@pytest.mark.parametrize("name,conn,table", [("square", fco.CONN_SQUARE, table_square),
                                             ("periodic", fco.CONN_PERIODIC, table_periodic),
                                             ("pillow", fco.CONN_PILLOW, table_pillow),
                                             ("cube", fco.CONN_SPHERE, table_cube)])
@pytest.mark.parametrize("seed", [0, 1])
def test_table_forest_equals_builtin_forest(name, conn, table, seed):
    """the forest of a table connectivity (uniform, randomly refined, 2:1
    balanced) has the built-in connectivity's leaves and neighbour table bit
    for bit; orientation codes agree on the spheres (both encode every
    crossing of a tree side), while the square's wrap and walls carry none
    built in and the identity (1) in a table"""
    a = _oracle(conn)
    b = _oracle(fco.CONN_TABLE, table=table())
    for lev in (0, 2):
        a.uniform(lev)
        b.uniform(lev)
        for x, y in zip(a.leaves(), b.leaves()):
            assert np.array_equal(x, y)
    _refine_some(a, seed)
    leaves = a.leaves()
    b.set_leaves(*leaves)
    assert b.is_balanced()
    for x, y in zip(leaves, b.leaves()):
        assert np.array_equal(x, y)
    na, nb = a.neighbors(), b.neighbors()
    assert np.array_equal(na[..., :3], nb[..., :3])
    if conn in (fco.CONN_SPHERE, fco.CONN_PILLOW):
        assert np.array_equal(na[..., 3], nb[..., 3])
    else:
        assert np.all(na[..., 3] == 0)
        assert set(np.unique(nb[..., 3]).tolist()) <= {0, 1}
        assert (nb[..., 3] == 1).any() == (name == "periodic")


def _brick_to_square(leaves):
    """brick leaf (t, l, x, y) as the leaf of the unit square one level finer"""
    t, l, x, y = [np.asarray(a, np.int64) for a in leaves]
    tx, ty = t % 2, t // 2
    return (np.zeros_like(t), l + 1, x + (tx << l), y + (ty << l))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brick_forest_is_the_square_one_level_finer(seed):
    """a 2 x 2 brick: the same leaves in the same order as the unit square one
    level finer (tree t = tx + 2 ty covers the quadrant that the square's
    Morton order visits t-th), the same neighbours; balancing either gives
    the same forest; orientation codes mark the crossings between trees"""
    br = _oracle(fco.CONN_TABLE, table=table_brick())
    sq = _oracle(fco.CONN_SQUARE, lmin=1, lmax=7)
    rng = np.random.default_rng(seed)
    br.uniform(1)
    for _ in range(3):                            # unbalanced refinement
        f = np.zeros(br.n, np.int8)
        f[rng.choice(br.n, max(1, br.n // 6), replace=False)] = 1
        br.adapt_topology(f)
    bl = br.leaves()
    sq.set_leaves(*_brick_to_square(bl))
    for x, y in zip(_brick_to_square(bl), sq.leaves()):
        assert np.array_equal(x, y)
    br.balance()
    sq.balance()
    for x, y in zip(_brick_to_square(br.leaves()), sq.leaves()):
        assert np.array_equal(x, y)
    nb, ns = br.neighbors(), sq.neighbors()
    assert np.array_equal(nb[..., :3], ns[..., :3])
    t = br.leaves()[0]
    tr = np.where(nb[..., 1] >= 0, t[np.maximum(nb[..., 1], 0)], -1)
    cross = (nb[..., 0] != fco.NB_NONE) & (tr != t[:, None])
    assert np.all(nb[..., 3][cross] == 1) and np.all(nb[..., 3][~cross] == 0)
    assert cross.any()


def test_table_connectivity_refuses_fields_and_bad_tables():
    from oracle.fco import OracleError
    o = _oracle(fco.CONN_TABLE)
    bad = table_brick()
    bad[0, 1] = (7, 0, 0)                          # a tree that does not exist
    with pytest.raises(OracleError):
        o.set_connectivity(bad)
    o.set_connectivity(table_brick())
    with pytest.raises(OracleError):
        o.init_fields(fco.INIT_ADV_SINE, [1.0, 0.5, 1.0, 1.0])
