"""Pins of the oracle's forest (Sec. 2, Sec. 4) against brute force.

* leaf order equals the (tree, Morton key) order computed here independently;
* 2:1 balance equals an O(N^2) pairwise balance (the coarsest balanced
  refinement is unique, so any correct algorithm gives the same leaves);
* the neighbour table equals an O(N) point-containment scan per probe;
* the cubed sphere's neighbour relation is mutual with inverse orientations,
  and exactly three trees meet at each of the eight cube corners;
* the paper's printed counts (tests/golden/paper_facts.txt) hold.
"""
import os

import numpy as np
import pytest

from oracle import fco
from oracle.fco import Oracle, OracleParams
from fc_inputs import random_forest_flags

L = 30
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def morton_py(X, Y):
    k = 0
    for b in range(L):
        k |= ((X >> b) & 1) << (2 * b)
        k |= ((Y >> b) & 1) << (2 * b + 1)
    return k


def random_unbalanced(seed, max_level=5, conn=fco.CONN_SQUARE):
    """Random forest built by random splits (not balanced)."""
    rng = np.random.default_rng(seed)
    ntrees = 6 if conn == fco.CONN_SPHERE else 1
    leaves = [(t, 0, 0, 0) for t in range(ntrees)]
    for _ in range(max_level):
        new = []
        for (t, l, x, y) in leaves:
            if l < max_level and rng.random() < 0.35:
                new += [(t, l + 1, 2 * x + (c & 1), 2 * y + (c >> 1)) for c in range(4)]
            else:
                new.append((t, l, x, y))
        leaves = new
    return leaves


def boxes(leaves, R):
    """(tree, x0, x1, y0, y1) in units of 2^-R"""
    out = []
    for (t, l, x, y) in leaves:
        s = 1 << (R - l)
        out.append((t, x * s, (x + 1) * s, y * s, (y + 1) * s))
    return out


def touching(a, b, R, periodic):
    if a[0] != b[0]:
        return False
    N = 1 << R
    shifts = [(dx, dy) for dx in (-N, 0, N) for dy in (-N, 0, N)] if periodic else [(0, 0)]
    for dx, dy in shifts:
        bx0, bx1, by0, by1 = b[1] + dx, b[2] + dx, b[3] + dy, b[4] + dy
        if a[1] <= bx1 and bx0 <= a[2] and a[3] <= by1 and by0 <= a[4]:
            overlap = min(a[2], bx1) > max(a[1], bx0) and min(a[4], by1) > max(a[3], by0)
            if not overlap:
                return True
    return False


def brute_balance(leaves, periodic=False):
    leaves = set(leaves)
    R = 12
    while True:
        lst = sorted(leaves)
        bx = boxes(lst, R)
        split = None
        for i in range(len(lst)):
            for j in range(len(lst)):
                if lst[i][1] < lst[j][1] - 1 and touching(bx[i], bx[j], R, periodic):
                    split = lst[i]
                    break
            if split:
                break
        if not split:
            return sorted(leaves)
        t, l, x, y = split
        leaves.remove(split)
        leaves |= {(t, l + 1, 2 * x + (c & 1), 2 * y + (c >> 1)) for c in range(4)}


def oracle_with(leaves, conn=fco.CONN_SQUARE, m=8, lmin=0, lmax=10):
    o = Oracle(OracleParams(conn=conn, m=m, min_level=lmin, max_level=lmax))
    a = np.array(leaves, dtype=np.int32)
    o.set_leaves(a[:, 0], a[:, 1], a[:, 2], a[:, 3])
    return o


def leaf_list(o):
    t, l, x, y = o.leaves()
    return list(zip(t.tolist(), l.tolist(), x.tolist(), y.tolist()))


@pytest.mark.parametrize("seed", range(6))
def test_order_is_morton(seed):
    lv = random_unbalanced(seed)
    o = oracle_with(lv)
    got = leaf_list(o)
    keys = [(t, morton_py(x << (L - l), y << (L - l))) for (t, l, x, y) in got]
    assert keys == sorted(keys)
    assert sorted(got) == sorted(lv)


@pytest.mark.parametrize("seed,periodic", [(s, p) for s in range(8) for p in (False, True)])
def test_balance_matches_pairwise_bruteforce(seed, periodic):
    lv = random_unbalanced(100 + seed, max_level=5)
    conn = fco.CONN_PERIODIC if periodic else fco.CONN_SQUARE
    o = oracle_with(lv, conn=conn)
    o.balance()
    assert o.is_balanced()
    assert sorted(leaf_list(o)) == brute_balance(lv, periodic)


def scan_leaf(lst, R, t, X2, Y2):
    """leaf whose box contains the doubled-coordinate point (X2, Y2), by scan"""
    for k, (tt, l, x, y) in enumerate(lst):
        if tt != t:
            continue
        s = 2 << (R - l)
        if x * s < X2 < (x + 1) * s and y * s < Y2 < (y + 1) * s:
            return k
    return -1


@pytest.mark.parametrize("seed,periodic", [(s, p) for s in range(5) for p in (False, True)])
def test_neighbor_table_matches_scan(seed, periodic):
    conn = fco.CONN_PERIODIC if periodic else fco.CONN_SQUARE
    o = oracle_with(random_unbalanced(200 + seed, max_level=5), conn=conn)
    o.balance()
    lst = leaf_list(o)
    tab = o.neighbors()
    R = 8
    N2 = 2 << R
    for k, (t, l, x, y) in enumerate(lst):
        s2 = 2 << (R - l)
        x0, x1, y0, y1 = x * s2, (x + 1) * s2, y * s2, (y + 1) * s2
        for d in range(8):
            if d < 4:
                # every fine-resolution point just outside the face
                if d < 2:
                    xo = x0 - 1 if d == 0 else x1 + 1
                    pts = [(xo, yy) for yy in range(y0 + 1, y1, 2)]
                else:
                    yo = y0 - 1 if d == 2 else y1 + 1
                    pts = [(xx, yo) for xx in range(x0 + 1, x1, 2)]
            else:
                xo = x0 - 1 if d in (4, 6) else x1 + 1
                yo = y0 - 1 if d in (4, 5) else y1 + 1
                pts = [(xo, yo)]
            found = []
            for (px, py) in pts:
                if periodic:
                    px, py = px % N2, py % N2
                elif not (0 < px < N2 and 0 < py < N2):
                    continue
                j = scan_leaf(lst, R, t, px, py)
                if j not in found:
                    found.append(j)
            e = tab[k, d]
            if not found:
                assert e[0] == fco.NB_NONE
                continue
            dl = lst[found[0]][1] - l
            if dl == 0:
                assert e[0] == fco.NB_SAME and found == [e[1]]
            elif dl == -1:
                assert e[0] == fco.NB_COARSER and found == [e[1]]
            else:
                assert dl == 1 and e[0] == fco.NB_FINER
                if d < 4:
                    assert found == [e[1], e[2]]
                else:
                    assert found == [e[1]]


def test_adapt_rules():
    """refine wins; families coarsen only when all four are flagged; balance after."""
    o = Oracle(OracleParams(m=8, min_level=1, max_level=5))
    o.uniform(3)
    n = o.n
    for seed in range(5):
        o.uniform(3)
        f = random_forest_flags(o.n, seed)
        before = leaf_list(o)
        o.adapt_topology(f)
        after = set(leaf_list(o))
        assert o.is_balanced()
        # every refined leaf's children exist (or deeper)
        for (t, l, x, y), fl in zip(before, f):
            if fl == 1:
                assert (t, l, x, y) not in after
        # a family is coarsened only if all four flagged -1
        for (t, l, x, y) in after:
            if l == 2:
                kids = [(t, 3, 2 * x + (c & 1), 2 * y + (c >> 1)) for c in range(4)]
                idx = [before.index(kk) for kk in kids]
                assert all(f[i] == -1 for i in idx)
    assert n == 64


def test_cubed_sphere_connectivity():
    lev = 2
    o = Oracle(OracleParams(conn=fco.CONN_SPHERE, equation=fco.EQ_ADV, m=8, min_level=lev, max_level=lev))
    assert o.n == 6 * 4 ** lev
    tab = o.neighbors()
    lst = leaf_list(o)
    none_corners = 0
    for k in range(o.n):
        for d in range(4):
            e = tab[k, d]
            assert e[0] == fco.NB_SAME
            j = e[1]
            back = [dd for dd in range(4) if tab[j, dd, 1] == k]
            assert len(back) == 1
            # orientation codes of the two directions are inverse maps
            o1, o2 = e[3], tab[j, back[0], 3]
            assert (o1 == 0) == (o2 == 0) == (lst[k][0] == lst[j][0])
            if o1:
                M1 = orient_matrix(o1)
                M2 = orient_matrix(o2)
                assert np.array_equal(M2 @ M1, np.eye(2, dtype=int))
        for d in range(4, 8):
            if tab[k, d, 0] == fco.NB_NONE:
                none_corners += 1
    assert none_corners == 24          # 8 cube corners x 3 leaves


def orient_matrix(code):
    c = code - 1
    swap, r0, r1 = (c >> 2) & 1, (c >> 1) & 1, c & 1
    s0, s1 = (-1 if r0 else 1), (-1 if r1 else 1)
    if not swap:
        return np.array([[s0, 0], [0, s1]])
    return np.array([[0, s0], [s1, 0]])


def test_paper_facts():
    """Counts printed in the paper (see the citations in the fixture)."""
    facts = {}
    with open(os.path.join(GOLDEN, "paper_facts.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split("=")
                facts[k.strip()] = [int(t) for t in v.split(",")]
    # Fig. 3 caption: 2^(2 l) patches at level l (one quadtree)
    for lev in facts["uniform_levels"]:
        o = Oracle(OracleParams(m=8, min_level=lev, max_level=lev))
        assert o.n == 2 ** (2 * lev)
    # Example 1: m = 8, levels 3 and 6 give 64x64 and 512x512
    m = facts["example1_m"][0]
    for lev, res in zip(facts["example1_levels"], facts["example1_resolution"]):
        o = Oracle(OracleParams(m=m, min_level=lev, max_level=lev))
        assert int(round(np.sqrt(o.n))) * m == res
