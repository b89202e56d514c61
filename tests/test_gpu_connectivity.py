"""Table connectivity on the GPU (Sec. 2: every tree a reference square, the
trees' connectivity given from outside) against the oracle's table forests:
for the tables of the square, the periodic square, the two-tree sphere, the
cubed sphere (written from its face frames alone) and a 2 x 2 brick, the GPU
forest's leaves and neighbour tables (kinds, neighbour ids, orientation code
of every crossing) equal the oracle's bit for bit, uniformly refined and
after 2:1 balancing of random unbalanced forests.  The calls that need
fields refuse such a context."""
import numpy as np
import pytest

from gpu_helpers import fcmod
from oracle import fco
from oracle.fco import Oracle, OracleParams
from test_oracle_connectivity import table_brick, table_cube, table_periodic, table_pillow, table_square

pytestmark = pytest.mark.gpu

TABLES = {"square": table_square, "periodic": table_periodic, "pillow": table_pillow, "cube": table_cube,
          "brick": table_brick}


def _pair(fc, table, lmin=0, lmax=7):
    ctx = fc.Context(conn=fc.FC_CONN_TABLE, equation=fc.FC_EQ_ADV, m=8, min_level=lmin, max_level=lmax, device=0)
    ctx.set_connectivity(table)
    ora = Oracle(OracleParams(conn=fco.CONN_TABLE, equation=fco.EQ_ADV, m=8, min_level=lmin, max_level=lmax))
    ora.set_connectivity(table)
    return ctx, ora


def _same(ctx, ora):
    for a, b in zip(ctx.forest_get_leaves(), ora.leaves()):
        assert np.array_equal(a, b)
    assert np.array_equal(ctx.forest_get_neighbors(), ora.neighbors())


@pytest.mark.parametrize("name", sorted(TABLES))
@pytest.mark.parametrize("level", [0, 1, 3])
def test_table_forest_uniform_bitexact(name, level):
    fc = fcmod()
    ctx, ora = _pair(fc, TABLES[name]())
    ctx.forest_uniform(level)
    ora.uniform(level)
    _same(ctx, ora)


@pytest.mark.parametrize("name", sorted(TABLES))
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_table_forest_balance_bitexact(name, seed):
    """random unbalanced leaves (the oracle's refinement of random flags,
    without balancing) imported into both, then 2:1 balanced by both"""
    fc = fcmod()
    ctx, ora = _pair(fc, TABLES[name]())
    ora.uniform(1)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        f = np.zeros(ora.n, np.int8)
        f[rng.choice(ora.n, max(1, ora.n // 5), replace=False)] = 1
        ora.adapt_topology(f)
    leaves = ora.leaves()
    ctx.forest_set_leaves(*leaves)
    ora.set_leaves(*leaves)
    ctx.forest_balance()
    ora.balance()
    assert ora.is_balanced()
    _same(ctx, ora)
    if name != "square":
        assert (ctx.forest_get_neighbors()[..., 3] > 0).any()     # crossings carry their codes


def test_table_context_refuses_fields_and_bad_tables():
    fc = fcmod()
    ctx = fc.Context(conn=fc.FC_CONN_TABLE, equation=fc.FC_EQ_ADV, m=8, min_level=1, max_level=3, device=0)
    bad = table_brick()
    bad[2, 3] = (3, 5, 0)                          # no side 5
    with pytest.raises(fc.FCError) as ei:
        ctx.set_connectivity(bad)
    assert ei.value.rc == fc.FC_ERR_INVALID_ARG
    ctx.set_connectivity(table_brick())
    assert ctx.n == 16
    with pytest.raises(fc.FCError) as ei:
        ctx.advance(1, 1e-3)
    assert ei.value.rc == fc.FC_ERR_UNIMPLEMENTED
    sq = fc.Context(conn=fc.FC_CONN_SQUARE, m=8, min_level=1, max_level=3, device=0)
    with pytest.raises(fc.FCError):
        sq.set_connectivity(table_brick())
