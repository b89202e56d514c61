"""Pins of the oracle's sub-cycled time stepping in two dimensions (Sec. 4:
each level advances with its own step; the ghost values a level reads from a
coarser neighbour must be time accurate between the coarse level's steps,
Sec. 3).

Invariants (constant states, mass, symmetry) do not see the weight with which
a coarser level's old and new states are blended at an intermediate substep
time, so these pins measure accuracy instead, on a fixed three-level forest
(a block refined once, its centre refined again):

  * smooth advection on the periodic square against the exact solution (the
    translated initial profile): the sub-cycled run is as accurate as the
    run with one global step (within 30 %), at two resolutions, and its error
    falls at second order between them;
  * shallow water with smooth humps on the periodic square against a uniform
    run at the finest level: the sub-cycled run's error is no larger than
    the global-step run's, per field, at two resolutions.

Each pin is then shown to fail on copies of the oracle with a planted
mistake in the blend weight: the weights of old and new swapped, the weight
frozen at the old or at the new state, and the weight taken from the next
finer level's substep clock.
"""
import os

import numpy as np
import pytest

from fc_inputs import humps_params
from oracle import fco
from oracle.fco import Oracle, OracleParams, build_oracle_variant, load_oracle_lib

M = 8
U, V = 1.0, 0.5


def three_level_forest(o, lmin):
    """uniform lmin, the middle half of the square refined once, its middle
    quarter refined again (2:1 balanced by construction)"""
    o.uniform(lmin)
    tr, lv, xs, ys = o.leaves()
    n0 = 1 << lmin
    f = np.zeros(o.n, np.int8)
    f[(xs >= n0 // 4) & (xs < 3 * n0 // 4) & (ys >= n0 // 4) & (ys < 3 * n0 // 4)] = 1
    o.adapt_topology(f)
    tr, lv, xs, ys = o.leaves()
    n1 = 2 * n0
    f = np.zeros(o.n, np.int8)
    f[(lv == lmin + 1) & (xs >= 3 * n1 // 8) & (xs < 5 * n1 // 8) & (ys >= 3 * n1 // 8) & (ys < 5 * n1 // 8)] = 1
    o.adapt_topology(f)
    assert o.is_balanced()
    assert set(o.leaves()[1].tolist()) == {lmin, lmin + 1, lmin + 2}


def _sine(x, y):
    return 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)


def _sample(o, t):
    """point samples of the translated profile at the cell centres, and cell areas"""
    tr, lv, xs, ys = o.leaves()
    q = np.zeros((o.n, 1, M, M))
    area = np.zeros(o.n)
    for k in range(o.n):
        dx = 1.0 / ((1 << lv[k]) * M)
        x = (xs[k] * M + np.arange(M) + 0.5) * dx
        y = (ys[k] * M + np.arange(M) + 0.5) * dx
        q[k, 0] = _sine((x[None, :] - U * t) % 1.0, (y[:, None] - V * t) % 1.0)
        area[k] = dx * dx
    return q, area


def advection_error(lmin, subcycle, lib=None, T=0.25, nu=0.8):
    """L1 error against the exact solution at time T; the step is set by the
    coarsest level under sub-cycling and by the finest with a global step, at
    Courant number nu in both cases"""
    o = Oracle(OracleParams(conn=fco.CONN_PERIODIC, equation=fco.EQ_ADV, m=M, min_level=lmin,
                            max_level=lmin + 2, adv_u=U, adv_v=V, subcycle=subcycle, refluxing=1), lib=lib)
    three_level_forest(o, lmin)
    q0, area = _sample(o, 0.0)
    o.set_fields(q0)
    dx_fine = 1.0 / ((1 << (lmin + 2)) * M)
    dt = nu * (4 * dx_fine if subcycle else dx_fine) / max(abs(U), abs(V))
    steps = int(np.ceil(T / dt))
    o.advance(steps, T / steps)
    qe, _ = _sample(o, T)
    return float((np.abs(o.fields() - qe)[:, 0].sum(axis=(1, 2)) * area).sum())


def advection_pin(lib=None):
    """(errors at lmin 2 and 3 sub-cycled, the same with a global step)"""
    es = [advection_error(l, 1, lib) for l in (2, 3)]
    eg = [advection_error(l, 0) for l in (2, 3)]
    return es, eg


def advection_pin_holds(es, eg):
    return all(s <= 1.3 * g for s, g in zip(es, eg)) and es[0] / es[1] >= 3.5


HUMPS = humps_params(n_humps=6, seed=3, width=(0.08, 0.15))


def _swe_run(lmin, subcycle, lib=None, uniform=False, coarse_steps=6):
    L = lmin + 2
    o = Oracle(OracleParams(conn=fco.CONN_PERIODIC, equation=fco.EQ_SWE, m=M, min_level=lmin, max_level=L,
                            subcycle=subcycle, refluxing=1), lib=lib)
    if uniform:
        o.uniform(L)
    else:
        three_level_forest(o, lmin)
    o.init_fields(fco.INIT_HUMPS, HUMPS)
    dt_coarse = 0.5 * 4.0 / ((1 << L) * M)      # Courant number about 0.8 on the coarsest level
    if subcycle:
        o.advance(coarse_steps, dt_coarse)
    else:
        o.advance(4 * coarse_steps, dt_coarse / 4)
    return o


def _average_onto(ref, o):
    """the uniform run's cells averaged onto o's cells, and o's cell areas"""
    m, F = o.m, o.F
    rt, rl, rx, ry = ref.leaves()
    L = int(rl[0])
    n = (1 << L) * m
    R = np.zeros((F, n, n))
    q = ref.fields()
    for k in range(ref.n):
        R[:, ry[k] * m:(ry[k] + 1) * m, rx[k] * m:(rx[k] + 1) * m] = q[k]
    tr, lv, xs, ys = o.leaves()
    out = np.zeros((o.n, F, m, m))
    area = np.zeros(o.n)
    for k in range(o.n):
        r = 1 << (L - lv[k])
        blk = R[:, ys[k] * m * r:(ys[k] + 1) * m * r, xs[k] * m * r:(xs[k] + 1) * m * r]
        out[k] = blk.reshape(F, m, r, m, r).mean(axis=(2, 4))
        area[k] = (1.0 / ((1 << lv[k]) * m)) ** 2
    return out, area


def swe_pin(lib=None):
    """per resolution: (per-field error sub-cycled, per-field error global)"""
    res = []
    for lmin in (2, 3):
        ref = _swe_run(lmin, 0, uniform=True)
        g = _swe_run(lmin, 0)
        s = _swe_run(lmin, 1, lib)
        qr, area = _average_onto(ref, g)
        err = [(np.abs(x.fields() - qr).sum(axis=(2, 3)) * area[:, None]).sum(axis=0) for x in (s, g)]
        res.append(tuple(err))
    return res


def swe_pin_holds(res):
    return all(np.all(es <= eg) for es, eg in res)


def test_subcycled_advection_matches_exact_solution():
    es, eg = advection_pin()
    assert advection_pin_holds(es, eg), (es, eg)


def test_subcycled_swe_no_less_accurate_than_global_step():
    res = swe_pin()
    assert swe_pin_holds(res), res


_BLEND = "v->alpha[l] = (b == a) ? 1.0 : (double)(T - a) / (double)(b - a);"
PLANTED = {
    "old_new_swapped": [("fco_sim.c", _BLEND,
                         "v->alpha[l] = (b == a) ? 1.0 : 1.0 - (double)(T - a) / (double)(b - a);")],
    "frozen_at_old": [("fco_sim.c", _BLEND, "v->alpha[l] = (b == a) ? 1.0 : 0.0;")],
    "frozen_at_new": [("fco_sim.c", _BLEND, "v->alpha[l] = 1.0;")],
    "finer_level_clock": [("fco_sim.c", "long long a = st->tick_old[l], b = st->tick_new[l];",
                           "int lf = l < FCO_MAXLEVEL ? l + 1 : l;\n"
                           "        long long a = st->tick_old[lf], b = st->tick_new[lf];")],
}


@pytest.mark.parametrize("mistake", sorted(PLANTED))
def test_planted_blend_mistakes_fail_the_pins(mistake, tmp_path):
    lib = load_oracle_lib(build_oracle_variant(os.fspath(tmp_path), PLANTED[mistake]))
    es, eg = advection_pin(lib)
    assert not advection_pin_holds(es, eg), (mistake, es, eg)
    assert not swe_pin_holds(swe_pin(lib)), mistake
