"""P12: the oracle's adaptive runs against the paper's printed adaptive
errors, plus an exactness pin of the regrid transfer.

* Table 1 (Section 4.1), right: tanh disc, a = (1, 0.5), CFL 0.6, levels 3-5,
  a patch refined where q_max - q_min > 0.001 (the paper's criterion), with
  subcycling and the conservative fix, error at t = 1 against the exact
  translate.  Printed 8.467527e-06; the oracle gives 8.478e-06 (+0.1 %).
* Table 3 (Section 4.3): smooth swirl, levels 3-4, with subcycling (printed
  5.758274e-06) and with global time stepping (5.724930e-06).  The paper does
  not state the swirl's refinement criterion; the same range criterion as
  Section 4.1 (refine above 0.001) is used, CFL 0.5 as for the uniform rows.
  The oracle gives 5.660e-06 both ways (-1.7 % and -1.1 %; its uniform level
  4 is -1.1 % off the printed 5.722927e-06).
Both runs regrid once per coarse step (coarsen a family whose four
indicators are below half the threshold) from an initial forest built by
the same criterion on the exact initial data.

The regrid pin: biquadratic data are reproduced exactly by the coarse ->
fine interpolation and by vertex copies, so after any regrid and ghost
exchange every average and point value of every leaf -- the nodes on a
leaf's right and top faces included, which a leaf owns where its neighbour
there is coarser -- equals the function's exact value.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import synth as S
from oracle.amr import OracleForest, new_leaves

G = S.G
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def _sorted(leaves):
    return sorted(leaves, key=lambda t: (t[0], t[2], t[1]))


def _initial(n, lmin, lmax, f, thr, dt0, field=None, a=0.0, b=0.0):
    """Uniform level lmin, then tag / refine the exact initial data once per
    level (the initial forest of an adaptive run)."""
    leaves = [(lmin, x, y) for y in range(1 << lmin) for x in range(1 << lmin)]
    for _ in range(lmax - lmin):
        F = OracleForest(O.ADVECTION, n, 1, lmax, leaves, (0, 0), (1, 1), dt0, a, b,
                         state=S.forest_state(n, 1, 1, lmax, leaves, [f], nq=4))
        tags, _ = F.tags(0, 0, thr, thr / 2)
        new = new_leaves(F.leaves, np.maximum(tags, 0), 1, lmin, lmax)
        if new == F.leaves:
            break
        leaves = new
    leaves = _sorted(leaves)
    F = OracleForest(O.ADVECTION, n, 1, lmax, leaves, (0, 0), (1, 1), dt0, a, b,
                     state=S.forest_state(n, 1, 1, lmax, leaves, [f], nq=4), field=field)
    F.sync_fill((1 << (lmax + 1)) - 1)
    return F


def _l1(F, exact, n):
    """Sum over leaves of |Q - Q_exact| dx dy over cell averages (reading 13)."""
    lat = S.Layout(n, 1).lattice(F.state.reshape(len(F.leaves), 1, 4, -1))
    err = 0.0
    for p, (l, ix, iy) in enumerate(F.leaves):
        w = 1.0 / (1 << l)
        h = w / n
        X, Y = np.meshgrid(ix * w + (np.arange(n) + 0.5) * h, iy * w + (np.arange(n) + 0.5) * h)
        err += np.abs(lat[p, 0, S.AVG, G:G + n, G:G + n] - S.cell_averages(exact, X, Y, h, h, 4)).sum() * h * h
    return err


def _adaptive_run(n, lmin, lmax, f, cfl, thr, subcycle=True, field=None, a=0.0, b=0.0):
    ns, dtc = S.steps_to(1.0, cfl * (1.0 / n) / 2 ** lmin)
    F = _initial(n, lmin, lmax, f, thr, dtc * 2 ** lmin, field, a, b)
    for k in range(ns):
        if k > 0:
            tags, _ = F.tags(0, 0, thr, thr / 2)
            F.regrid(tags, lmin)
        F.coarse_step(subcycle=subcycle)
    assert abs(F.time - 1.0) < 1e-12 and F.levels[-1] == lmax
    return F


def test_p12_table1_dynamic_refinement_levels_3_5():
    printed = GOLD["table1_advection_amr"]["dynamic_3_5"]
    thr = GOLD["table1_advection_amr"]["dynamic_threshold"]
    n = 16
    F = _adaptive_run(n, 3, 5, S.tanh_disc, 0.6, thr, a=1.0, b=0.5)
    err = _l1(F, S.translated(S.tanh_disc, 1.0, 0.5, 1.0), n)
    assert abs(err / printed - 1.0) < 0.01, (err, printed)


@pytest.mark.parametrize("subcycle", [True, False])
def test_p12_table3_swirl_levels_3_4(subcycle):
    printed = GOLD["table3_swirl_amr"]["subcycled_3_4" if subcycle else "global_3_4"]
    n = 16
    F = _adaptive_run(n, 3, 4, S.swirl_gaussians, 0.5, 1e-3, subcycle=subcycle, field=O.SWIRL)
    err = _l1(F, S.swirl_gaussians, n)   # the swirl returns the data to their start at t = 1
    assert abs(err / printed - 1.0) < 0.02, (err, printed)


def _exact_entries(f, n, leaf):
    """Exact averages and point values of the lattice lines [0, n] of a leaf
    of the unit square."""
    l, ix, iy = leaf
    w = 1.0 / (1 << l)
    h = w / n
    I = np.arange(n + 1)
    out = {}
    for k in (S.CORNER, S.XMID, S.YMID):
        xs = ix * w + I * h + (0.5 * h if k == S.YMID else 0.0)
        ys = iy * w + I * h + (0.5 * h if k == S.XMID else 0.0)
        X, Y = np.meshgrid(xs, ys)
        out[k] = f(X, Y)
    X, Y = np.meshgrid(ix * w + (I[:n] + 0.5) * h, iy * w + (I[:n] + 0.5) * h)
    out[S.AVG] = S.cell_averages(f, X, Y, h, h, 3)
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_p8_regrid_and_exchange_exact_for_biquadratics(seed):
    """Random refine / coarsen tags on a forest of levels 2-4 holding a
    biquadratic: after each regrid and exchange, every cell average and every
    point value on the cells' boundaries (node lines 0 .. n of each leaf) is
    exact to round-off.  Checked on the leaves in [1/4, 3/4]^2: the data are
    not periodic, so the reconstructions of cells on the periodic seam (and
    whatever is interpolated from them) are not the biquadratic."""
    f = lambda x, y: 0.3 + x - 2 * y + 1.5 * x * y + x * x - 0.5 * y * y + x * x * y - 2 * x * y * y \
        + 3 * x * x * y * y
    n, lmin, lmax = 8, 2, 4
    rng = np.random.default_rng(seed)
    leaves = _sorted(S.balanced_forest(1, lmin, 3, lambda l, x, y: (x + y) % 3 == 0))
    F = OracleForest(O.ADVECTION, n, 1, lmax, leaves, (0, 0), (1, 1), 0.01, 1.0, 0.5,
                     state=S.forest_state(n, 1, 1, lmax, leaves, [f], nq=3))
    F.sync_fill((1 << (lmax + 1)) - 1)
    changed = checked = 0
    for _ in range(4):
        tags = rng.choice(np.array([-1, 0, 1], np.int8), size=len(F.leaves), p=[0.45, 0.25, 0.3])
        changed += bool(F.regrid(tags, lmin))
        lat = S.Layout(n, 1).lattice(F.state.reshape(len(F.leaves), 1, 4, -1))
        for p, leaf in enumerate(F.leaves):
            l, ix, iy = leaf
            q = 1 << (l - 2)   # leaves per quarter of the domain side
            if not (q <= ix < 3 * q and q <= iy < 3 * q):
                continue
            ex = _exact_entries(f, n, leaf)
            for k, e in ex.items():
                ni = n + 1 if k in (S.CORNER, S.XMID) else n
                nj = n + 1 if k in (S.CORNER, S.YMID) else n
                d = np.abs(lat[p, 0, k, G:G + nj, G:G + ni] - e[:nj, :ni]).max()
                assert d < 1e-12, (leaf, k, d)
            checked += 1
    assert changed >= 3 and checked > 20
