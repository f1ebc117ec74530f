"""Pins of the oracle's adaptive-mesh pieces (Section 3 of the paper).

P7  conservation to round-off across coarse-fine faces with subcycling and
    the conservative fix;
P8  coarse -> fine interpolation conserves and is exact for biquadratics;
    fine -> coarse averaging of an interpolation is the identity;
P9  a forest of same-level leaves reproduces the uniform run bit for bit;
P12 constants survive subcycling; third-order convergence on adaptive grids.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth as S
from oracle.amr import OracleForest, new_leaves

G = S.G


def _diag(l, ix, iy):
    return ix == iy


def _forest(eq, n, lmin, lmax, funcs, cfl, a=1.0, b=0.5, c=1.0, lo=(0.0, 0.0), hi=(1.0, 1.0), refine=_diag,
            nq=3):
    leaves = S.balanced_forest(1, lmin, lmax, refine)
    nc = 1 if eq == O.ADVECTION else 3
    st = S.forest_state(n, nc, 1, lmax, leaves, funcs, lo, hi, nq=nq)
    dx0 = (hi[0] - lo[0]) / n
    speed = max(abs(a), abs(b)) if eq == O.ADVECTION else c
    dt0 = cfl * dx0 / speed
    F = OracleForest(eq, n, 1, lmax, leaves, lo, hi, dt0, a, b, c, state=st)
    F.sync_fill((1 << (lmax + 1)) - 1)
    return F


def test_p9_same_level_forest_equals_uniform_run():
    n, l = 8, 2
    leaves = S.balanced_forest(1, l, l, lambda *a: False)
    grid = S.UniformGrid(S.Layout(n, 3), 4, 4)
    st = S.pack_owned(grid, S.random_owned(grid, 3))
    dt = 0.4 * grid.dx
    F = OracleForest(O.ACOUSTICS, n, 1, l, leaves, (0, 0), (1, 1), dt * 4, state=np.nan_to_num(st))
    F.sync_fill((1 << (l + 1)) - 1)
    for _ in range(3):
        F.coarse_step()
    ref = O.run_uniform(O.cfg(1, n, grid.dx, grid.dy, dt, c=1.0), 4, 4, 3, st)
    assert np.array_equal(S.unpack_owned(grid, F.state.reshape(st.shape)), S.unpack_owned(grid, ref))


@pytest.mark.parametrize("eq", [O.ADVECTION, O.ACOUSTICS])
def test_p7_mass_conserved_across_coarse_fine_faces(eq):
    """Section 3.2: with the Berger-Colella fix the total of every component
    is conserved to round-off on a refined periodic grid with subcycling."""
    funcs = [S.sinsin_plus_gaussian] if eq == O.ADVECTION else S.pulse_plus_vortex()
    F = _forest(eq, 8, 2, 3, funcs, 0.6 if eq == O.ADVECTION else 0.4)
    m0 = F.mass()
    for _ in range(3):
        F.coarse_step()
    m1 = F.mass()
    scale = max(1.0, np.abs(m0).max())
    assert np.abs(m1 - m0).max() < 1e-14 * scale * 10


def test_p7_without_reflux_mass_is_not_conserved():
    """The same run with the fix disabled loses conservation, so the pin above
    really exercises the correction."""
    F = _forest(O.ADVECTION, 8, 2, 3, [S.sinsin_plus_gaussian], 0.6)
    F.reflux = lambda mask: None
    m0 = F.mass()
    for _ in range(2):
        F.coarse_step()
    assert abs(F.mass()[0] - m0[0]) > 1e-10


def test_p12_constants_survive_subcycling():
    """Section 4.3: constant states are kept on refined grids with subcycling
    (the paper reports 1e-13 for its variable-velocity case)."""
    F = _forest(O.ACOUSTICS, 8, 2, 3, [lambda x, y: 1 + 0 * x, lambda x, y: 2 + 0 * x,
                                       lambda x, y: -1 + 0 * x], 0.4)
    for _ in range(3):
        F.coarse_step()
    lat = S.Layout(8, 3).lattice(F.state.reshape(len(F.leaves), 3, 4, -1))
    for k, v in enumerate([1.0, 2.0, -1.0]):
        assert np.abs(lat[:, k, :, G:G + 8, G:G + 8] - v).max() < 1e-13


def test_p8_interpolation_exact_for_biquadratics_and_conservative():
    """Section 3.1, coarse -> fine: the children's point values are the
    parent's reconstruction, their averages come from Simpson's rule which is
    exact for it; for biquadratic data everything is exact, and for any data
    the four children's averages sum to four times the parent's."""
    n = 8
    f = lambda x, y: 1 + x - 2 * y + 3 * x * y + x * x - y * y + 2 * x * x * y - x * y * y + 4 * x * x * y * y
    leaves = S.balanced_forest(1, 1, 1, lambda *a: False)
    st = S.forest_state(n, 1, 1, 2, leaves, [f], nq=4)
    F = OracleForest(O.ADVECTION, n, 1, 2, leaves, (0, 0), (1, 1), 0.1, 1.0, 0.0, state=st)
    tags = np.array([1, 0, 0, 0], np.int8)
    F.regrid(tags, 1)
    assert len(F.leaves) == 7
    kids = [k for k, (l, _, _) in enumerate(F.leaves) if l == 2]
    exact = S.forest_state(n, 1, 1, 2, F.leaves, [f], nq=4)
    lat, E = S.Layout(n, 1).lattice(F.state.reshape(len(F.leaves), 1, 4, -1)), \
        S.Layout(n, 1).lattice(exact.reshape(len(F.leaves), 1, 4, -1))
    for k in kids:
        assert np.abs(lat[k, 0, :, G:G + n, G:G + n] - E[k, 0, :, G:G + n, G:G + n]).max() < 1e-13
    # conservation for arbitrary data
    rnd = S.random_state(S.Layout(n, 1), 4, seed=5)
    F2 = OracleForest(O.ADVECTION, n, 1, 2, leaves, (0, 0), (1, 1), 0.1, 1.0, 0.0, state=rnd)
    F2.sync_fill(0b111)
    parent = S.Layout(n, 1).lattice(F2.state.reshape(4, 1, 4, -1))[0, 0, S.AVG, G:G + n, G:G + n].sum()
    m0 = F2.mass()
    F2.regrid(tags, 1)
    assert abs(F2.mass()[0] - m0[0]) < 1e-15 * abs(parent) * 10 + 1e-16
    # fine -> coarse of the interpolation restores the parent's averages
    before = S.Layout(n, 1).lattice(F2.state.reshape(len(F2.leaves), 1, 4, -1)).copy()
    F3 = OracleForest(O.ADVECTION, n, 1, 2, leaves, (0, 0), (1, 1), 0.1, 1.0, 0.0, state=rnd)
    F3.sync_fill(0b111)
    orig = S.Layout(n, 1).lattice(F3.state.reshape(4, 1, 4, -1))[0, 0].copy()
    F3.regrid(tags, 1)
    F3.regrid(-np.ones(len(F3.leaves), np.int8), 1)
    back = S.Layout(n, 1).lattice(F3.state.reshape(len(F3.leaves), 1, 4, -1))
    k0 = F3.leaves.index((1, 0, 0))
    assert np.abs(back[k0, 0, S.AVG, G:G + n, G:G + n] - orig[S.AVG, G:G + n, G:G + n]).max() < 1e-14
    # point values: a node of the parent is a vertex of a child and is copied back
    assert np.abs(back[k0, 0, S.CORNER, G:G + n, G:G + n] - orig[S.CORNER, G:G + n, G:G + n]).max() < 1e-14
    del before


def test_regrid_balance_and_family_coarsening():
    """Refinement of one leaf next to a coarse leaf forces 2:1 balance; a
    family coarsens only when all four members ask for it."""
    leaves = S.balanced_forest(1, 1, 1, lambda *a: False)
    new = new_leaves(leaves, np.array([1, 0, 0, 0], np.int8), 1, 1, 3)
    assert len(new) == 7
    new2 = new_leaves(new, np.array([1 if l == 2 and x == 0 and y == 0 else 0 for (l, x, y) in new], np.int8),
                      1, 1, 3)
    # a level-3 leaf next to level-1 leaves would break the balance: they split
    lv = [l for l, _, _ in new2]
    assert max(lv) == 3 and min(lv) >= 1
    for (l, x, y) in new2:
        assert l >= 1
    tags = np.array([-1 if l == 2 else 0 for (l, _, _) in new], np.int8)
    assert new_leaves(new, tags, 1, 1, 3) == leaves
    tags[-1] = 0 if new[-1][0] == 2 else tags[-1]
    part = [(-1 if (l == 2 and not (x == 1 and y == 1)) else 0) for (l, x, y) in new]
    assert new_leaves(new, np.array(part, np.int8), 1, 1, 3) == new


def test_p12_advection_third_order_on_refined_grids():
    """Section 4.1 (Table 1, diagonal refinement): the error on refined
    grids with subcycling decreases at third order."""
    f = lambda x, y: np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    errs = []
    for (lmin, lmax) in [(2, 3), (3, 4)]:
        F = _forest(O.ADVECTION, 8, lmin, lmax, [f], 0.6, nq=5)
        lpres = min(F.levels)
        ns, dtc = S.steps_to(1.0, 0.6 * (1.0 / 8) / 2 ** lpres)
        F.dt0 = dtc * 2 ** lpres
        for _ in range(ns):
            F.coarse_step()
        ex = S.translated(f, 1.0, 0.5, 1.0)
        lat = S.Layout(8, 1).lattice(F.state.reshape(len(F.leaves), 1, 4, -1))
        err = 0.0
        for p, (l, ix, iy) in enumerate(F.leaves):
            w = 1.0 / (1 << l)
            h = w / 8
            xc = ix * w + (np.arange(8) + 0.5) * h
            yc = iy * w + (np.arange(8) + 0.5) * h
            X, Y = np.meshgrid(xc, yc)
            err += np.abs(lat[p, 0, S.AVG, G:G + 8, G:G + 8] - S.cell_averages(ex, X, Y, h, h, 5)).sum() * h * h
        errs.append(err)
    eoc = math.log2(errs[0] / errs[1])
    assert 2.5 < eoc < 3.6, (errs, eoc)
