"""Oracle against the paper's printed numbers and measured convergence rates.

P10: third-order experimental order of convergence (EOC) on smooth data.
P11: the uniform-grid L1 errors of Table 1 (advection) and Table 4
(acoustics), stored with their citations in tests/golden/paper_tables.json.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synth as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def _run_adv(f, level, cfl, a=1.0, b=0.5, n=16, T=1.0):
    P = 2 ** level
    grid = S.UniformGrid(S.Layout(n, 1), P, P)
    st = grid.state([f], nq=5)
    ns, dt = S.steps_to(T, S.cfl_dt("advection", cfl, grid.dx, grid.dy, a, b))
    out = O.run_uniform(O.cfg(O.ADVECTION, n, grid.dx, grid.dy, dt, a, b), P, P, ns, st)
    return grid.l1_error(out, 0, S.translated(f, a, b, T))


def _run_lukacova(level, cfl=0.4, n=16):
    P = 2 ** level
    grid = S.UniformGrid(S.Layout(n, 3), P, P, (-1.0, -1.0), (1.0, 1.0))
    st = grid.state(S.lukacova_exact(0.0), nq=5)
    ns, dt = S.steps_to(1.0, S.cfl_dt("acoustics", cfl, grid.dx, grid.dy))
    out = O.run_uniform(O.cfg(O.ACOUSTICS, n, grid.dx, grid.dy, dt, c=1.0), P, P, ns, st)
    ex = S.lukacova_exact(1.0)
    return [grid.l1_error(out, k, ex[k]) for k in range(3)]


def test_p11_table1_level4_advection_error():
    """Section 4.1, Table 1: L1 error 6.461135e-05 on the uniform level-4 grid
    (16 x 16 patches of 16^2 cells, tanh disc, a = (1, 0.5), CFL 0.6, t = 1).
    The oracle reproduces it to well under 1 % (the remaining difference is
    the paper's unstated quadrature of the initial averages)."""
    err = _run_adv(S.tanh_disc, 4, 0.6)
    ref = GOLD["table1_advection_uniform"]["level4_256"]
    assert abs(err / ref - 1.0) < 0.01, (err, ref)


def test_p10_advection_third_order_smooth():
    """Third-order convergence (Section 4, 'third order accurate') of the
    L1 error for smooth data, 32^2 -> 64^2 -> 128^2 cells."""
    f = lambda x, y: np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    e = [_run_adv(f, lv, 0.6, n=16) for lv in (1, 2, 3)]
    eoc = [math.log2(e[k] / e[k + 1]) for k in range(2)]
    assert all(2.8 < r < 3.3 for r in eoc), eoc


def test_p10_p11_acoustics_lukacova():
    """Section 4.5.1, Table 4: the pressure error converges at third order
    (paper: EOC 2.9975) and, read as an area-normalised L1 norm on
    [-1, 1]^2, lies within 15 % of the printed level-2 value 2.231166e-04.
    The printed u,v column is not reproduced by any norm reading tried
    (recorded as a discrepancy), so only its order is checked here."""
    e1 = _run_lukacova(1)
    e2 = _run_lukacova(2)
    eoc_p = math.log2(e1[0] / e2[0])
    assert 2.7 < eoc_p < 3.3, eoc_p
    ref = GOLD["table4_acoustics_uniform"]["level2_p"]
    assert abs((e2[0] / 4.0) / ref - 1.0) < 0.15, (e2[0] / 4.0, ref)
    eoc_u = math.log2(e1[1] / e2[1])
    assert eoc_u > 2.7, eoc_u
    # u and v errors are mirror images of each other (symmetric datum)
    assert abs(e2[1] - e2[2]) < 1e-9 * e2[1]
