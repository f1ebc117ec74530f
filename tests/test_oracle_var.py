"""Pins of the variable-velocity advection oracle (Sections 4.2 and 4.3)
against closed forms, an independent ODE solver, the paper's constant-state
results and Table 3."""
import json
import os

import numpy as np
import pytest

import oracle as O
import synth as S

G = S.G


def _quad(x, y):
    return 1.0 + 0.3 * x - 0.2 * y + 0.5 * x * x - 0.4 * x * y + 0.7 * y * y


def _patch_from(f, n, x0, y0, dx, dy):
    grid = S.UniformGrid(S.Layout(n, 1), 1, 1, (x0, y0), (x0 + n * dx, y0 + n * dy))
    return grid.state([f], nq=3, ghosts=True, periodic=False)[0]


def test_solid_body_nodes_exact_for_quadratic_data():
    """The foot is the node rotated by -pi tau (Eq. characteristics_advtwo)
    and the reconstruction reproduces quadratics, so the evolved point values
    equal q at the rotated node exactly."""
    n, dx = 8, 0.05
    x0, y0 = -0.3, -0.2
    patch = _patch_from(_quad, n, x0, y0, dx, dx)
    tau = 0.02
    vc = O.VarCfg(n, O.SOLID_BODY, dx, dx, tau, x0, y0, 0.0)
    for ty, (ox, oy) in ((O.CORNER, (0, 0)), (O.XMID, (0, 0.5)), (O.YMID, (0.5, 0))):
        for i, j in ((0, 0), (3, 5), (8, 2), (-1, 7)):
            x, y = x0 + (i + ox) * dx, y0 + (j + oy) * dx
            c, s = np.cos(np.pi * tau), np.sin(np.pi * tau)
            exact = _quad(x * c + y * s, -x * s + y * c)
            got = O.node_evolve_var(vc, patch, ty, i, j, tau)
            assert abs(got - exact) < 1e-13, (ty, i, j, got, exact)


def test_swirl_velocity_is_the_centred_difference_of_the_stream_function():
    """Eq. swirlODE: second-order differences of Psi = sin^2 sin^2 cos / pi;
    the error against the exact derivatives falls by 4 when dy halves."""
    x, y, t = 0.31, 0.17, 0.23
    exact_a = -np.sin(np.pi * x) ** 2 * np.sin(2 * np.pi * y) * np.cos(np.pi * t)
    exact_b = np.sin(np.pi * y) ** 2 * np.sin(2 * np.pi * x) * np.cos(np.pi * t)
    errs = []
    for h in (1 / 32, 1 / 64):
        ab = O.var_velocity(O.VarCfg(8, O.SWIRL, h, h, 0.01, 0, 0, 0), x, y, t)
        errs.append(np.hypot(ab[0] - exact_a, ab[1] - exact_b))
    assert 3.8 < errs[0] / errs[1] < 4.2


def test_swirl_foot_is_one_classical_runge_kutta_step():
    """Against an independent high-accuracy integration (scipy) of the
    characteristic ODE backwards from t + tau to t: the local error of one
    classical Runge-Kutta step is O(tau^5), so halving tau divides it by ~32."""
    integrate = pytest.importorskip("scipy.integrate")
    h = 1 / 64
    vc = O.VarCfg(8, O.SWIRL, h, h, 0.01, 0.0, 0.0, 0.2)
    x, y = 0.43, 0.61

    def rhs(t, z):
        return O.var_velocity(vc, z[0], z[1], t)

    errs = []
    for tau in (0.02, 0.01):
        sol = integrate.solve_ivp(rhs, (vc.t + tau, vc.t), [x, y], rtol=1e-13, atol=1e-14, method="DOP853")
        ref = sol.y[:, -1]
        got = O.var_foot(vc, x, y, tau)
        errs.append(np.hypot(*(got - ref)))
    assert errs[0] < 2e-8
    assert 20 < errs[0] / errs[1] < 45, errs


@pytest.mark.parametrize("field", [O.SOLID_BODY, O.SWIRL])
def test_constant_states_are_preserved(field):
    """Remark of Section 4.2 (solid body) and Theorem of Section 4.3 (swirl):
    the fluxes of a constant telescope, so the averages stay constant."""
    n, px = 8, 4
    lo, hi = ((-1.0, -1.0), (1.0, 1.0)) if field == O.SOLID_BODY else ((0.0, 0.0), (1.0, 1.0))
    grid = S.UniformGrid(S.Layout(n, 1), px, px, lo, hi)
    st = S.periodic_state(grid, [lambda x, y: 1.0 + 0.0 * x * y], nq=2)
    vmax = np.pi * np.sqrt(2.0) if field == O.SOLID_BODY else 1.0
    vc = O.VarCfg(n, field, grid.dx, grid.dy, 0.5 * grid.dx / vmax, 0.0, 0.0, 0.1)
    out = O.run_uniform_var(vc, px, px, lo, 12, st)
    assert np.abs(grid.interior_averages(out, 0) - 1.0).max() < 1e-13


def test_solid_body_third_order_convergence():
    """A smooth Gaussian rotated a quarter turn on [-1, 1]^2: errors fall by
    about 8 per halving of the mesh width."""
    f = S.gaussian(0.3, 0.2, 0.12)
    errs = []
    for px in (4, 8):
        n = 8
        grid = S.UniformGrid(S.Layout(n, 1), px, px, (-1.0, -1.0), (1.0, 1.0))
        st = S.periodic_state(grid, [f], nq=4)
        nsteps, dt = S.steps_to(0.5, 0.6 * grid.dx / (np.pi * 1.42))
        vc = O.VarCfg(n, O.SOLID_BODY, grid.dx, grid.dy, dt, 0.0, 0.0, 0.0)
        out = O.run_uniform_var(vc, px, px, (-1.0, -1.0), nsteps, st)
        ex = lambda x, y: f(x * np.cos(np.pi * 0.5) + y * np.sin(np.pi * 0.5),
                            -x * np.sin(np.pi * 0.5) + y * np.cos(np.pi * 0.5))
        errs.append(grid.l1_error(out, 0, ex, nq=4))
    eoc = np.log2(errs[0] / errs[1])
    assert eoc > 2.6, (errs, eoc)


def test_swirl_reproduces_table3_level4():
    """Table 3 (Section 4.3): smooth swirl at t = 1 on 256^2 cells.  With
    CFL 0.5 (the paper does not state it; CFL 0.4 and 0.6 give errors 8 %
    above and 9 % below) the oracle's error is within 2 % of the printed
    value; at 512^2 (not run here) it is 7.168e-7 against 7.268e-7."""
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
    printed = ref["table3_swirl_uniform"]["levels"]["4"]["error"]
    n, px = 16, 16
    grid = S.UniformGrid(S.Layout(n, 1), px, px)
    st = S.periodic_state(grid, [S.swirl_gaussians], nq=4)
    nsteps, dt = S.steps_to(1.0, 0.5 * grid.dx)
    vc = O.VarCfg(n, O.SWIRL, grid.dx, grid.dy, dt, 0.0, 0.0, 0.0)
    out = O.run_uniform_var(vc, px, px, (0.0, 0.0), nsteps, st)
    err = grid.l1_error(out, 0, S.swirl_gaussians, nq=4)
    assert abs(err / printed - 1.0) < 0.02, (err, printed)
