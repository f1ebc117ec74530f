"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test states the pin it implements.  None of them re-types the oracle's
formulas: they compare with closed-form exact solutions, brute-force
quadrature of the defining integral, invariants, or special cases.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synth as S

G = S.G


def _poly(coef):
    """Polynomial sum coef[(m, n)] x^m y^n as a numpy callable."""
    return lambda x, y: sum(c * x ** m * y ** n for (m, n), c in coef.items())


# ---------------------------------------------------------------- P1: Eq. poly
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_p1_reconstruction_reproduces_biquadratics(seed):
    """Section 2, Eq. poly: the reconstruction from 8 boundary point values and
    the cell average reproduces any biquadratic exactly (values and
    derivatives) and its cell average equals Q_{i,j}."""
    rng = np.random.default_rng(seed)
    coef = {(m, n): rng.uniform(-2, 2) for m in range(3) for n in range(3)}
    f = _poly(coef)
    lay = S.Layout(6, 1)
    grid = S.UniformGrid(lay, 1, 1, (0.0, 0.0), (0.6, 0.9))
    st = grid.state([f], ghosts=True, periodic=False, nq=4)
    dx, dy = grid.dx, grid.dy
    fx = lambda x, y: sum(c * m * x ** (m - 1) * y ** n for (m, n), c in coef.items() if m > 0)
    fy = lambda x, y: sum(c * n * x ** m * y ** (n - 1) for (m, n), c in coef.items() if n > 0)
    for (i, j) in [(0, 0), (2, 4), (-2, -1), (7, 7)]:
        for xi, eta in rng.uniform(-1, 1, size=(5, 2)):
            x, y = (i + 0.5 + 0.5 * xi) * dx, (j + 0.5 + 0.5 * eta) * dy
            assert abs(O.recon_eval(6, 1, st[0], 0, i, j, xi, eta, 0, 0, dx, dy) - f(x, y)) < 1e-12
            assert abs(O.recon_eval(6, 1, st[0], 0, i, j, xi, eta, 1, 0, dx, dy) - fx(x, y)) < 1e-10
            assert abs(O.recon_eval(6, 1, st[0], 0, i, j, xi, eta, 0, 1, dx, dy) - fy(x, y)) < 1e-10
        # average of the reconstruction (5x5 Gauss-Legendre, exact for degree 9)
        gx, gw = np.polynomial.legendre.leggauss(5)
        avg = sum(gw[a] * gw[b] * O.recon_eval(6, 1, st[0], 0, i, j, gx[a], gx[b])
                  for a in range(5) for b in range(5)) / 4.0
        lat = lay.lattice(st)
        assert abs(avg - lat[0, 0, S.AVG, j + G, i + G]) < 1e-13


def test_p1_reconstruction_interpolates_random_nodes():
    """The reconstruction passes through the 8 stored point values and has
    the stored average, for arbitrary (non-polynomial) data."""
    lay = S.Layout(4, 1)
    st = S.random_state(lay, 1, seed=7)
    lat = lay.lattice(st)
    for (i, j) in [(0, 0), (1, 3), (-2, 5)]:
        I, J = i + G, j + G
        pts = {(-1, -1): lat[0, 0, S.CORNER, J, I], (1, -1): lat[0, 0, S.CORNER, J, I + 1],
               (-1, 1): lat[0, 0, S.CORNER, J + 1, I], (1, 1): lat[0, 0, S.CORNER, J + 1, I + 1],
               (-1, 0): lat[0, 0, S.XMID, J, I], (1, 0): lat[0, 0, S.XMID, J, I + 1],
               (0, -1): lat[0, 0, S.YMID, J, I], (0, 1): lat[0, 0, S.YMID, J + 1, I]}
        for (xi, eta), v in pts.items():
            assert abs(O.recon_eval(4, 1, st[0], 0, i, j, xi, eta) - v) < 1e-14
        gx, gw = np.polynomial.legendre.leggauss(5)
        avg = sum(gw[a] * gw[b] * O.recon_eval(4, 1, st[0], 0, i, j, gx[a], gx[b])
                  for a in range(5) for b in range(5)) / 4.0
        assert abs(avg - lat[0, 0, S.AVG, J, I]) < 1e-14


# ------------------------------------------------- P2/P3: Section 2.1 advection
ADV_CASES = [(1.0, 0.5, 0.6), (-0.7, 0.4, 0.75), (0.3, -1.1, 0.9), (-0.5, -0.5, 0.4), (1.0, 0.0, 0.5)]


@pytest.mark.parametrize("a,b,cfl", ADV_CASES)
def test_p2_p3_advection_step_exact_for_q2_minus_x2y2(a, b, cfl):
    """Eq. advection-update is exact translation, and Simpson's rule in (y, t)
    is exact for the resulting fluxes when the data lie in the span of the
    Q2 monomials except x^2 y^2: one full step (all point values, all
    averages of interior + first ghost layer) equals the exact solution."""
    rng = np.random.default_rng(11)
    coef = {(m, n): rng.uniform(-1, 1) for m in range(3) for n in range(3) if (m, n) != (2, 2)}
    f = _poly(coef)
    n = 8
    lay = S.Layout(n, 1)
    grid = S.UniformGrid(lay, 1, 1, (0.1, -0.2), (0.9, 0.6))
    st = grid.state([f], ghosts=True, periodic=False, nq=4)
    dt = S.cfl_dt("advection", cfl, grid.dx, grid.dy, a, b)
    cf = O.cfg(O.ADVECTION, n, grid.dx, grid.dy, dt, a, b)
    out = O.step_patch(cf, st[0])
    ex = grid.state([lambda x, y: f(x - a * dt, y - b * dt)], ghosts=True, periodic=False, nq=4)[0]
    L, E = lay.lattice(out)[0], lay.lattice(ex)[0]
    r = slice(G - 1, G + n + 1)          # cells / lines -1 .. N
    r1 = slice(G - 1, G + n + 2)         # lines -1 .. N+1
    scale = np.abs(E).max()
    assert np.abs(L[S.AVG][r, r] - E[S.AVG][r, r]).max() < 1e-13 * scale
    assert np.abs(L[S.CORNER][r1, r1] - E[S.CORNER][r1, r1]).max() < 1e-13 * scale
    assert np.abs(L[S.XMID][r, r1] - E[S.XMID][r, r1]).max() < 1e-13 * scale
    assert np.abs(L[S.YMID][r1, r] - E[S.YMID][r1, r]).max() < 1e-13 * scale


def test_p2_advection_node_exact_translation_biquadratic():
    """Point values of Eq. advection-update are exact for any biquadratic
    (x^2 y^2 included): the foot value of the exact reconstruction."""
    f = _poly({(2, 2): 1.3, (1, 2): -0.4, (2, 0): 0.7, (0, 1): 2.0, (0, 0): -1.0})
    n = 6
    lay = S.Layout(n, 1)
    grid = S.UniformGrid(lay, 1, 1)
    st = grid.state([f], ghosts=True, periodic=False, nq=5)
    a, b = -0.8, 0.35
    dt = S.cfl_dt("advection", 0.95, grid.dx, grid.dy, a, b)
    cf = O.cfg(O.ADVECTION, n, grid.dx, grid.dy, dt, a, b)
    offs = {O.CORNER: (0.0, 0.0), O.XMID: (0.0, 0.5), O.YMID: (0.5, 0.0)}
    for ty, (ox, oy) in offs.items():
        for (i, j) in [(0, 0), (3, 2), (-1, -1), (n, n)]:
            for tau in (0.5 * dt, dt):
                x, y = (i + ox) * grid.dx, (j + oy) * grid.dy
                v = O.node_evolve(cf, st[0], ty, i, j, tau)[0]
                assert abs(v - f(x - a * tau, y - b * tau)) < 1e-13


# ------------------------------------------ P4: Eq. sphe-mean by brute force
def _brute_node(patch, n, dx, dy, c, tau, xn, yn):
    """Eq. ERFormula evaluated by brute-force quadrature of Eq. sphe-mean.

    s = R sin(theta) removes the weak singularity: M_R{f} = 1/(2 pi)
    int_0^{2 pi} int_0^{pi/2} f(x + R sin(theta) e_phi) sin(theta) dtheta dphi,
    and d_R M_R{f} = 1/(2 pi) int int grad f . e_phi sin^2(theta).  The disc is
    split at cell faces into angular pieces (each integrand is then a
    polynomial) and Gauss-Legendre is used in theta and phi on every piece."""
    R = c * tau
    tq, tw = np.polynomial.legendre.leggauss(24)
    th = 0.25 * np.pi * (tq + 1.0)
    thw = 0.25 * np.pi * tw
    # phi break points at the cell faces through the node: multiples of pi/2
    pq, pw = np.polynomial.legendre.leggauss(24)

    def ev(comp, x, y, mx, my):
        i, j = int(math.floor(x / dx)), int(math.floor(y / dy))
        xi = 2.0 * (x / dx - i) - 1.0
        eta = 2.0 * (y / dy - j) - 1.0
        return O.recon_eval(n, 3, patch, comp, i, j, xi, eta, mx, my, dx, dy)

    acc = dict(Mp=0.0, dMp=0.0, Mu=0.0, dMu=0.0, Mv=0.0, dMv=0.0, Mdiv=0.0, Mpx=0.0, Mpy=0.0)
    for q in range(4):
        p0, p1 = q * 0.5 * np.pi, (q + 1) * 0.5 * np.pi
        phis = 0.5 * (p1 - p0) * (pq + 1.0) + p0
        phw = 0.5 * (p1 - p0) * pw
        for f, wf in zip(phis, phw):
            e = (math.cos(f), math.sin(f))
            for t, wt in zip(th, thw):
                s = R * math.sin(t)
                x, y = xn + s * e[0], yn + s * e[1]
                w = wf * wt * math.sin(t) / (2 * np.pi)
                wd = wf * wt * math.sin(t) ** 2 / (2 * np.pi)
                vals = {k: [ev(k, x, y, 0, 0), ev(k, x, y, 1, 0), ev(k, x, y, 0, 1)] for k in range(3)}
                acc["Mp"] += w * vals[0][0]
                acc["dMp"] += wd * (vals[0][1] * e[0] + vals[0][2] * e[1])
                acc["Mu"] += w * vals[1][0]
                acc["dMu"] += wd * (vals[1][1] * e[0] + vals[1][2] * e[1])
                acc["Mv"] += w * vals[2][0]
                acc["dMv"] += wd * (vals[2][1] * e[0] + vals[2][2] * e[1])
                acc["Mdiv"] += w * (vals[1][1] + vals[2][2])
                acc["Mpx"] += w * vals[0][1]
                acc["Mpy"] += w * vals[0][2]
    p = acc["Mp"] + R * (acc["dMp"] - acc["Mdiv"])
    u = acc["Mu"] + R * (acc["dMu"] - acc["Mpx"])
    v = acc["Mv"] + R * (acc["dMv"] - acc["Mpy"])
    return np.array([p, u, v])


@pytest.mark.parametrize("node", [(O.CORNER, 2, 3), (O.XMID, 1, 1), (O.YMID, 3, 2)])
def test_p4_spherical_means_match_brute_force(node):
    """Section 2.3, Eqs. ERFormula and sphe-mean: the oracle's closed-form
    sector integrals agree with brute-force quadrature of the defining
    integral on random piecewise-biquadratic data (dx != dy)."""
    ty, i, j = node
    n = 4
    lay = S.Layout(n, 3)
    st = S.random_state(lay, 1, seed=3)
    dx, dy = 0.3, 0.25
    c = 1.7
    dt = 0.5 * min(dx, dy) / c
    cf = O.cfg(O.ACOUSTICS, n, dx, dy, dt, c=c)
    ox, oy = {O.CORNER: (0, 0), O.XMID: (0, 0.5), O.YMID: (0.5, 0)}[ty]
    for tau in (0.5 * dt, dt):
        got = O.node_evolve(cf, st[0], ty, i, j, tau)
        ref = _brute_node(st[0], n, dx, dy, c, tau, (i + ox) * dx, (j + oy) * dy)
        assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


# ---------------------------------------- P5: exact wave solution, curl-free data
def test_p5_acoustic_nodes_exact_for_curl_free_polynomial_data():
    """For u0 = 0 and biquadratic p0 the vorticity vanishes, Eq. ERFormula is
    exact (Section 2.3), and the solution of the wave system is
    p = p0 + R^2/2 Lap p0 + R^4/24 Lap^2 p0, u = -R grad p0 - R^3/6 grad Lap p0."""
    rng = np.random.default_rng(5)
    C = {(m, n): rng.uniform(-1, 1) for m in range(3) for n in range(3)}
    p0 = _poly(C)
    zero = lambda x, y: 0.0 * x
    cc = lambda m, n: C.get((m, n), 0.0)
    # Laplacian of sum C_mn x^m y^n and its derivatives, written out by monomial
    def lap(x, y):
        return (2 * cc(2, 0) + 2 * cc(2, 1) * y + 2 * cc(2, 2) * y * y
                + 2 * cc(0, 2) + 2 * cc(1, 2) * x + 2 * cc(2, 2) * x * x)
    lap2 = 8 * cc(2, 2)
    def px(x, y):
        return sum(C[(m, n)] * m * x ** (m - 1) * y ** n for (m, n) in C if m > 0)
    def py(x, y):
        return sum(C[(m, n)] * n * x ** m * y ** (n - 1) for (m, n) in C if n > 0)
    lapx = lambda x, y: 2 * cc(1, 2) + 4 * cc(2, 2) * x
    lapy = lambda x, y: 2 * cc(2, 1) + 4 * cc(2, 2) * y
    n = 6
    lay = S.Layout(n, 3)
    grid = S.UniformGrid(lay, 1, 1, (-0.3, 0.2), (0.9, 1.4))
    st = grid.state([p0, zero, zero], ghosts=True, periodic=False, nq=4)
    c = 0.8
    dt = S.cfl_dt("acoustics", 0.5, grid.dx, grid.dy, c=c)
    cf = O.cfg(O.ACOUSTICS, n, grid.dx, grid.dy, dt, c=c)
    offs = {O.CORNER: (0.0, 0.0), O.XMID: (0.0, 0.5), O.YMID: (0.5, 0.0)}
    for ty, (ox, oy) in offs.items():
        for (i, j) in [(0, 0), (2, 5), (-1, 4), (n, n)]:
            for tau in (0.5 * dt, dt):
                R = c * tau
                x, y = grid.lo[0] + (i + ox) * grid.dx, grid.lo[1] + (j + oy) * grid.dy
                exact = np.array([p0(x, y) + R * R / 2 * lap(x, y) + R ** 4 / 24 * lap2,
                                  -R * px(x, y) - R ** 3 / 6 * lapx(x, y),
                                  -R * py(x, y) - R ** 3 / 6 * lapy(x, y)])
                got = O.node_evolve(cf, st[0], ty, i, j, tau)
                assert np.abs(got - exact).max() < 1e-13


# ---------------------------------------------------- P6: stationary states
def test_p6_constant_states_preserved():
    """Constants are stationary for both PDEs; one periodic step keeps them to
    round-off (each flux difference cancels)."""
    for eq, nc, vals in [(O.ADVECTION, 1, [0.7]), (O.ACOUSTICS, 3, [1.0, -2.0, 0.5])]:
        lay = S.Layout(8, nc)
        grid = S.UniformGrid(lay, 2, 2)
        st = grid.state([lambda x, y, v=v: v + 0 * x for v in vals], nq=2)
        dt = 0.4 * grid.dx
        cf = O.cfg(eq, 8, grid.dx, grid.dy, dt, 1.0, -0.5, 1.0)
        out = O.run_uniform(cf, 2, 2, 3, st)
        own = S.unpack_owned(grid, out)
        for k, v in enumerate(vals):
            assert np.abs(own[k] - v).max() < 1e-14


def test_p6_linear_rotation_is_stationary_for_acoustics():
    """p = const, u = w(-y, x): divergence-free with constant vorticity, so
    Eq. ERFormula is exact and the state is stationary; one step on a patch
    with exact ghosts leaves every updated value unchanged."""
    w = 1.3
    n = 8
    lay = S.Layout(n, 3)
    grid = S.UniformGrid(lay, 1, 1, (-0.5, -0.4), (0.7, 0.8))
    funcs = [lambda x, y: 2.0 + 0 * x, lambda x, y: -w * y, lambda x, y: w * x]
    st = grid.state(funcs, ghosts=True, periodic=False, nq=3)
    dt = S.cfl_dt("acoustics", 0.5, grid.dx, grid.dy)
    cf = O.cfg(O.ACOUSTICS, n, grid.dx, grid.dy, dt, c=1.0)
    out = O.step_patch(cf, st[0])
    L, E = lay.lattice(out), lay.lattice(st[0])
    r = slice(G - 1, G + n + 1)
    assert np.abs(L[:, :, r, r] - E[:, :, r, r]).max() < 1e-14


# ----------------------------------------------------- P7: conservation
@pytest.mark.parametrize("eq", [O.ADVECTION, O.ACOUSTICS])
def test_p7_mass_conserved_periodic(eq):
    """Eq. 2dfv with single-valued face fluxes conserves sum Q dx dy exactly
    up to round-off on a periodic array of patches."""
    nc = 1 if eq == O.ADVECTION else 3
    lay = S.Layout(8, nc)
    grid = S.UniformGrid(lay, 3, 2)
    own = S.random_owned(grid, seed=21)
    st = S.pack_owned(grid, own)
    dt = 0.4 * grid.dx
    cf = O.cfg(eq, 8, grid.dx, grid.dy, dt, 0.9, -0.6, 1.0)
    out = O.run_uniform(cf, 3, 2, 4, st)
    o2 = S.unpack_owned(grid, out)
    for k in range(nc):
        m0, m1 = own[k, S.AVG].sum(), o2[k, S.AVG].sum()
        assert abs(m1 - m0) < 1e-12 * np.abs(own[k, S.AVG]).sum()


# ------------------------------------------- P9: single patch == multi patch
@pytest.mark.parametrize("eq", [O.ADVECTION, O.ACOUSTICS])
def test_p9_single_patch_equals_multi_patch(eq):
    """A uniform grid as one patch or as several same-level patches with
    copied ghosts (Section 3.1, case 3) gives bitwise identical results."""
    nc = 1 if eq == O.ADVECTION else 3
    big = S.UniformGrid(S.Layout(16, nc), 1, 1)
    small = S.UniformGrid(S.Layout(8, nc), 2, 2)
    own = S.random_owned(big, seed=4)
    dt = 0.45 * big.dx
    cfb = O.cfg(eq, 16, big.dx, big.dy, dt, 0.8, 0.3, 1.0)
    cfs = O.cfg(eq, 8, small.dx, small.dy, dt, 0.8, 0.3, 1.0)
    ob = O.run_uniform(cfb, 1, 1, 3, S.pack_owned(big, own))
    os_ = O.run_uniform(cfs, 2, 2, 3, S.pack_owned(small, own))
    assert np.array_equal(S.unpack_owned(big, ob), S.unpack_owned(small, os_))


def test_fill_periodic_copies_neighbour_entries():
    """Same-level ghost fill on a periodic patch array reproduces the
    analytic ghost values of a periodic function exactly (pure copies)."""
    lay = S.Layout(4, 1)
    grid = S.UniformGrid(lay, 3, 2)
    f = lambda x, y: np.sin(2 * np.pi * x) + np.cos(2 * np.pi * y)
    full = grid.state([f], ghosts=True, nq=2)
    st = grid.state([f], ghosts=False, nq=2)
    O.fill_periodic(4, 1, 3, 2, st)
    lat_a, lat_b = lay.lattice(full), lay.lattice(st)
    # the analytic ghost values come from wrapped coordinates: equal to round-off
    assert np.abs(lat_a - lat_b).max() < 1e-12
    assert not np.isnan(lat_b).any()
