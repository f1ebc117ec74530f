"""Parity of variable-velocity advection (af_patch_step_var; solid-body
rotation and swirl, Sections 4.2 and 4.3) with the FP64 oracle through the C
ABI: uniform periodic runs in every tiling, subcycled adaptive runs, and the
paper's constant-state results on the GPU."""
import numpy as np
import pytest

import oracle as O
import synth as S
from fp32_parity import lockstep_amr
from oracle.amr import OracleForest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def af():
    from paper_2205_07572_gb300 import af as _af, build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _af


def _nerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = {
    0: ((-1.0, -1.0), (1.0, 1.0), S.gaussian(0.3, 0.2, 0.15), np.pi * 1.6),
    1: ((0.0, 0.0), (1.0, 1.0), S.swirl_gaussians, 1.0),
}


def _uniform(af, field, prec, n, px, steps, tiling=None, const=False):
    from paper_2205_07572_gb300.uniform import UniformRun
    lo, hi, f, vmax = CASES[field]
    if const:
        f = lambda x, y: 1.0 + 0.0 * x * y
    grid = S.UniformGrid(S.Layout(n, 1), px, px, lo, hi)
    st = S.periodic_state(grid, [f], nq=3)
    if prec:
        st = st.astype(np.float32).astype(np.float64)
    dt = 0.45 * grid.dx / vmax
    vc = O.VarCfg(n, field, grid.dx, grid.dy, dt, 0.0, 0.0, 0.1)
    ref = O.run_uniform_var(vc, px, px, lo, steps, st)
    cfg = af.config(af.ADVECTION, prec, n)
    run = UniformRun(cfg, px, px, grid.dx, grid.dy, dt, state=st, tiling=tiling, field=field, lo=lo, t0=0.1)
    for _ in range(steps):
        run.step()
    torch.cuda.synchronize()
    return grid, run.state.double().cpu().numpy().reshape(st.shape), ref


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("field", [0, 1])
def test_uniform_run_matches_oracle(af, field, prec):
    grid, got, ref = _uniform(af, field, prec, 16, 3, 5)
    g, r = grid.interior_averages(got, 0), grid.interior_averages(ref, 0)
    assert _nerr(g, r) < TOL[prec], _nerr(g, r)
    og, orf = S.unpack_owned(grid, got), S.unpack_owned(grid, ref)
    assert _nerr(og, orf) < TOL[prec]


@pytest.mark.parametrize("field", [0, 1])
def test_every_tiling_matches_oracle(af, field):
    tilings = af.step_tilings()
    for k in range(len(tilings)):
        grid, got, ref = _uniform(af, field, 0, 16, 2, 2, tiling=k)
        og, orf = S.unpack_owned(grid, got), S.unpack_owned(grid, ref)
        assert _nerr(og, orf) < 1e-12, (k, tilings[k])


@pytest.mark.parametrize("field", [0, 1])
def test_constant_state_preserved_on_gpu(af, field):
    """Remark of Section 4.2 / Theorem of Section 4.3, FP64 on the GPU."""
    grid, got, _ = _uniform(af, field, 0, 16, 3, 20, const=True)
    assert np.abs(grid.interior_averages(got, 0) - 1.0).max() < 1e-13


@pytest.mark.parametrize("prec", [0, 1])
def test_subcycled_swirl_amr_matches_oracle(af, prec):
    """Levels 2-3 along the diagonal, swirl, two coarse steps with
    subcycling, reflux and ghost exchange; same answer as the oracle."""
    from paper_2205_07572_gb300.amr import AMRRun
    n, lmax = 8, 3
    leaves = sorted(S.balanced_forest(1, 2, 3, lambda l, x, y: x == y), key=lambda t: (t[0], t[2], t[1]))
    st = S.forest_state(n, 1, 1, lmax, leaves, [S.swirl_gaussians], nq=3)
    if prec:
        st = st.astype(np.float32).astype(np.float64)
    dx0 = 1.0 / n
    dt0 = 0.45 * dx0
    Fo = OracleForest(O.ADVECTION, n, 1, lmax, leaves, (0, 0), (1, 1), dt0, state=st, field=O.SWIRL, t0=0.2)
    Fo.sync_fill((1 << (lmax + 1)) - 1)
    run = AMRRun(af.config(af.ADVECTION, prec, n), 1, lmax, leaves, st, (0, 0), (1, 1), dt0, field=af.FIELD_SWIRL)
    run.time = 0.2
    m0 = run.mass()
    lay = S.Layout(n, 1)

    def compare(F, tol):
        g = lay.lattice(run.state_in_order(F.leaves).reshape(len(leaves), 1, 4, -1))[..., 2:2 + n, 2:2 + n]
        r = lay.lattice(F.state.reshape(len(leaves), 1, 4, -1))[..., 2:2 + n, 2:2 + n]
        assert _nerr(g, r) < tol, _nerr(g, r)

    lockstep_amr(Fo, run, 2, compare, prec, torch.cuda.synchronize)
    if prec == 0:
        assert abs(run.mass()[0] - m0[0]) < 1e-13 * abs(m0[0])
        assert abs(Fo.time - run.time) < 1e-15


def test_subcycled_swirl_constant_state_matches_oracle(af):
    """Section 4.3: with subcycling the fine fluxes summed at intermediate
    times are not balanced exactly by the coarse ones, so a constant state
    drifts slightly; on this coarse forest (levels 2-3 of 8 x 8 patches) the
    drift is ~1e-9 after four coarse steps, and the GPU's drift is the
    oracle's."""
    from paper_2205_07572_gb300.amr import AMRRun
    n, lmax = 8, 3
    leaves = sorted(S.balanced_forest(1, 2, 3, lambda l, x, y: x == y), key=lambda t: (t[0], t[2], t[1]))
    st = S.forest_state(n, 1, 1, lmax, leaves, [lambda x, y: 1.0 + 0.0 * x * y], nq=2)
    dt0 = 0.45 / n
    run = AMRRun(af.config(af.ADVECTION, 0, n), 1, lmax, leaves, st, (0, 0), (1, 1), dt0, field=af.FIELD_SWIRL)
    Fo = OracleForest(O.ADVECTION, n, 1, lmax, leaves, (0, 0), (1, 1), dt0, state=st, field=O.SWIRL)
    Fo.sync_fill((1 << (lmax + 1)) - 1)
    for _ in range(4):
        run.coarse_step()
        Fo.coarse_step()
    torch.cuda.synchronize()
    lay = S.Layout(n, 1)
    g = lay.lattice(run.state_in_order(Fo.leaves).reshape(len(leaves), 1, 4, -1))[:, 0, 0, 2:2 + n, 2:2 + n]
    r = lay.lattice(Fo.state.reshape(len(leaves), 1, 4, -1))[:, 0, 0, 2:2 + n, 2:2 + n]
    err_gpu, err_orc = np.abs(g - 1.0).max(), np.abs(r - 1.0).max()
    assert err_orc < 1e-8 and abs(err_gpu - err_orc) < 1e-3 * err_orc, (err_gpu, err_orc)
    assert np.abs(g - r).max() < 1e-14


def test_subcycled_swirl_constant_state_paper_configuration(af):
    """Section 4.3's experiment: constant 1, swirl, levels 3-4 along the
    diagonal (16 x 16-cell patches), subcycling, to t = 1.  The paper
    observes an error of size 1e-13 at a CFL number it does not state; at
    CFL 0.5 this run gives 6e-12 (the drift comes from the subcycled fluxes
    at intermediate times and falls steeply with the time step)."""
    from paper_2205_07572_gb300.amr import AMRRun
    n, lmax = 16, 4
    leaves = sorted(S.balanced_forest(1, 3, 4, lambda l, x, y: x == y), key=lambda t: (t[0], t[2], t[1]))
    st = S.forest_state(n, 1, 1, lmax, leaves, [lambda x, y: 1.0 + 0.0 * x * y], nq=2)
    dx0 = 1.0 / n
    nsteps, dt0 = S.steps_to(1.0, 0.5 * dx0 / 8)      # coarsest present level is 3
    run = AMRRun(af.config(af.ADVECTION, 0, n), 1, lmax, leaves, st, (0, 0), (1, 1), dt0 * 8,
                 field=af.FIELD_SWIRL)
    assert run.forest.levels[0] == 3
    for _ in range(nsteps):
        run.coarse_step()
    torch.cuda.synchronize()
    assert abs(run.time - 1.0) < 1e-12
    lay = S.Layout(n, 1)
    g = lay.lattice(run.current().double().cpu().numpy().reshape(run.forest.nleaf, 1, 4, -1))
    err = np.abs(g[:, 0, 0, 2:2 + n, 2:2 + n] - 1.0).max()
    assert err < 2e-11, err


def _patch_with_neighbour_halo(grid, lat, p):
    """Lattice of patch p with every ghost entry taken from the owned entry of
    the same global node or cell (periodic), as the step's halo reads it."""
    n, g, w = grid.layout.n, S.G, grid.layout.w
    ix, iy = p % grid.px, p // grid.px
    gx = (ix * n + np.arange(w) - g) % (grid.px * n)
    gy = (iy * n + np.arange(w) - g) % (grid.py * n)
    q = (gy[:, None] // n) * grid.px + gx[None, :] // n
    return lat[q, :, :, (gy % n)[:, None] + g, (gx % n)[None, :] + g].transpose(2, 3, 0, 1)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("field", [0, 1])
def test_bench_workload_full_size_sampled_patches_match_oracle(af, field, prec):
    """The benchmark's variable-velocity workloads at full size (4096^2 cells
    as 256 x 256 patches of 16 x 16; swirl on the unit square, solid body on
    [-1, 1]^2; dt = 0.45 dx / max speed), one step from t = 0 in both tilings
    the benchmark chooses between (18 x 18 element-wise staged, 16 x 16 bulk
    staged): sampled patches match the oracle's single-patch step, every
    owned DOF."""
    from paper_2205_07572_gb300.uniform import UniformRun
    n, P = 16, 256
    lo, hi = ((0.0, 0.0), (1.0, 1.0)) if field == 1 else ((-1.0, -1.0), (1.0, 1.0))
    f = S.swirl_gaussians if field == 1 else S.gaussian(0.3, 0.2, 0.1)
    vmax = 1.0 if field == 1 else np.pi * 1.01
    grid = S.UniformGrid(S.Layout(n, 1), P, P, lo, hi)
    st = S.periodic_state(grid, [f], nq=2, dtype=np.float32 if prec else np.float64)
    dt = 0.45 * grid.dx / vmax
    cfg = af.config(af.ADVECTION, prec, n)
    lay = S.Layout(n, 1)
    lat = lay.lattice(st.reshape(P * P, 1, 4, -1).astype(np.float64))
    scale = np.abs(lat[:, 0, :, S.G:S.G + n, S.G:S.G + n]).max()
    samples = [0, P - 1, P * (P - 1), P * P - 1, P * 128 + 128, P * 77 + 200, 40000]
    tl = [t[:3] for t in af.step_tilings()]
    for k in (tl.index((18, 18, 256)), tl.index((16, 16, 128))):
        run = UniformRun(cfg, P, P, grid.dx, grid.dy, dt, state=st, tiling=k, field=field, lo=lo)
        af.step_wait_timeouts(reset=True)
        run.step()
        torch.cuda.synchronize()
        got = run.state[torch.tensor(samples, device="cuda")].double().cpu().numpy().reshape(len(samples), 1, 4, -1)
        for i, p in enumerate(samples):
            ix, iy = p % P, p // P
            vc = O.VarCfg(n, field, grid.dx, grid.dy, dt, lo[0] + ix * n * grid.dx, lo[1] + iy * n * grid.dy, 0.0)
            patch = np.zeros((1, 4, lay.plane))
            lay.lattice(patch)[...] = _patch_with_neighbour_halo(grid, lat, p)
            ref = lay.lattice(O.step_patch_var(vc, patch))[..., S.G:S.G + n, S.G:S.G + n]
            g = lay.lattice(got[i])[..., S.G:S.G + n, S.G:S.G + n]
            err = np.abs(g - ref).max() / scale
            assert err < TOL[prec], (k, p, err)
        assert af.step_wait_timeouts() == 0
        del run
