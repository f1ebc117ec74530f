"""Parity of af_patch_step (CUDA, called through the C ABI) with the FP64 oracle.

Tolerances (normwise relative per component: max|gpu - oracle| / max|oracle|):
FP64 1e-12, FP32 1e-5.  For FP32 the oracle runs on the FP32-rounded inputs,
so the difference measured is the FP32 arithmetic of the kernel only; runs of
K steps hold every step, restarted from the GPU's own FP32 state, to 1e-5 and
the trajectory to K x 1e-5 (fp32_parity).
"""
import numpy as np
import pytest

import oracle as O
import synth as S
from fp32_parity import TOL32

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


def _normwise(gpu, ref, ncomp):
    g = gpu.reshape(gpu.shape[0], ncomp, -1)
    r = ref.reshape(ref.shape[0], ncomp, -1)
    errs = []
    for c in range(ncomp):
        d = np.nanmax(np.abs(g[:, c] - r[:, c]))
        s = np.nanmax(np.abs(r[:, c]))
        errs.append(d / max(s, 1e-300))
    return max(errs)


def _dt(eq, cfl, dx, dy, a, b, c):
    return S.cfl_dt("advection" if eq == 0 else "acoustics", cfl, dx, dy, a, b, c)


CASES = [
    # eq, n, npatch, a, b, cfl
    (0, 8, 3, 1.0, 0.5, 0.6),
    (0, 16, 2, -0.7, 0.9, 0.95),
    (0, 32, 2, 0.4, -1.0, 0.75),
    (0, 64, 1, -1.0, -0.3, 0.4),
    (1, 8, 3, 0.0, 0.0, 0.5),
    (1, 16, 2, 0.0, 0.0, 0.4),
    (1, 32, 2, 0.0, 0.0, 0.45),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("eq,n,npatch,a,b,cfl", CASES)
def test_step_own_ghosts_matches_oracle(af, prec, eq, n, npatch, a, b, cfl):
    """No neighbour table: every patch reads its own (filled) ghost ring and
    advances interior + first ghost layer, exactly the oracle's step."""
    nc = 1 if eq == 0 else 3
    lay = S.Layout(n, nc)
    st = S.random_state(lay, npatch, seed=100 + n + eq)
    npdt = np.float64 if prec == 0 else np.float32
    st = st.astype(npdt).astype(np.float64)
    dx, dy = 0.37 / n, 0.29 / n
    c = 1.3
    dt = _dt(eq, cfl, dx, dy, a, b, c)
    cf = O.cfg(eq, n, dx, dy, dt, a, b, c)
    ref = np.stack([O.step_patch(cf, st[p]) for p in range(npatch)])
    cfg = af.config(eq, prec, n, a, b, c)
    work = af.build_step_work(cfg, np.arange(npatch))
    tdt = torch.float64 if prec == 0 else torch.float32
    din = torch.from_numpy(st.reshape(npatch, -1)).to(tdt).cuda()
    dout = din.clone()
    wd = torch.from_numpy(work).cuda()
    af.patch_step(cfg, wd, len(work) // 64, din, dout, dt, dx, dy)
    torch.cuda.synchronize()
    got = dout.double().cpu().numpy().reshape(ref.shape)
    assert _normwise(got, ref, nc) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("eq", [0, 1])
def test_uniform_periodic_multistep_matches_oracle(af, prec, eq):
    """Periodic array of same-level patches, halo read from neighbours (fused
    same-level ghost copy), several steps: interior-owned DOFs equal the
    oracle's fill-then-step run; the mass sum is conserved."""
    from paper_2205_07572_gb300.uniform import UniformRun
    nc = 1 if eq == 0 else 3
    n, px, py, steps = 16, 3, 2, 6
    grid = S.UniformGrid(S.Layout(n, nc), px, py)
    own = S.random_owned(grid, seed=7 + eq)
    if prec == 1:
        own = own.astype(np.float32).astype(np.float64)
    st = S.pack_owned(grid, own)
    a, b, c = 0.8, -0.45, 1.0
    dt = _dt(eq, 0.45, grid.dx, grid.dy, a, b, c)
    cfo = O.cfg(eq, n, grid.dx, grid.dy, dt, a, b, c)
    ref = O.run_uniform(cfo, px, py, steps, st)
    cfg = af.config(eq, prec, n, a, b, c)
    run = UniformRun(cfg, px, py, grid.dx, grid.dy, dt, state=np.nan_to_num(st))
    for s_ in range(steps):
        if prec:   # the oracle's step from the GPU's own FP32 state
            torch.cuda.synchronize()
            cur = np.nan_to_num(run.state.double().cpu().numpy().reshape(st.shape))
            one = S.unpack_owned(grid, O.run_uniform(cfo, px, py, 1, cur))
        run.step()
        if prec:
            torch.cuda.synchronize()
            g1 = S.unpack_owned(grid, run.state.double().cpu().numpy().reshape(st.shape))
            for k in range(nc):
                err = np.abs(g1[k] - one[k]).max() / np.abs(one[k]).max()
                assert err < TOL32, ("step", s_, k, err)
    torch.cuda.synchronize()
    got = run.state.double().cpu().numpy().reshape(st.shape)
    g_own, r_own = S.unpack_owned(grid, got), S.unpack_owned(grid, ref)
    for k in range(nc):
        err = np.abs(g_own[k] - r_own[k]).max() / np.abs(r_own[k]).max()
        assert err < TOL[prec] * (steps if prec == 1 else 1), (k, err)
        if prec == 0:
            assert abs(g_own[k, S.AVG].sum() - own[k, S.AVG].sum()) < 1e-11 * np.abs(own[k, S.AVG]).sum()


@pytest.mark.parametrize("prec", [0, 1])
def test_flux_registers_match_oracle(af, prec):
    """dt * F on the four patch faces accumulated in FP64 registers."""
    n, npatch = 16, 2
    lay = S.Layout(n, 3)
    st = S.random_state(lay, npatch, seed=9)
    st = st.astype(np.float32).astype(np.float64) if prec else st
    dx = dy = 1.0 / n
    dt = 0.4 * dx
    cf = O.cfg(1, n, dx, dy, dt, c=1.0)
    ref = np.zeros((npatch, 4, 3, n))
    for p in range(npatch):
        fr = np.zeros(4 * 3 * n)
        O.step_patch(cf, st[p], fr)
        O.step_patch(cf, st[p], fr)  # accumulates twice
        ref[p] = fr.reshape(4, 3, n)
    cfg = af.config(1, prec, n, c=1.0)
    work = af.build_step_work(cfg, np.arange(npatch))
    tdt = torch.float64 if prec == 0 else torch.float32
    din = torch.from_numpy(st.reshape(npatch, -1)).to(tdt).cuda()
    dout = din.clone()
    freg = torch.zeros((npatch, 4, 3, n), dtype=torch.float64, device="cuda")
    wd = torch.from_numpy(work).cuda()
    af.patch_step(cfg, wd, len(work) // 64, din, dout, dt, dx, dy, freg)
    af.patch_step(cfg, wd, len(work) // 64, din, dout, dt, dx, dy, freg)
    torch.cuda.synchronize()
    got = freg.cpu().numpy()
    err = np.abs(got - ref).max() / np.abs(ref).max()
    assert err < TOL[prec]


def test_config1_full_run_matches_oracle_and_exact(af):
    """2-D advection, a = (1, 0.5), one periodic 64 x 64 patch, FP64, smooth
    datum sin(2 pi x) sin(2 pi y) + Gaussian (sigma 0.05), CFL 0.4, T = 1:
    the whole run matches the oracle and its L1 error against the exact
    translated solution equals the oracle's."""
    from paper_2205_07572_gb300.uniform import UniformRun
    n = 64
    grid = S.UniformGrid(S.Layout(n, 1), 1, 1)
    st = grid.state([S.sinsin_plus_gaussian], nq=5)
    ns, dt = S.steps_to(1.0, S.cfl_dt("advection", 0.4, grid.dx, grid.dy, 1.0, 0.5))
    ref = O.run_uniform(O.cfg(0, n, grid.dx, grid.dy, dt, 1.0, 0.5), 1, 1, ns, st)
    run = UniformRun(af.config(0, 0, n, 1.0, 0.5), 1, 1, grid.dx, grid.dy, dt, state=np.nan_to_num(st))
    for _ in range(ns):
        run.step()
    torch.cuda.synchronize()
    got = run.state.cpu().numpy().reshape(st.shape)
    g, r = S.unpack_owned(grid, got), S.unpack_owned(grid, ref)
    assert np.abs(g - r).max() / np.abs(r).max() < 1e-12
    ex = S.translated(S.sinsin_plus_gaussian, 1.0, 0.5, 1.0)
    e_gpu, e_orc = grid.l1_error(got, 0, ex), grid.l1_error(ref, 0, ex)
    assert abs(e_gpu - e_orc) < 1e-9 * e_orc
    assert e_gpu < 1e-3  # sanity only; the oracle's accuracy is pinned separately


@pytest.mark.parametrize("prec", [0, 1])
def test_config2_full_size_two_steps_match_oracle(af, prec):
    """2-D acoustics, 512 x 512 cells as 16 x 16 patches of 32 x 32 with two
    ghost layers, Gaussian pulse + stationary vortex, CFL 0.4 (the literal
    configuration; the benchmark's 4096^2 scale-up is checked on sampled
    patches below): two steps in the default tiling match the oracle on every
    interior DOF."""
    from paper_2205_07572_gb300.uniform import UniformRun
    n, P = 32, 16
    grid = S.UniformGrid(S.Layout(n, 3), P, P)
    st = grid.state(S.pulse_plus_vortex(), nq=3)
    if prec == 1:
        st = st.astype(np.float32).astype(np.float64)
    dt = S.cfl_dt("acoustics", 0.4, grid.dx, grid.dy)
    ref = O.run_uniform(O.cfg(1, n, grid.dx, grid.dy, dt, c=1.0), P, P, 2, st)
    run = UniformRun(af.config(1, prec, n, c=1.0), P, P, grid.dx, grid.dy, dt, state=np.nan_to_num(st))
    run.step()
    run.step()
    torch.cuda.synchronize()
    got = run.state.double().cpu().numpy().reshape(st.shape)
    g, r = S.unpack_owned(grid, got), S.unpack_owned(grid, ref)
    for k in range(3):
        assert np.abs(g[k] - r[k]).max() / np.abs(r[k]).max() < TOL[prec]


def test_lukacova_gpu_error_equals_oracle(af):
    """Lukacova acoustics (Section 4.5.1), level 2 (64^2 cells in 16^2
    patches), FP64, to t = 1: the GPU run's L1 errors equal the oracle's."""
    from paper_2205_07572_gb300.uniform import UniformRun
    n, P = 16, 4
    grid = S.UniformGrid(S.Layout(n, 3), P, P, (-1.0, -1.0), (1.0, 1.0))
    st = grid.state(S.lukacova_exact(0.0), nq=5)
    ns, dt = S.steps_to(1.0, S.cfl_dt("acoustics", 0.4, grid.dx, grid.dy))
    ref = O.run_uniform(O.cfg(1, n, grid.dx, grid.dy, dt, c=1.0), P, P, ns, st)
    run = UniformRun(af.config(1, 0, n, c=1.0), P, P, grid.dx, grid.dy, dt, state=np.nan_to_num(st))
    for _ in range(ns):
        run.step()
    torch.cuda.synchronize()
    got = run.state.cpu().numpy().reshape(st.shape)
    ex = S.lukacova_exact(1.0)
    for k in range(3):
        eg, eo = grid.l1_error(got, k, ex[k]), grid.l1_error(ref, k, ex[k])
        assert abs(eg - eo) < 1e-8 * eo, (k, eg, eo)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("eq,n", [(1, 32), (1, 16), (0, 32), (0, 8)])
def test_every_tiling_matches_oracle(af, prec, eq, n):
    """Every compiled tile shape (the autotuner's search space) gives the
    oracle's step, for patches that advance their ghost layer (own ghosts)
    and for interior-only patches with neighbour halos (periodic grid)."""
    from paper_2205_07572_gb300.uniform import UniformRun
    nc = 1 if eq == 0 else 3
    tdt = torch.float64 if prec == 0 else torch.float32
    a, b, c = 0.9, -0.4, 1.0
    # own ghosts
    lay = S.Layout(n, nc)
    st = S.random_state(lay, 2, seed=60 + n).astype(np.float32 if prec else np.float64).astype(np.float64)
    dx, dy = 1.0 / n, 1.3 / n
    dt = _dt(eq, 0.45, dx, dy, a, b, c)
    cf = O.cfg(eq, n, dx, dy, dt, a, b, c)
    ref = np.stack([O.step_patch(cf, st[p]) for p in range(2)])
    # periodic grid
    grid = S.UniformGrid(S.Layout(n, nc), 2, 2)
    own = S.random_owned(grid, seed=61 + n)
    if prec:
        own = own.astype(np.float32).astype(np.float64)
    pst = S.pack_owned(grid, own)
    pdt = _dt(eq, 0.45, grid.dx, grid.dy, a, b, c)
    pcf = O.cfg(eq, n, grid.dx, grid.dy, pdt, a, b, c)
    pref = S.unpack_owned(grid, O.run_uniform(pcf, 2, 2, 2, pst))
    cfg = af.config(eq, prec, n, a, b, c)
    for k in range(len(af.step_tilings())):
        if af.step_tilings()[k][3]:
            continue  # the persistent tiling is refused (test_abi)
        work = af.build_step_work(cfg, np.arange(2), tiling=k)
        din = torch.from_numpy(st.reshape(2, -1)).to(tdt).cuda()
        dout = din.clone()
        af.patch_step(cfg, torch.from_numpy(work).cuda(), len(work) // 64, din, dout, dt, dx, dy, tiling=k)
        torch.cuda.synchronize()
        got = dout.double().cpu().numpy().reshape(ref.shape)
        assert _normwise(got, ref, nc) < TOL[prec], ("own ghosts", k)
        run = UniformRun(cfg, 2, 2, grid.dx, grid.dy, pdt, state=np.nan_to_num(pst), tiling=k)
        for s_ in range(2):
            torch.cuda.synchronize()
            cur = np.nan_to_num(run.state.double().cpu().numpy().reshape(pst.shape))
            one = S.unpack_owned(grid, O.run_uniform(pcf, 2, 2, 1, cur))   # the oracle's step from the GPU's
            run.step()
            torch.cuda.synchronize()
            g = S.unpack_owned(grid, run.state.double().cpu().numpy().reshape(pst.shape))
            for comp in range(nc):
                err = np.abs(g[comp] - one[comp]).max() / np.abs(one[comp]).max()
                assert err < TOL[prec], ("periodic step", k, s_, comp, err)
        for comp in range(nc):
            err = np.abs(g[comp] - pref[comp]).max() / np.abs(pref[comp]).max()
            assert err < TOL[prec] * (2 if prec else 1), ("periodic", k, comp, err)


@pytest.mark.parametrize("bands", [1, 5, 16])
def test_host_state_step_matches_device_step(af, bands):
    """UniformRun.step_host (state in pinned host memory, banded copies
    overlapping the step) gives the device step's result bit for bit."""
    from paper_2205_07572_gb300.uniform import UniformRun
    n, px = 8, 16
    grid = S.UniformGrid(S.Layout(n, 3), px, px)
    st = S.periodic_state(grid, S.pulse_plus_vortex(), nq=2)
    cfg = af.config(af.ACOUSTICS, af.F64, n, c=1.0)
    dev = UniformRun(cfg, px, px, grid.dx, grid.dy, 0.4 * grid.dx, state=st)
    hrun = UniformRun(cfg, px, px, grid.dx, grid.dy, 0.4 * grid.dx, state=None)
    host = torch.from_numpy(st.reshape(dev.a.shape).copy()).pin_memory()
    for _ in range(3):
        dev.step()
        hrun.step_host(host, bands)
    torch.cuda.synchronize()
    got = host.numpy().reshape(st.shape)
    ref = dev.state.cpu().numpy().reshape(st.shape)
    assert np.array_equal(S.unpack_owned(grid, got), S.unpack_owned(grid, ref))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("steps", [7, 12])
def test_graph_replayed_steps_equal_eager_steps(af, prec, steps):
    """UniformRun.advance (pairs of steps replayed from one captured CUDA
    graph, an odd last step eagerly) gives the state of the same number of
    step() calls bit for bit; a second advance replays the same graph (from
    either buffer), and one after a change of the time step captures again."""
    from paper_2205_07572_gb300.uniform import UniformRun
    n, px = 32, 4
    grid = S.UniformGrid(S.Layout(n, 3), px, px)
    st = np.nan_to_num(S.periodic_state(grid, S.pulse_plus_vortex(), nq=2))
    cfg = af.config(af.ACOUSTICS, prec, n, c=1.0)
    eager = UniformRun(cfg, px, px, grid.dx, grid.dy, 0.4 * grid.dx, state=st)
    graph = UniformRun(cfg, px, px, grid.dx, grid.dy, 0.4 * grid.dx, state=st)
    for _ in range(2 * steps):
        eager.step()
    graph.advance(steps)
    assert graph._graph is not None
    graph.advance(steps)
    # a changed time step is captured again, not replayed with the old one
    eager.dt = graph.dt = 0.3 * grid.dx
    for _ in range(6):
        eager.step()
    graph.advance(6)
    torch.cuda.synchronize()
    assert abs(graph.t - eager.t) < 1e-12
    a, b = eager.state.cpu().numpy(), graph.state.cpu().numpy()
    assert np.isfinite(a).all()
    assert np.array_equal(S.unpack_owned(grid, a.reshape(st.shape).astype(np.float64)),
                          S.unpack_owned(grid, b.reshape(st.shape).astype(np.float64)))


def _resplit(work, n, cuts):
    """Work items of one full-width tile per row band: each patch's items
    replaced by tiles [cuts[k], cuts[k + 1]) x [0, n)."""
    w = np.frombuffer(work.tobytes(), dtype=np.int32).reshape(-1, 16).copy()
    first = w[np.unique(w[:, 0], return_index=True)[1]]
    out = []
    for item in first:
        for y0, y1 in zip(cuts[:-1], cuts[1:]):
            it = item.copy()
            h = it.view(np.int16)
            h[20:24] = [0, n, y0, y1]
            out.append(it)
    return np.ascontiguousarray(np.stack(out)).view(np.uint8).reshape(-1)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("eq,n,k", [(1, 32, 3), (0, 32, 3), (1, 32, 0), (1, 16, 4), (0, 16, 4), (1, 18, 6), (0, 18, 7),
                                    (1, 10, 8), (1, 16, 9)])
def test_bulk_staging_equals_elementwise_staging(af, prec, eq, n, k):
    """Full-width tiles whose window is staged by bulk (TMA) copies plus the
    neighbours' halo, and tiles staged element by element, give the same
    step bit for bit in one kernel: the row bands of the second and third
    work lists start on rows whose 16-byte phase differs from row 0's (the
    element-wise path) or equals it (bulk), and all three agree with the
    oracle.  No bounded wait gives up.  Compared: the owned degrees of
    freedom (the ghost ring of such patches is not kept)."""
    from paper_2205_07572_gb300.uniform import UniformRun
    nc = 1 if eq == 0 else 3
    tdt = torch.float64 if prec == 0 else torch.float32
    grid = S.UniformGrid(S.Layout(n, nc), 3, 3)
    own = S.random_owned(grid, seed=90 + n + eq)
    if prec:
        own = own.astype(np.float32).astype(np.float64)
    pst = S.pack_owned(grid, own)
    dt = _dt(eq, 0.45, grid.dx, grid.dy, 0.9, -0.4, 1.0)
    pref = S.unpack_owned(grid, O.run_uniform(O.cfg(eq, n, grid.dx, grid.dy, dt, 0.9, -0.4, 1.0), 3, 3, 1, pst))
    cfg = af.config(eq, prec, n, 0.9, -0.4, 1.0)
    run = UniformRun(cfg, 3, 3, grid.dx, grid.dy, dt, state=np.nan_to_num(pst), tiling=k)
    tmy = af.step_tilings()[k][1]
    odd = [0] + list(range(tmy - 3, n, tmy)) + [n]            # starts 0 (bulk), tmy-3, ... (element-wise)
    four = [0] + list(range(4, n, tmy)) + [n]                 # every start a multiple of 4: all bulk
    af.step_wait_timeouts(reset=True)
    outs = []
    for work in (run.work.cpu().numpy(), _resplit(run.work.cpu().numpy(), n, odd),
                 _resplit(run.work.cpu().numpy(), n, four)):
        din = run.a.clone()
        dout = din.clone()
        af.patch_step(cfg, torch.from_numpy(work).cuda(), len(work) // 64, din, dout, dt, grid.dx, grid.dy,
                      tiling=k)
        torch.cuda.synchronize()
        outs.append(np.nan_to_num(dout.cpu().numpy()))
    # the owned degrees of freedom; the ghost ring of a patch with eight
    # same-level neighbours is not kept (bulk-staged tiles write whole rows)
    own = [S.unpack_owned(grid, o.astype(np.float64).reshape(pst.shape)) for o in outs]
    assert all(np.array_equal(own[0][c], o[c]) for o in own[1:] for c in range(nc))
    g = own[0]
    for comp in range(nc):
        err = np.abs(g[comp] - pref[comp]).max() / np.abs(pref[comp]).max()
        assert err < TOL[prec], (comp, err)
    assert af.step_wait_timeouts() == 0


@pytest.mark.parametrize("px", [3, 48])
def test_bulk_wait_timeout_is_reported(af, px):
    """Failure injection from the host: one work item carries
    AF_WORK_SKIP_BULK_COPY, so its bulk copies are never issued and its
    bounded wait (about a second) runs out.  Nothing faults: the tile's
    outputs stay unwritten, every other tile is exact, af_step_wait_timeouts
    reports one timeout, and the next step is normal."""
    from paper_2205_07572_gb300.uniform import UniformRun
    n = 32
    grid = S.UniformGrid(S.Layout(n, 3), px, px)
    pst = S.pack_owned(grid, S.random_owned(grid, seed=5).astype(np.float32).astype(np.float64))
    cfg = af.config(af.ACOUSTICS, af.F32, n, c=1.0)
    k = af.step_tilings().index((32, 8, 128, 0))
    run = UniformRun(cfg, px, px, grid.dx, grid.dy, 0.4 * grid.dx, state=np.nan_to_num(pst), tiling=k)
    work = run.work.cpu().numpy()
    items = np.frombuffer(work.tobytes(), dtype=np.int32).reshape(-1, 16).copy()
    victim = 4
    items[victim, 12] |= af.WORK_SKIP_BULK_COPY
    bad = np.ascontiguousarray(items).view(np.uint8).reshape(-1)

    def step(w):
        out = torch.full_like(run.a, 7.0)
        af.patch_step(cfg, torch.from_numpy(w).cuda(), len(w) // 64, run.a, out, run.dt, grid.dx, grid.dy, tiling=k)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    ref = step(work)
    af.step_wait_timeouts(reset=True)
    got = step(bad)
    assert af.step_wait_timeouts(reset=True) == 1
    p = items[victim, 0]
    y0, y1 = items[victim].view(np.int16)[22:24]
    diff = np.nonzero((got != ref).any(axis=1))[0]
    assert p in diff.tolist() and ((got == ref) | (got == 7.0)).all()
    assert diff.tolist() == [p]
    lay = S.Layout(n, 3)
    avg = lay.lattice(got[p].reshape(1, 3, 4, -1))[0, :, 0]          # [comp, J, I]
    assert (avg[:, S.G + y0:S.G + y1, S.G:S.G + n] == 7.0).all()
    assert np.array_equal(step(work), ref)
    assert af.step_wait_timeouts() == 0


def _pack_periodic(grid, owned):
    """pack_owned with the ghost ring filled from the periodic neighbours."""
    lay = grid.layout
    n, g = lay.n, S.G
    st = lay.empty(grid.npatch)
    lat = lay.lattice(st)
    loc = np.arange(lay.w) - g
    X, Y = grid.px * n, grid.py * n
    for p in range(grid.npatch):
        ix, iy = p % grid.px, p // grid.px
        gx, gy = (ix * n + loc) % X, (iy * n + loc) % Y
        lat[p] = owned[:, :, gy[:, None], gx[None, :]]
    return np.nan_to_num(st)


@pytest.mark.parametrize("prec", [0, 1])
def test_bulk_tiles_read_own_ghosts_where_no_neighbour_is_listed(af, prec):
    """A bulk-staged tile whose work item lists no neighbour on a side takes
    that side's halo -- ghost rows included -- from the patch's own ghost
    ring.  With the ring filled periodically the step equals the one with all
    eight neighbours listed, bit for bit."""
    from paper_2205_07572_gb300.uniform import UniformRun
    n, px = 32, 3
    grid = S.UniformGrid(S.Layout(n, 3), px, px)
    own = S.random_owned(grid, seed=21)
    if prec:
        own = own.astype(np.float32).astype(np.float64)
    st = _pack_periodic(grid, own)
    cfg = af.config(af.ACOUSTICS, prec, n, c=1.0)
    k = af.step_tilings().index((32, 8, 128, 0))
    run = UniformRun(cfg, px, px, grid.dx, grid.dy, 0.4 * grid.dx, state=st, tiling=k)
    base = run.work.cpu().numpy()
    items = np.frombuffer(base.tobytes(), dtype=np.int32).reshape(-1, 16).copy()
    h = items.view(np.int16)
    for it, hh in zip(items, h):
        p = it[0]
        if hh[22] == 0 and p % 2 == 0:
            it[4] = -1                        # no S neighbour listed
        if hh[23] == n and p % 3 == 0:
            it[9] = -1                        # no NE neighbour listed
        if p % 4 == 1:
            it[2] = -1                        # no W neighbour listed
    cut = np.ascontiguousarray(items).view(np.uint8).reshape(-1)
    outs = []
    for w in (base, cut):
        dout = torch.zeros_like(run.a)
        af.patch_step(cfg, torch.from_numpy(w).cuda(), len(w) // 64, run.a, dout, run.dt, grid.dx, grid.dy, tiling=k)
        torch.cuda.synchronize()
        outs.append(S.unpack_owned(grid, dout.double().cpu().numpy().reshape(st.shape)))
    assert np.array_equal(outs[0], outs[1])
    assert af.step_wait_timeouts() == 0


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n", [8, 32])
def test_pack_and_unpack_owned_match_the_layout(af, prec, n):
    """af_pack_owned gathers exactly the owned entries (i, j in [0, n) of every
    plane) into [patch][comp][plane][n][n]; af_unpack_owned scatters them back
    and leaves the ghost ring and padding untouched.  Bit for bit."""
    nc, npatch = 3, 5
    cfg = af.config(af.ACOUSTICS, prec, n, c=1.0)
    tdt = torch.float64 if prec == 0 else torch.float32
    lay = S.Layout(n, nc)
    rng = np.random.default_rng(n)
    st = torch.from_numpy(rng.normal(size=(npatch, af.patch_words(n, nc)))).to(tdt).cuda()
    own = torch.empty((npatch, af.owned_words(n, nc)), dtype=tdt, device="cuda")
    af.pack_owned(cfg, npatch, st, own)
    torch.cuda.synchronize()
    lat = lay.lattice(st.cpu().numpy().reshape(npatch, nc, 4, -1))
    ref = lat[..., S.G:S.G + n, S.G:S.G + n].reshape(npatch, -1)
    assert np.array_equal(own.cpu().numpy(), ref)
    back = torch.full_like(st, 3.0)
    af.unpack_owned(cfg, npatch, own, back)
    torch.cuda.synchronize()
    b = back.cpu().numpy().reshape(npatch, nc, 4, -1)
    blat = lay.lattice(b)
    assert np.array_equal(blat[..., S.G:S.G + n, S.G:S.G + n], lat[..., S.G:S.G + n, S.G:S.G + n])
    mask = np.ones(b.shape, bool)
    lay.lattice(mask)[..., S.G:S.G + n, S.G:S.G + n] = False
    assert (b[mask] == 3.0).all()


@pytest.mark.parametrize("bands", [1, 5, 16])
def test_host_owned_step_matches_device_step(af, bands):
    """UniformRun.step_host_owned (compact owned state in pinned host memory,
    banded copies, unpack / step / pack on the device) gives the device step's
    owned entries bit for bit, three steps running."""
    from paper_2205_07572_gb300.uniform import UniformRun
    n, px = 16, 8
    grid = S.UniformGrid(S.Layout(n, 3), px, px)
    st = S.periodic_state(grid, S.pulse_plus_vortex(), nq=2)
    cfg = af.config(af.ACOUSTICS, af.F32, n, c=1.0)
    dev = UniformRun(cfg, px, px, grid.dx, grid.dy, 0.4 * grid.dx, state=st)
    hrun = UniformRun(cfg, px, px, grid.dx, grid.dy, 0.4 * grid.dx, state=None)
    own = torch.empty((grid.npatch, af.owned_words(n, 3)), dtype=torch.float32, device="cuda")
    af.pack_owned(cfg, grid.npatch, dev.a, own)
    host = own.cpu().pin_memory()
    for _ in range(3):
        dev.step()
        hrun.step_host_owned(host, bands)
    torch.cuda.synchronize()
    af.pack_owned(cfg, grid.npatch, dev.a, own)
    torch.cuda.synchronize()
    assert np.array_equal(host.numpy(), own.cpu().numpy())


@pytest.mark.parametrize("prec", [0, 1])
def test_fma_probe_computes_its_chains(af, prec):
    """af_fma_throughput (the ALU-roof probe) runs the chains it claims: every
    thread's stored sum equals the eight recurrences a <- a * m + c."""
    blocks, iters = 3, 50
    tdt, ndt = (torch.float64, np.float64) if prec == 0 else (torch.float32, np.float32)
    sink = torch.zeros(blocks * 256, dtype=tdt, device="cuda")
    af.fma_throughput(prec, blocks, iters, sink)
    torch.cuda.synchronize()
    got = sink.cpu().numpy().reshape(blocks, 256)
    t = np.arange(256)
    m, c = ndt(0.9999999), ndt(1e-7)
    ref = np.zeros(256, np.float64)
    for k in range(8):
        a = (ndt(1) + (t + k).astype(ndt) * ndt(1e-7)).astype(np.float64)
        for _ in range(iters):
            a = a * float(m) + float(c)
        ref += a
    tol = 1e-12 if prec == 0 else 1e-5
    assert np.allclose(got, ref[None, :], rtol=tol, atol=0)
    assert af.lib().af_fma_probe_threads() == 256 * 8


@pytest.fixture(scope="module")
def bench_workload():
    """The benchmark's workload: 4096 x 4096 cells as 128 x 128 periodic
    patches of 32 x 32, Gaussian pulse + stationary vortex (FP64 state)."""
    grid = S.UniformGrid(S.Layout(32, 3), 128, 128)
    return grid, S.periodic_state(grid, S.pulse_plus_vortex(), nq=2, dtype=np.float64)


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
def test_bench_workload_full_size_sampled_patches_match_oracle(af, bench_workload, prec):
    """The benchmark's workload at full size, one step in the launch
    configuration it times (the 32 x 8-cell, 128-thread tiling: bulk-staged
    tiles, packed FP32x2 node evaluation, whole-row writes): sampled patches
    -- corners, edges, the pulse, the vortex -- match the oracle's single-patch
    step on the same input, every owned DOF, normwise against each
    component's largest value on the grid."""
    from paper_2205_07572_gb300.uniform import UniformRun
    grid, st64 = bench_workload
    n, P, nc = 32, 128, 3
    st = st64 if prec == 0 else st64.astype(np.float32)
    dt = 0.4 * grid.dx
    cfg = af.config(af.ACOUSTICS, prec, n, c=1.0)
    k = af.step_tilings().index((32, 8, 128, 0))
    run = UniformRun(cfg, P, P, grid.dx, grid.dy, dt, state=st, tiling=k)
    af.step_wait_timeouts(reset=True)
    run.step()
    torch.cuda.synchronize()
    samples = [0, P - 1, P * (P - 1), P * P - 1, P * 64 + 64, P * 64 + 20, P * 30 + 97, 12345]
    got = run.state[torch.tensor(samples, device="cuda")].double().cpu().numpy().reshape(len(samples), nc, 4, -1)
    lay = S.Layout(n, nc)
    lat = lay.lattice(st.reshape(P * P, nc, 4, -1).astype(np.float64))
    scale = [np.abs(lat[:, c, :, S.G:S.G + n, S.G:S.G + n]).max() for c in range(nc)]
    cf = O.cfg(1, n, grid.dx, grid.dy, dt, c=1.0)
    for i, p in enumerate(samples):
        patch = np.zeros((nc, 4, lay.plane))
        lay.lattice(patch)[...] = _patch_with_neighbour_halo(grid, lat, p)
        ref = lay.lattice(O.step_patch(cf, patch))[..., S.G:S.G + n, S.G:S.G + n]
        g = lay.lattice(got[i])[..., S.G:S.G + n, S.G:S.G + n]
        for c in range(nc):
            err = np.abs(g[c] - ref[c]).max() / scale[c]
            assert err < TOL[prec], (p, c, err)
    assert af.step_wait_timeouts() == 0


@pytest.mark.parametrize("neighbours", [False, True])
def test_whole_patch_bulk_staging_equals_elementwise_staging(af, neighbours):
    """FP32 16 x 16 patches that advance their first ghost layer: the 18 x 18
    tiling stages the whole patch lattice by one bulk copy per plane (window
    pitch = lattice width), the 18 x 10 tiling element by element; both give
    the same step bit for bit, with the patches' own ghost rings, and with
    same-level neighbours in some directions (their entries read from the
    neighbours)."""
    n, P, nc = 16, 6, 3
    lay = S.Layout(n, nc)
    st = S.random_state(lay, P, seed=321).astype(np.float32).reshape(P, -1)
    cfg = af.config(af.ACOUSTICS, af.F32, n, c=1.0)
    nbr = None
    if neighbours:   # a ring of six patches: W/E neighbours same-level, the rest not
        nbr = np.full((P, 8), -1, np.int32)
        for p in range(P):
            nbr[p, 0], nbr[p, 1] = (p - 1) % P, (p + 1) % P
        nbr[2, 1] = -1                      # patch 2 misses its E neighbour: extended anyway
    tl = [t[:3] for t in af.step_tilings()]
    dt = 0.4 / n
    outs = []
    af.step_wait_timeouts(reset=True)
    for k in (tl.index((18, 18, 256)), tl.index((18, 10, 192))):
        work = af.build_step_work(cfg, np.arange(P), nbr=nbr, tiling=k)
        w = np.frombuffer(work.tobytes(), dtype=np.int16).reshape(-1, 32)
        assert (w[:, 20] == -1).all() and (w[:, 21] == n + 1).all()    # every item covers [-1, n+1) in x
        din = torch.from_numpy(st).cuda()
        dout = din.clone()
        af.patch_step(cfg, torch.from_numpy(work).cuda(), len(work) // 64, din, dout, dt, 1.0 / n, 1.0 / n,
                      tiling=k)
        torch.cuda.synchronize()
        outs.append(dout.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert af.step_wait_timeouts() == 0
