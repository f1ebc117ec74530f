"""Parity of the adaptive-mesh entry points (af_fill_ghosts, af_transfer,
af_reflux, af_tag, af_mass) and of whole subcycled runs with the FP64 oracle,
through the C ABI.  FP64 1e-12, FP32 1e-5 (normwise relative; runs of K
coarse steps as fp32_parity states: each coarse step from the GPU's own FP32
state within 1e-5, the trajectory within K x 1e-5)."""
import numpy as np
import pytest

import oracle as O
import synth as S
from fp32_parity import lockstep_amr
from oracle.amr import OracleForest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

G = S.G
TOL = {0: 1e-12, 1: 1e-5}


@pytest.fixture(scope="module")
def af():
    from paper_2205_07572_gb300 import af as _af, build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _af


def _diag_forest(lmin, lmax, extra=None):
    def pred(l, ix, iy):
        return ix == iy or (extra is not None and extra(l, ix, iy))
    return S.balanced_forest(1, lmin, lmax, pred)


def _ip(a):
    import ctypes
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _oracle_fill(leaves, lmax, n, nc, st, dst, src, same_only=0):
    lv = np.array([l for l, _, _ in leaves], np.int32)
    ix = np.array([x for _, x, _ in leaves], np.int32)
    iy = np.array([y for _, _, y in leaves], np.int32)
    out = np.empty_like(st)
    O.lib().orc_fill_amr(n, nc, len(leaves), _ip(lv), _ip(ix), _ip(iy), 1, lmax, dst, src, same_only,
                         O._dp(st), O._dp(out))
    return out


def _device_forest(af, leaves, lmax):
    from paper_2205_07572_gb300.amr import Forest
    return Forest(1, lmax, leaves)


def _sorted(leaves):
    return sorted(leaves, key=lambda t: (t[0], t[2], t[1]))


def _nerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("eq", [0, 1])
def test_fill_matches_oracle(af, eq, prec):
    n, lmax = 8, 4
    nc = 1 if eq == 0 else 3
    leaves = _sorted(_diag_forest(2, 4, lambda l, x, y: l == 3 and x == 5 and y == 2))
    st = S.random_state(S.Layout(n, nc), len(leaves), seed=31).reshape(len(leaves), -1)
    if prec:
        st = st.astype(np.float32).astype(np.float64)
    allm = (1 << (lmax + 1)) - 1
    ref = _oracle_fill(leaves, lmax, n, nc, st, allm, allm)
    F = _device_forest(af, leaves, lmax)
    cfg = af.config(eq, prec, n, 1.0, 0.5, 1.0)
    d = torch.from_numpy(st).to(torch.float64 if prec == 0 else torch.float32).cuda()
    af.fill_ghosts(cfg, F.c, allm, allm, af.FILL_ALL_PATCHES, d)
    torch.cuda.synchronize()
    got = d.double().cpu().numpy()
    assert _nerr(got, ref) < TOL[prec]
    # same-level-only exchange of one level
    ref2 = _oracle_fill(leaves, lmax, n, nc, st, 1 << 3, 1 << 3, 1)
    d2 = torch.from_numpy(st).to(d.dtype).cuda()
    af.fill_ghosts(cfg, F.c, 1 << 3, 1 << 3, af.FILL_ALL_PATCHES | af.FILL_SAME_LEVEL_ONLY, d2)
    torch.cuda.synchronize()
    assert _nerr(d2.double().cpu().numpy(), ref2) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_transfer_matches_oracle(af, prec):
    from paper_2205_07572_gb300.amr import regrid_leaves
    n, lmax, nc = 8, 4, 3
    leaves = _sorted(_diag_forest(1, 3))
    st = S.random_state(S.Layout(n, nc), len(leaves), seed=5).reshape(len(leaves), -1)
    if prec:
        st = st.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(2)
    tags = rng.choice([-1, -1, 0, 1], size=len(leaves)).astype(np.int8)
    F = _device_forest(af, leaves, lmax)
    new = regrid_leaves(F, tags, 1)
    assert new != leaves
    lv = lambda L_, k: np.array([t[k] for t in L_], np.int32)
    ref = np.zeros((len(new), st.shape[1]))
    O.lib().orc_transfer(n, nc, 1, lmax, len(leaves), _ip(lv(leaves, 0)), _ip(lv(leaves, 1)), _ip(lv(leaves, 2)),
                         O._dp(st), len(new), _ip(lv(new, 0)), _ip(lv(new, 1)), _ip(lv(new, 2)), O._dp(ref))
    Fn = _device_forest(af, new, lmax)
    cfg = af.config(1, prec, n, c=1.0)
    tdt = torch.float64 if prec == 0 else torch.float32
    d_old = torch.from_numpy(st).to(tdt).cuda()
    d_new = torch.zeros((len(new), st.shape[1]), dtype=tdt, device="cuda")
    af.transfer(cfg, F.c, d_old, Fn.c, d_new)
    torch.cuda.synchronize()
    got = d_new.double().cpu().numpy()
    lay = S.Layout(n, nc)
    g = lay.lattice(got.reshape(len(new), nc, 4, -1))[..., G:G + n, G:G + n]
    r = lay.lattice(ref.reshape(len(new), nc, 4, -1))[..., G:G + n, G:G + n]
    assert _nerr(g, r) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_reflux_matches_oracle(af, prec):
    n, lmax, nc = 8, 3, 3
    leaves = _sorted(_diag_forest(2, 3))
    st = S.random_state(S.Layout(n, nc), len(leaves), seed=8).reshape(len(leaves), -1)
    if prec:
        st = st.astype(np.float32).astype(np.float64)
    freg = np.random.default_rng(4).uniform(-1, 1, size=(len(leaves), 4 * nc * n))
    lv = np.array([l for l, _, _ in leaves], np.int32)
    ix = np.array([x for _, x, _ in leaves], np.int32)
    iy = np.array([y for _, _, y in leaves], np.int32)
    ref_st, ref_fr = st.copy(), freg.copy()
    O.lib().orc_reflux_amr(n, nc, len(leaves), _ip(lv), _ip(ix), _ip(iy), 1, lmax, 0b1100, 0.125, 0.125,
                           O._dp(ref_fr), O._dp(ref_st))
    F = _device_forest(af, leaves, lmax)
    cfg = af.config(1, prec, n, c=1.0)
    d = torch.from_numpy(st).to(torch.float64 if prec == 0 else torch.float32).cuda()
    dfr = torch.from_numpy(freg).cuda()
    af.reflux(cfg, F.c, 0b1100, 0.125, 0.125, dfr, d)
    torch.cuda.synchronize()
    assert np.array_equal(dfr.cpu().numpy() == 0, ref_fr == 0)
    assert _nerr(dfr.cpu().numpy(), ref_fr) < 1e-15
    assert _nerr(d.double().cpu().numpy(), ref_st) < TOL[prec]


@pytest.mark.parametrize("kind", [0, 1])
def test_tag_and_mass_match_oracle(af, kind):
    n, lmax, nc = 16, 3, 3
    leaves = _sorted(_diag_forest(2, 3))
    st = S.forest_state(n, nc, 1, lmax, leaves, S.pulse_plus_vortex(), nq=2).reshape(len(leaves), -1)
    lv = np.array([l for l, _, _ in leaves], np.int32)
    tags_ref = np.zeros(len(leaves), np.int8)
    ind_ref = np.zeros(len(leaves))
    import ctypes
    thr = (0.05, 0.01) if kind == 0 else (2.0, 0.5)
    O.lib().orc_tag(n, nc, len(leaves), _ip(lv), O._dp(st), 0, kind, 1 / 16, 1 / 16, thr[0], thr[1],
                    tags_ref.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), O._dp(ind_ref))
    m_ref = np.zeros(nc)
    O.lib().orc_mass(n, nc, len(leaves), _ip(lv), O._dp(st), 1 / 16, 1 / 16, O._dp(m_ref))
    F = _device_forest(af, leaves, lmax)
    cfg = af.config(1, 0, n, c=1.0)
    d = torch.from_numpy(st).cuda()
    t = torch.zeros(len(leaves), dtype=torch.int8, device="cuda")
    ind = torch.zeros(len(leaves), dtype=torch.float64, device="cuda")
    af.tag(cfg, F.c, d, 0, kind, 1 / 16, 1 / 16, thr[0], thr[1], t, ind)
    scratch = torch.zeros(af.mass_scratch_bytes(len(leaves), nc) // 8, dtype=torch.float64, device="cuda")
    m = torch.zeros(nc, dtype=torch.float64, device="cuda")
    af.mass(cfg, F.c, d, 1 / 16, 1 / 16, scratch, m)
    torch.cuda.synchronize()
    assert np.array_equal(t.cpu().numpy(), tags_ref)
    assert _nerr(ind.cpu().numpy(), ind_ref) < 1e-13
    assert np.abs(m.cpu().numpy() - m_ref).max() < 1e-13 * max(1.0, np.abs(m_ref).max())
    assert (tags_ref == 1).any() and (tags_ref != 1).any()


def _runs(af, eq, prec, n, lmin, lmax, funcs, cfl, leaves=None, mode="batched", graphs=False):
    from paper_2205_07572_gb300.amr import AMRRun
    nc = 1 if eq == 0 else 3
    leaves = leaves or _sorted(_diag_forest(lmin, lmax))
    st = S.forest_state(n, nc, 1, lmax, leaves, funcs, nq=3)
    if prec:
        st = st.astype(np.float32).astype(np.float64)
    dx0 = 1.0 / n
    dt0 = cfl * dx0 / (1.0 if eq == 0 else 1.0)
    Fo = OracleForest(eq, n, 1, lmax, leaves, (0, 0), (1, 1), dt0, 1.0, 0.5, 1.0, state=st)
    Fo.sync_fill((1 << (lmax + 1)) - 1)
    run = AMRRun(af.config(eq, prec, n, 1.0, 0.5, 1.0), 1, lmax, leaves, st, (0, 0), (1, 1), dt0, mode=mode,
                 graphs=graphs)
    return Fo, run


def _compare(Fo, run, n, nc, tol):
    got = run.state_in_order(Fo.leaves)
    lay = S.Layout(n, nc)
    g = lay.lattice(got.reshape(len(Fo.leaves), nc, 4, -1))[..., G:G + n, G:G + n]
    r = lay.lattice(Fo.state.reshape(len(Fo.leaves), nc, 4, -1))[..., G:G + n, G:G + n]
    for c in range(nc):
        assert _nerr(g[:, c], r[:, c]) < tol, (c, _nerr(g[:, c], r[:, c]))


@pytest.mark.parametrize("mode", ["batched", "per_level", "per_patch"])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("eq", [0, 1])
def test_subcycled_amr_run_matches_oracle(af, eq, prec, mode):
    """Fixed diagonal forest, levels 2-3, several coarse steps with
    subcycling, reflux and ghost exchange (Section 3.2), in each of the
    driver's launch modes."""
    n = 8
    funcs = [S.sinsin_plus_gaussian] if eq == 0 else S.pulse_plus_vortex()
    Fo, run = _runs(af, eq, prec, n, 2, 3, funcs, 0.6 if eq == 0 else 0.4, mode=mode)
    m0 = run.mass()
    nc = 1 if eq == 0 else 3
    lockstep_amr(Fo, run, 3, lambda F, tol: _compare(F, run, n, nc, tol), prec, torch.cuda.synchronize)
    if prec == 0:
        assert np.abs(run.mass() - m0).max() < 1e-13 * max(1.0, np.abs(m0).max())


def test_three_level_amr_run_matches_oracle(af):
    """Levels 2-4 (Fig. subcycle's three-level schedule), FP64 acoustics."""
    n = 8
    leaves = _sorted(S.balanced_forest(1, 2, 4, lambda l, x, y: x == y))
    Fo, run = _runs(af, 1, 0, n, 2, 4, S.pulse_plus_vortex(), 0.4, leaves=leaves)
    for _ in range(2):
        Fo.coarse_step()
        run.coarse_step()
    torch.cuda.synchronize()
    _compare(Fo, run, n, 3, 1e-12)


@pytest.mark.parametrize("prec", [0, 1])
def test_dynamic_regrid_run_matches_oracle(af, prec):
    """Coarse steps with a regrid after each (range indicator, Section 4.1's
    criterion) on both sides: same forests, same data."""
    n, lmin, lmax = 8, 2, 4
    f = lambda x, y: np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / 0.01)
    leaves = _sorted(S.balanced_forest(1, lmin, lmin, lambda *a: False))
    Fo, run = _runs(af, 0, prec, n, lmin, lmax, [f], 0.6, leaves=leaves)
    for it in range(3):
        if prec:   # FP32: this coarse step (regrid included) from the GPU's own state
            torch.cuda.synchronize()
            Fo.state = np.nan_to_num(run.state_in_order(Fo.leaves)).reshape(Fo.state.shape)
        to, _ = Fo.tags(0, 0, 0.05, 0.01)
        tg, _ = run.tags(0, 0, 0.05, 0.01)
        order = {leaf: k for k, leaf in enumerate(run.forest.leaves)}
        assert np.array_equal(tg[[order[l] for l in Fo.leaves]], to)
        Fo.regrid(to, lmin)
        run.regrid(tg, lmin)
        assert Fo.leaves == run.forest.leaves
        Fo.coarse_step()
        run.coarse_step()
        torch.cuda.synchronize()
        if prec:
            _compare(Fo, run, n, 1, TOL[1])
    assert len(set(l for l, _, _ in Fo.leaves)) >= 2
    _compare(Fo, run, n, 1, TOL[prec])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_regrid_transfer_matches_oracle_and_is_exact_for_biquadratics(af, seed):
    """Random refine / coarsen tags on a biquadratic (levels 2-4): after each
    regrid (af_forest_regrid, af_transfer, exchange) every cell average and
    every point value on the leaves' left and bottom lines and inside them
    equals the oracle's regrid, and is exact on the leaves in [1/4, 3/4]^2
    (the data are not periodic, so cells on the periodic seam are not).  A
    refined leaf owns the nodes on its right and top faces where the
    neighbour across is coarser; they reach that neighbour's left and bottom
    lines through the exchange, so a transfer that left them unset fails
    here."""
    from paper_2205_07572_gb300.amr import AMRRun
    f = lambda x, y: 0.3 + x - 2 * y + 1.5 * x * y + x * x - 0.5 * y * y + x * x * y - 2 * x * y * y \
        + 3 * x * x * y * y
    n, lmin, lmax = 8, 2, 4
    leaves = _sorted(S.balanced_forest(1, lmin, 3, lambda l, x, y: (x + y) % 3 == 0))
    st = S.forest_state(n, 1, 1, lmax, leaves, [f], nq=3)
    Fo = OracleForest(0, n, 1, lmax, leaves, (0, 0), (1, 1), 0.01, 1.0, 0.5, state=st)
    Fo.sync_fill((1 << (lmax + 1)) - 1)
    run = AMRRun(af.config(0, 0, n, 1.0, 0.5), 1, lmax, leaves, st, (0, 0), (1, 1), 0.01)
    rng = np.random.default_rng(seed)
    lay = S.Layout(n, 1)
    exact_leaves = 0
    for _ in range(4):
        tags = rng.choice(np.array([-1, 0, 1], np.int8), size=len(Fo.leaves), p=[0.45, 0.25, 0.3])
        order = {leaf: k for k, leaf in enumerate(Fo.leaves)}
        Fo.regrid(tags, lmin)
        run.regrid(tags[[order[lf] for lf in run.forest.leaves]], lmin)
        assert Fo.leaves == run.forest.leaves
        torch.cuda.synchronize()
        g = lay.lattice(run.state_in_order(Fo.leaves).reshape(len(Fo.leaves), 1, 4, -1))[:, 0, :, G:G + n, G:G + n]
        r = lay.lattice(Fo.state.reshape(len(Fo.leaves), 1, 4, -1))[:, 0, :, G:G + n, G:G + n]
        assert np.abs(g - r).max() < 1e-12
        for p, (l, ix, iy) in enumerate(Fo.leaves):
            q = 1 << (l - 2)
            if not (q <= ix < 3 * q and q <= iy < 3 * q):
                continue
            w = 1.0 / (1 << l)
            h = w / n
            I = np.arange(n)
            for k in (S.CORNER, S.XMID, S.YMID):
                X, Y = np.meshgrid(ix * w + I * h + (0.5 * h if k == S.YMID else 0.0),
                                   iy * w + I * h + (0.5 * h if k == S.XMID else 0.0))
                assert np.abs(g[p, k] - f(X, Y)).max() < 1e-12, ((l, ix, iy), k)
            exact_leaves += 1
    assert exact_leaves > 20


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replayed_amr_run_matches_oracle(af, prec):
    """Levels 2-4, batched launches captured in CUDA graphs: the first coarse
    step from each level parity runs eagerly, the second is captured, the
    rest are replays -- six coarse steps exercise both graphs."""
    n = 8
    leaves = _sorted(S.balanced_forest(1, 2, 4, lambda l, x, y: x == y))
    Fo, run = _runs(af, 1, prec, n, 2, 4, S.pulse_plus_vortex(), 0.4, leaves=leaves, graphs=True)
    m0 = run.mass()
    lockstep_amr(Fo, run, 6, lambda F, tol: _compare(F, run, n, 3, tol), prec, torch.cuda.synchronize)
    assert len([g for g in run.graphs.values() if g is not None]) == 2
    if prec == 0:
        assert np.abs(run.mass() - m0).max() < 1e-13 * max(1.0, np.abs(m0).max())


def test_pair_entry_points_match_single_array(af):
    """af_*_pair on a state split between two arrays (levels 2 and 4 current
    in buf[1], level 3 in buf[0]; the stale entries are NaN) give the results
    of the single-array calls on the assembled state."""
    n, lmax, nc = 8, 4, 3
    leaves = _sorted(S.balanced_forest(1, 2, 4, lambda l, x, y: x == y))
    st = S.forest_state(n, nc, 1, lmax, leaves, S.pulse_plus_vortex(), nq=2).reshape(len(leaves), -1)
    st = np.nan_to_num(st)  # plane padding: only the stale halves hold NaN
    F = _device_forest(af, leaves, lmax)
    cfg = af.config(1, 0, n, c=1.0)
    parity = (1 << 2) | (1 << 4)
    one = torch.from_numpy(st).cuda()
    b0 = torch.full_like(one, float("nan"))
    b1 = torch.full_like(one, float("nan"))
    for l in F.levels:
        sl = F.level_slice(l)
        (b1 if (parity >> l) & 1 else b0)[sl] = one[sl]
    pair = af.state_pair(b0, b1, parity)

    def assemble():
        out = b0.clone()
        for l in F.levels:
            if (parity >> l) & 1:
                sl = F.level_slice(l)
                out[sl] = b1[sl]
        return out

    allm = (1 << (lmax + 1)) - 1
    af.fill_ghosts(cfg, F.c, allm, allm, 0, one)
    af.fill_ghosts_pair(cfg, F.c, allm, allm, 0, pair)
    freg = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, (len(leaves), 4 * nc * n))).cuda()
    freg2 = freg.clone()
    af.reflux(cfg, F.c, 0b11100, 1 / 8, 1 / 8, freg, one)
    af.reflux_pair(cfg, F.c, 0b11100, 1 / 8, 1 / 8, freg2, pair)
    torch.cuda.synchronize()
    assert torch.equal(assemble(), one)
    assert torch.equal(freg, freg2)
    t1 = torch.zeros(len(leaves), dtype=torch.int8, device="cuda")
    t2 = torch.zeros_like(t1)
    i1 = torch.zeros(len(leaves), dtype=torch.float64, device="cuda")
    i2 = torch.zeros_like(i1)
    af.tag(cfg, F.c, one, 0, 0, 1 / 8, 1 / 8, 0.05, 0.01, t1, i1)
    af.tag_pair(cfg, F.c, pair, 0, 0, 1 / 8, 1 / 8, 0.05, 0.01, t2, i2)
    sc = torch.zeros(af.mass_scratch_bytes(len(leaves), nc) // 8, dtype=torch.float64, device="cuda")
    m1 = torch.zeros(nc, dtype=torch.float64, device="cuda")
    m2 = torch.zeros_like(m1)
    af.mass(cfg, F.c, one, 1 / 8, 1 / 8, sc, m1)
    af.mass_pair(cfg, F.c, pair, 1 / 8, 1 / 8, sc, m2)
    torch.cuda.synchronize()
    assert torch.equal(t1, t2) and torch.equal(i1, i2) and torch.equal(m1, m2)
    from paper_2205_07572_gb300.amr import regrid_leaves
    new = regrid_leaves(F, np.where(np.arange(len(leaves)) % 3 == 0, 1, -1).astype(np.int8), 2)
    Fn = _device_forest(af, new, lmax)
    n1 = torch.zeros((len(new), st.shape[1]), dtype=torch.float64, device="cuda")
    n2 = torch.zeros_like(n1)
    af.transfer(cfg, F.c, one, Fn.c, n1)
    af.transfer_pair(cfg, F.c, pair, Fn.c, n2)
    torch.cuda.synchronize()
    assert torch.equal(n1, n2)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("eq", [0, 1])
def test_planned_fill_equals_direct_fill_bitwise(af, eq, prec):
    """af_fill_ghosts_planned == af_fill_ghosts bit for bit (all levels, and
    the synchronised sets of the finest two and three levels), on a state
    split between two arrays; the plan counts match the entries written."""
    n, lmax = 8, 4
    nc = 1 if eq == 0 else 3
    leaves = _sorted(_diag_forest(2, 4, lambda l, x, y: l == 3 and x == 5 and y == 2))
    st = np.nan_to_num(S.random_state(S.Layout(n, nc), len(leaves), seed=77).reshape(len(leaves), -1))
    F = _device_forest(af, leaves, lmax)
    cfg = af.config(eq, prec, n, 1.0, 0.5, 1.0)
    tdt = torch.float64 if prec == 0 else torch.float32
    plan, n_a, n_b = af.ghost_plan(cfg, F.c)
    assert n_a > 0 and n_b > 0
    allm = (1 << (lmax + 1)) - 1
    for levels in (allm, 0b11000, 0b11100):
        one = torch.from_numpy(st).to(tdt).cuda()
        af.fill_ghosts(cfg, F.c, levels, levels, 0, one)
        parity = 0b01010
        b0 = torch.from_numpy(st).to(tdt).cuda()
        b1 = torch.full_like(b0, float("nan"))
        for l in F.levels:
            if (parity >> l) & 1:
                sl = F.level_slice(l)
                b1[sl] = b0[sl]
                b0[sl] = float("nan")
        af.fill_ghosts_planned(cfg, F.c, levels, 0, plan, n_a, n_b, af.state_pair(b0, b1, parity))
        torch.cuda.synchronize()
        got = b0.clone()
        for l in F.levels:
            if (parity >> l) & 1:
                sl = F.level_slice(l)
                got[sl] = b1[sl]
        assert torch.equal(got, one), levels
    with pytest.raises(af.AFError):
        af.fill_ghosts_planned(cfg, F.c, 0b01100, 0, plan, n_a, n_b, af.state_pair(one, None, 0))


@pytest.mark.parametrize("prec", [0, 1])
def test_amr_run_with_bulk_staged_tiles_matches_oracle(af, prec):
    """16 x 16-cell patches in one 16 x 16 tile each: patches surrounded by
    same-level neighbours are staged by bulk (TMA) copies, patches that
    advance their ghost layer element by element; two subcycled coarse
    steps of acoustics agree with the oracle."""
    from paper_2205_07572_gb300.amr import AMRRun
    n, lmax = 16, 3
    leaves = _sorted(S.balanced_forest(1, 2, lmax, lambda l, x, y: x == y and x < 2))
    st = S.forest_state(n, 3, 1, lmax, leaves, S.pulse_plus_vortex(), nq=3)
    if prec:
        st = st.astype(np.float32).astype(np.float64)
    dx0 = 1.0 / n
    dt0 = 0.4 * dx0
    Fo = OracleForest(1, n, 1, lmax, leaves, (0, 0), (1, 1), dt0, 1.0, 0.5, 1.0, state=st)
    Fo.sync_fill((1 << (lmax + 1)) - 1)
    k = [t[:2] for t in af.step_tilings()].index((16, 16))
    run = AMRRun(af.config(1, prec, n, 1.0, 0.5, 1.0), 1, lmax, leaves, st, (0, 0), (1, 1), dt0, tiling=k)
    af.step_wait_timeouts(reset=True)
    lockstep_amr(Fo, run, 2, lambda F, tol: _compare(F, run, n, 3, tol), prec, torch.cuda.synchronize)
    assert af.step_wait_timeouts() == 0


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("graphs", [False, True])
def test_amr_run_with_a_second_tiling_for_extended_leaves(af, prec, graphs):
    """Leaves with eight same-level neighbours in one 16 x 16 tile each
    (bulk-staged), leaves that advance their ghost layer in one 18 x 18 tile
    (ext_tiling: a second work list, a second launch per substep); eager and
    graph-replayed subcycled coarse steps agree with the oracle."""
    from paper_2205_07572_gb300.amr import AMRRun
    n, lmax = 16, 3
    leaves = _sorted(S.balanced_forest(1, 2, lmax, lambda l, x, y: x == y and x < 2))
    st = S.forest_state(n, 3, 1, lmax, leaves, S.pulse_plus_vortex(), nq=3)
    if prec:
        st = st.astype(np.float32).astype(np.float64)
    dx0 = 1.0 / n
    dt0 = 0.4 * dx0
    Fo = OracleForest(1, n, 1, lmax, leaves, (0, 0), (1, 1), dt0, 1.0, 0.5, 1.0, state=st)
    Fo.sync_fill((1 << (lmax + 1)) - 1)
    tl = [t[:2] for t in af.step_tilings()]
    run = AMRRun(af.config(1, prec, n, 1.0, 0.5, 1.0), 1, lmax, leaves, st, (0, 0), (1, 1), dt0,
                 tiling=tl.index((16, 16)), ext_tiling=tl.index((18, 18)), graphs=graphs)
    assert len(run.work_groups) == 2 and all(nw > 0 for _, nw, _, _ in run.work_groups)
    lockstep_amr(Fo, run, 4, lambda F, tol: _compare(F, run, n, 3, tol), prec, torch.cuda.synchronize)


@pytest.mark.parametrize("case", ["advection_levels2-6", "acoustics_levels3-7"])
def test_bench_amr_workloads_conserve_mass_at_full_size(af, case):
    """The benchmark's adaptive workloads at full size (736 and 4944 leaves of
    16 x 16 cells, forests from the method's own tagging and regridding), in
    the launch configuration it times (batched, graph-replayed, 16 x 16
    tiles): FP64 mass is conserved to round-off over four coarse steps with
    subcycling, the conservative fix and the planned ghost exchange, on
    these periodic domains (Section 3.2)."""
    import bench
    from paper_2205_07572_gb300.amr import AMRRun
    leaves, st = bench.amr_initial(case)
    c = bench.AMR_CASES[case]
    n = bench.AMR_N
    dx0 = (c["hi"][0] - c["lo"][0]) / (c["B"] * n)
    dt0 = bench.CFL * dx0 / (max(abs(c["a"]), abs(c["b"])) if c["eq"] == 0 else 1.0)
    k = [t[:3] for t in af.step_tilings()].index((16, 16, 128))
    run = AMRRun(af.config(c["eq"], af.F64, n, c["a"], c["b"], 1.0), c["B"], c["lmax"], leaves, st, c["lo"],
                 c["hi"], dt0, graphs=True, tiling=k)
    assert run.forest.nleaf == len(leaves) and len(run.forest.levels) >= 3
    m0 = run.mass()
    for _ in range(4):
        run.coarse_step()
    torch.cuda.synchronize()
    m1 = run.mass()
    assert np.abs(m1 - m0).max() < 1e-12 * max(1.0, np.abs(m0).max()), (m0, m1)
    assert af.step_wait_timeouts() == 0


def _input_as_kernel_reads(lat, nbr, p, n):
    """Lattice of leaf p as the step kernel stages it: its own entries (ghost
    ring from the exchange), with every entry in a direction that has a
    same-level neighbour read from that neighbour's entry at the same place
    (the same-level ghost copy fused into the kernel's halo load)."""
    out = lat[p].copy()
    w = n + 2 * G + 1
    for J in range(w):
        for I in range(w):
            li, lj = I - G, J - G
            sx = -1 if li < 0 else (1 if li >= n else 0)
            sy = -1 if lj < 0 else (1 if lj >= n else 0)
            if sx == 0 and sy == 0:
                continue
            d = (0 if sx < 0 else 1) if sy == 0 else ((2 if sy < 0 else 3) if sx == 0 else
                                                       4 + (sx > 0) + 2 * (sy > 0))
            q = nbr[p, d]
            if q >= 0:
                out[:, :, J, I] = lat[q, :, :, lj - sy * n + G, li - sx * n + G]
    return out


@pytest.mark.parametrize("tile", [(16, 16, 128), (18, 18, 256), (18, 18, 128)])
@pytest.mark.parametrize("prec", [0, 1])
def test_bench_acoustics_forest_sampled_leaves_match_oracle(af, prec, tile):
    """The benchmark's acoustics forest at full size (levels 3-7, 4944
    leaves of 16 x 16 cells), in the launch configuration it times (batched
    work list, 16 x 16-cell tiles, after graph-replayed coarse steps) and in
    the default tiling of 16 x 16 patches (18 x 18 tiles: whole-patch bulk
    staging for leaves that advance their ghost layer): the
    first substep of a coarse step advances every level in one launch;
    sampled leaves of every level -- with and without coarser or finer
    neighbours -- equal the oracle's single-patch step on the input the
    kernel read, every interior average and point value (FP64 1e-12, FP32
    1e-5, normwise against each component's largest value on the
    samples)."""
    import bench
    from paper_2205_07572_gb300.amr import AMRRun
    case = "acoustics_levels3-7"
    leaves, st = bench.amr_initial(case)
    c = bench.AMR_CASES[case]
    n, nc = bench.AMR_N, 3
    dx0 = (c["hi"][0] - c["lo"][0]) / (c["B"] * n)
    dt0 = bench.CFL * dx0
    k = [t[:3] for t in af.step_tilings()].index(tile)
    run = AMRRun(af.config(1, prec, n, c=1.0), c["B"], c["lmax"], leaves, st, c["lo"], c["hi"], dt0,
                 graphs=True, tiling=k)
    assert run.forest.nleaf > 4000
    for _ in range(4):
        run.coarse_step()
    torch.cuda.synchronize()
    F = run.forest
    lay = S.Layout(n, nc)
    before = lay.lattice(run.current().double().cpu().numpy().reshape(F.nleaf, nc, 4, -1)).copy()
    af.step_wait_timeouts(reset=True)
    run.advance_from(F.levels[0])
    torch.cuda.synchronize()
    after = lay.lattice(run.current().double().cpu().numpy().reshape(F.nleaf, nc, 4, -1))
    assert af.step_wait_timeouts() == 0
    rng = np.random.default_rng(5)
    ext = (F.nbr < 0).any(axis=1)
    samples = []
    for l in F.levels:
        for kind in (True, False):
            idx = np.nonzero((F.level == l) & (ext == kind))[0]
            if len(idx):
                samples += rng.choice(idx, size=min(4, len(idx)), replace=False).tolist()
    assert ext[samples].any() and (~ext[samples]).any()
    got, ref = [], []
    for p in samples:
        l = int(F.level[p])
        cf = O.cfg(1, n, dx0 / (1 << l), dx0 / (1 << l), dt0 / (1 << l), c=1.0)
        patch = np.zeros((nc, 4, lay.plane))
        lay.lattice(patch)[...] = _input_as_kernel_reads(before, F.nbr, p, n)
        ref.append(lay.lattice(O.step_patch(cf, patch))[..., G:G + n, G:G + n])
        got.append(after[p][..., G:G + n, G:G + n])
    got, ref = np.array(got), np.array(ref)
    for comp in range(nc):
        err = np.abs(got[:, comp] - ref[:, comp]).max() / np.abs(ref[:, comp]).max()
        assert err < TOL[prec], (comp, err)


@pytest.mark.parametrize("tile", [(16, 16, 128), (18, 18, 256), (18, 18, 128)])
def test_regrid_where_a_neighbour_family_coarsens_matches_oracle(af, tile):
    """A leaf with eight same-level neighbours advances only its interior,
    so the copies it keeps of the point values on its right and top faces
    (owned then by its neighbours) are not current.  When the family to its
    right (or above) coarsens, the leaf becomes the owner of those values
    (Section 3.2: the finer grid's values on a coarse-fine face): the regrid
    must take them from their previous owners.  Two coarse steps, a regrid
    that coarsens the families right of and above an unchanged leaf, one
    more coarse step: equal to the oracle (FP64 1e-12)."""
    from paper_2205_07572_gb300.amr import AMRRun
    n, lmax = 16, 3
    block = {(x, y) for x in (1, 2, 3) for y in (1, 2, 3)}
    leaves = _sorted(S.balanced_forest(1, 2, lmax, lambda l, x, y: l == 2 and (x, y) in block))
    st = S.forest_state(n, 3, 1, lmax, leaves, S.pulse_plus_vortex(), nq=3)
    dx0 = 1.0 / n
    dt0 = 0.4 * dx0
    Fo = OracleForest(1, n, 1, lmax, leaves, (0, 0), (1, 1), dt0, 1.0, 0.5, 1.0, state=st)
    Fo.sync_fill((1 << (lmax + 1)) - 1)
    k = [t[:3] for t in af.step_tilings()].index(tile)
    run = AMRRun(af.config(1, 0, n, c=1.0), 1, lmax, leaves, st, (0, 0), (1, 1), dt0, tiling=k)
    assert (run.forest.nbr[run.forest.leaves.index((3, 5, 5))] >= 0).all()   # eight same-level neighbours
    for _ in range(2):
        Fo.coarse_step()
        run.coarse_step()
    # coarsen the families (level-2 parents) right of and above leaf (3, 5, 5)
    gone = {(3, 2), (2, 3)}
    tags = np.array([-1 if (l == 3 and (x // 2, y // 2) in gone) else 0 for (l, x, y) in Fo.leaves], np.int8)
    order = {leaf: i for i, leaf in enumerate(Fo.leaves)}
    Fo.regrid(tags, 2)
    run.regrid(tags[[order[lf] for lf in run.forest.leaves]], 2)
    assert Fo.leaves == run.forest.leaves and (2, 3, 2) in Fo.leaves and (3, 5, 5) in Fo.leaves
    Fo.coarse_step()
    run.coarse_step()
    torch.cuda.synchronize()
    _compare(Fo, run, n, 3, TOL[0])
