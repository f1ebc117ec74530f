"""Host-side AMR logic of the GPU driver (no GPU needed): the forest map, the
neighbour tables and the regrid rules, checked against the oracle's
independent implementation of the same rules and against direct geometry."""
import numpy as np
import pytest

import synth as S
from oracle.amr import new_leaves


@pytest.fixture(scope="module")
def amr():
    from paper_2205_07572_gb300 import amr as _amr, build
    build.build()
    return _amr


def _sorted(leaves):
    return sorted(leaves, key=lambda t: (t[0], t[2], t[1]))


@pytest.mark.parametrize("seed", range(6))
def test_regrid_rules_agree_with_oracle(amr, seed):
    rng = np.random.default_rng(seed)
    B, lmin, lmax = 1 + seed % 2, 1, 4
    leaves = _sorted(S.balanced_forest(B, lmin, 3, lambda l, x, y: rng.random() < 0.3))
    F = amr.Forest(B, lmax, leaves, device="cpu")
    for _ in range(3):
        tags = rng.choice([-1, -1, 0, 1], size=len(F.leaves)).astype(np.int8)
        mine = amr.regrid_leaves(F, tags, lmin)
        ref = new_leaves(F.leaves, tags, B, lmin, lmax)
        assert mine == ref
        F = amr.Forest(B, lmax, mine, device="cpu")


def test_forest_map_and_neighbours(amr):
    leaves = _sorted(S.balanced_forest(2, 1, 3, lambda l, x, y: x == y))
    F = amr.Forest(2, 3, leaves, device="cpu")
    for k, (l, x, y) in enumerate(F.leaves):
        assert F.region(l, x, y) == k
    nb = F.neighbours(range(F.nleaf))
    for k, (l, x, y) in enumerate(F.leaves):
        side = 2 << l
        for d, (sx, sy) in enumerate([(-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (1, -1), (-1, 1), (1, 1)]):
            key = (l, (x + sx) % side, (y + sy) % side)
            expect = F.leaves.index(key) if key in F.leaves else -1
            assert nb[k, d] == expect
    # every level-l slice is contiguous
    for l in F.levels:
        sl = F.level_slice(l)
        assert all(F.level[sl] == l)


def test_forest_from_arrays_in_any_order(amr):
    """Forest(arrays=) stores the leaves sorted by (level, row, column)
    whatever the input order, exactly as from the list of tuples."""
    leaves = _sorted(S.balanced_forest(2, 1, 4, lambda l, x, y: (x + y) % 3 == 0))
    F = amr.Forest(2, 4, leaves, device="cpu")
    perm = np.random.default_rng(3).permutation(len(leaves))
    arr = np.array(leaves, np.int32)[perm]
    G = amr.Forest(2, 4, device="cpu", arrays=(arr[:, 0], arr[:, 1], arr[:, 2]))
    assert G.leaves == F.leaves == leaves
    assert np.array_equal(G.nbr, F.nbr) and np.array_equal(G.map, F.map)
    assert G.same_leaves(arr[:, 0], arr[:, 1], arr[:, 2])
    assert not G.same_leaves(arr[1:, 0], arr[1:, 1], arr[1:, 2])


def test_forest_map_entries_by_direct_geometry(amr):
    """af_forest_build_map: at every level, a region that is a leaf holds its
    index, a region inside a coarser leaf q holds -2 - q, a region holding
    finer leaves holds -1 (checked region by region from the leaves'
    extents); a forest whose leaves overlap is refused."""
    from paper_2205_07572_gb300 import af
    B, lmax = 2, 3
    leaves = _sorted(S.balanced_forest(B, 1, 3, lambda l, x, y: x == y))
    F = amr.Forest(B, lmax, leaves, device="cpu")
    for l in range(lmax + 1):
        side = B << l
        off = F.offsets[l]
        for y in range(side):
            for x in range(side):
                got = int(F.map[off + y * side + x])
                inside = [k for k, (m, ix, iy) in enumerate(F.leaves)
                          if m <= l and (x >> (l - m)) == ix and (y >> (l - m)) == iy]
                if inside:
                    (k,) = inside
                    assert got == (k if F.leaves[k][0] == l else -2 - k), (l, x, y)
                else:
                    assert got == -1, (l, x, y)
    lv = np.array([1, 2], np.int32)
    with pytest.raises(af.AFError):   # leaf (2, 0, 0) lies inside leaf (1, 0, 0)
        af.forest_build_map(B, lmax, lv, np.zeros(2, np.int32), np.zeros(2, np.int32))


def test_batched_schedule_advances_each_level_by_its_substeps(amr, monkeypatch):
    """Host logic of the batched driver, with the library calls recorded
    instead of launched: at every time of the subcycled schedule one step
    call covers exactly the work items of the levels due (a suffix of the
    leaf order), each level is advanced 2^(l - lmin) times per coarse step
    from the array its parity bit names, and the conservative fix plus ghost
    exchange run at the synchronised times (Section 3.2)."""
    from paper_2205_07572_gb300 import af
    calls = []
    monkeypatch.setattr(af, "patch_step_pair",
                        lambda cfg, tiling, work, nwork, pair, *a, **k: calls.append(("step", work, nwork, pair.parity)))
    monkeypatch.setattr(af, "fill_ghosts_pair", lambda cfg, F, dst, src, flags, pair, *a, **k:
                        calls.append(("fill", dst, src, pair.parity)))
    monkeypatch.setattr(af, "reflux_pair", lambda cfg, F, sync, *a, **k: calls.append(("reflux", sync)))
    leaves = _sorted(S.balanced_forest(1, 2, 4, lambda l, x, y: x == y))
    cfg = af.config(af.ACOUSTICS, af.F64, 8, c=1.0)
    st = np.zeros((len(leaves), af.patch_words(8, 3)))
    run = amr.AMRRun(cfg, 1, 4, leaves, st, (0, 0), (1, 1), 0.01, device="cpu")
    calls.clear()
    base = run.work_all.data_ptr()
    counts = {l: 0 for l in run.forest.levels}
    p_before = run.parity
    lmin = run.forest.levels[0]
    run.coarse_step()
    assert run.parity == p_before ^ (1 << lmin)    # only the coarsest level flips
    par = p_before
    wl = run.work_all.numpy().view(np.int32).reshape(-1, 16)[:, 1]
    for c in calls:
        if c[0] == "step":
            first = (c[1] - base) // 64
            due = set(wl[first:first + c[2]].tolist())
            assert first + c[2] == run.nwork and due == set(range(min(due), 5)) & set(run.forest.levels)
            assert c[3] == par
            for l in due:
                counts[l] += 1
            par ^= sum(1 << l for l in range(min(due), 5))
        elif c[0] == "fill":
            assert c[1] == c[2] and c[3] == par
    assert counts == {l: 1 << (l - lmin) for l in run.forest.levels}
    syncs = [c[1] for c in calls if c[0] == "reflux"]
    nsub = 1 << (4 - lmin)
    expect = []
    for s in range(nsub):
        m = sum(1 << l for l in range(lmin, 5) if (s + 1) % (1 << (4 - l)) == 0)
        if bin(m).count("1") > 1:
            expect.append(m)
    assert syncs == expect and len(syncs) >= 1
    assert run.launches_per_coarse_step() == nsub + 4 * len(expect)
    assert run.cell_updates_per_coarse_step() == sum(
        int((run.forest.level == l).sum()) * 64 << (l - lmin) for l in run.forest.levels)


def test_native_regrid_rejects_bad_input(amr):
    from paper_2205_07572_gb300 import af
    F = amr.Forest(1, 3, [(1, x, y) for y in range(2) for x in range(2)], device="cpu")
    assert amr.regrid_leaves(F, np.zeros(4, np.int8), 1) == F.leaves
    assert len(amr.regrid_leaves(F, np.array([1, 0, 0, 0], np.int8), 1)) == 7
    import ctypes as C
    L = amr._lib()
    lv = np.array([1, 1], np.int32)
    xy = np.array([0, 0], np.int32)
    cnt = C.c_int32(0)
    tags = np.zeros(2, np.int8)
    st = L.af_forest_regrid(2, 1, 1, 3, amr._ip(lv), amr._ip(xy), amr._ip(xy), tags.ctypes.data, 0, None, None,
                            None, C.byref(cnt))
    assert st == 1  # duplicate leaf: AF_ERR_ARG
    lv2 = np.array([5], np.int32)
    st = L.af_forest_regrid(1, 1, 1, 3, amr._ip(lv2), amr._ip(xy), amr._ip(xy), tags.ctypes.data, 0, None, None,
                            None, C.byref(cnt))
    assert st == 1  # level above lmax
