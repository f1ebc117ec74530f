"""Pins of the oracle's refinement indicator (orc_tag: the Section 3
criteria, range of Section 4.1 / 4.5.2 and centred differences of Section
4.4) and of its regrid rules (oracle.amr.new_leaves: refine tagged leaves,
coarsen complete families, 2:1 balance, Section 3), against closed forms and
brute-force invariants that do not use the oracle's own code:

  * the range and centred-difference indicators of linear and quadratic cell
    averages, whose values are known exactly;
  * the threshold rule at and around its boundaries;
  * on random forests and tags: the new forest tiles the domain, is 2:1
    balanced across faces and corners (periodically), keeps its levels in
    [lmin, lmax], refines every refine-tagged leaf, and coarsens only
    complete families of four leaves all tagged for it.
"""
import ctypes as C
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import synth as S
from oracle.amr import new_leaves


def _tag(n, level, avgs, kind, dx0, dy0, refine_thr, coarsen_thr):
    """orc_tag of component 0 of patches whose cell averages are avgs[p]."""
    lay = S.Layout(n, 1)
    st = np.zeros((len(level), 1, 4, lay.plane))
    lay.lattice(st)[:, 0, S.AVG, S.G:S.G + n, S.G:S.G + n] = avgs
    lv = np.ascontiguousarray(level, np.int32)
    t = np.zeros(len(level), np.int8)
    ind = np.zeros(len(level))
    O.lib().orc_tag(n, 1, len(level), lv.ctypes.data_as(C.POINTER(C.c_int32)), O._dp(st), 0, kind, dx0, dy0,
                    refine_thr, coarsen_thr, t.ctypes.data_as(C.POINTER(C.c_int8)), O._dp(ind))
    return t, ind


def _centres(n, level, ix, iy, dx0, dy0):
    hx, hy = dx0 / 2 ** level, dy0 / 2 ** level
    xc = (ix * n + np.arange(n) + 0.5) * hx
    yc = (iy * n + np.arange(n) + 0.5) * hy
    return np.meshgrid(xc, yc), hx, hy


@pytest.mark.parametrize("n", [8, 16])
def test_indicators_of_linear_data(n):
    """q = alpha x + beta y: the averages are the centre values, so the range
    over a patch is (|alpha| hx + |beta| hy)(n - 1) and every centred
    difference quotient is |alpha| or |beta|."""
    rng = np.random.default_rng(n)
    dx0, dy0 = 0.25, 0.5
    levels = np.array([0, 1, 2, 3, 1])
    al, be = rng.normal(size=5) * 3, rng.normal(size=5) * 3
    avgs, rng_ref, grad_ref = [], [], []
    for p, l in enumerate(levels):
        (X, Y), hx, hy = _centres(n, l, p, 2 * p, dx0, dy0)
        avgs.append(al[p] * X + be[p] * Y)
        rng_ref.append((abs(al[p]) * hx + abs(be[p]) * hy) * (n - 1))
        grad_ref.append(max(abs(al[p]), abs(be[p])))
    _, ind0 = _tag(n, levels, np.array(avgs), 0, dx0, dy0, 1e9, -1.0)
    _, ind1 = _tag(n, levels, np.array(avgs), 1, dx0, dy0, 1e9, -1.0)
    assert np.allclose(ind0, rng_ref, rtol=1e-12, atol=0)
    assert np.allclose(ind1, grad_ref, rtol=1e-10, atol=0)


def test_centred_difference_indicator_of_a_quadratic():
    """q = x^2 (+ y-independent): averages x_c^2 + hx^2 / 12, so the centred
    quotient at cell i is exactly 2 x_i; over the cells whose two neighbours
    are in the patch (i in 1 .. n-2) the indicator is 2 max |x_i|."""
    n, dx0, dy0 = 16, 1.0, 1.0
    levels = np.array([2, 3])
    avgs, ref = [], []
    for p, l in enumerate(levels):
        (X, _), hx, _ = _centres(n, l, 3 + p, 1, dx0, dy0)
        avgs.append(X ** 2 + hx ** 2 / 12)
        ref.append(2 * np.abs(X[0, 1:n - 1]).max())
    _, ind = _tag(n, levels, np.array(avgs), 1, dx0, dy0, 1e9, -1.0)
    assert np.allclose(ind, ref, rtol=1e-10, atol=0)


def test_threshold_rule():
    """tag = 1 if indicator >= refine threshold, -1 if below the coarsening
    threshold, else 0; a patch whose only non-zero average is v has range
    exactly v, so the boundaries are tested with equality."""
    n = 8
    vs = np.array([0.0, 0.25, 0.5, 0.75, 1.0, 2.0])
    avgs = np.zeros((len(vs), n, n))
    avgs[:, 3, 4] = vs
    t, ind = _tag(n, np.zeros(len(vs), int), avgs, 0, 1.0, 1.0, 1.0, 0.5)
    assert np.array_equal(ind, vs)
    assert t.tolist() == [-1, -1, 0, 0, 1, 1]


# ---------------------------------------------------------------- regrid
def _box(leaf, lmax):
    l, x, y = leaf
    s = 1 << (lmax - l)
    return x * s, y * s, s


def _touch(a, b, period):
    """Closed boxes (x, y, size) overlap or share a face or corner, periodically."""
    def gap(p0, s0, p1, s1):
        d = (p1 - p0) % period
        return d <= s0 or (period - d) % period <= s1

    return gap(a[0], a[2], b[0], b[2]) and gap(a[1], a[2], b[1], b[2])


def _check_forest(new, B, lmin, lmax):
    period = B << lmax
    # levels, tiling (areas add up, no leaf inside another)
    assert all(lmin <= l <= lmax for l, _, _ in new)
    assert sum(Fraction(1, 4 ** l) for l, _, _ in new) == B * B
    have = set(new)
    for (l, x, y) in new:
        for k in range(1, l - lmin + 1):
            assert (l - k, x >> k, y >> k) not in have, "a leaf inside another"
    # 2:1 balance across faces and corners
    boxes = [(leaf, _box(leaf, lmax)) for leaf in new]
    for i, (a, ba) in enumerate(boxes):
        for b, bb in boxes[i + 1:]:
            if abs(a[0] - b[0]) > 1:
                assert not _touch(ba, bb, period), (a, b)


def _ancestor_in(leaf, leaves, lmin):
    l, x, y = leaf
    return any((l - k, x >> k, y >> k) in leaves for k in range(1, l - lmin + 1))


@pytest.mark.parametrize("seed", range(6))
def test_regrid_invariants_on_random_forests(seed):
    rng = np.random.default_rng(seed)
    B, lmin, lmax = (1, 1, 4) if seed % 2 == 0 else (2, 1, 3)
    leaves = S.balanced_forest(B, lmin, lmax, lambda l, x, y: rng.random() < 0.35)
    _check_forest(leaves, B, lmin, lmax)
    tags = rng.choice(np.array([-1, 0, 1], np.int8), size=len(leaves), p=[0.45, 0.3, 0.25])
    new = new_leaves(leaves, tags, B, lmin, lmax)
    _check_forest(new, B, lmin, lmax)
    old, out = set(leaves), set(new)
    tag = dict(zip(leaves, tags.tolist()))
    # every refine-tagged leaf below lmax is replaced by finer leaves
    for leaf, t in tag.items():
        if t == 1 and leaf[0] < lmax:
            assert leaf not in out and not _ancestor_in(leaf, out, lmin)
    # a new leaf coarser than the old forest there is a complete family, all tagged -1
    for (l, x, y) in out - old:
        kids = [(l + 1, 2 * x + a, 2 * y + b) for a in (0, 1) for b in (0, 1)]
        if any(k in old for k in kids):
            assert all(k in old and tag[k] == -1 for k in kids)
    # no tags: a balanced forest is left as it is
    assert new_leaves(leaves, np.zeros(len(leaves), np.int8), B, lmin, lmax) == \
        sorted(leaves, key=lambda t: (t[0], t[2], t[1]))


def test_balance_check_catches_an_unbalanced_forest():
    """The brute-force balance check above is itself sharp: a level-3 leaf
    next to a level-1 leaf (corner contact included) fails it."""
    leaves = S.balanced_forest(1, 1, 3, lambda l, x, y: l < 3 and x == 0 and y == 0)
    _check_forest(leaves, 1, 1, 3)
    # replace the balanced neighbourhood by one level-1 leaf touching level-3 leaves
    bad = [t for t in leaves if not (t[0] == 2 and (t[1], t[2]) in {(2, 0), (2, 1), (3, 0), (3, 1)})]
    bad.append((1, 1, 0))
    with pytest.raises(AssertionError):
        _check_forest(bad, 1, 1, 3)
