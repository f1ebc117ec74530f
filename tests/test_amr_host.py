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
