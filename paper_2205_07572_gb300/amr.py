"""Host driver of the adaptive Active Flux method (Section 3) on the GPU.

The forest (a periodic B x B brick of quadtrees), its device description, the
per-level work lists of af_patch_step and the subcycling schedule live here;
every arithmetic step -- the patch step, the ghost exchange, the conservative
fix, the regrid transfer, the indicator and the mass totals -- is a call into
libaf.so.

Leaves are kept sorted by level (then row-major), so the patches of one level
are a contiguous slice of the state array.  A level is advanced from the
state buffer into a scratch buffer and the slice is copied back.
"""
from __future__ import annotations

import numpy as np

from . import af


def _leaf_order(leaves):
    return sorted(leaves, key=lambda t: (t[0], t[2], t[1]))


class Forest:
    """Leaves (level, ix, iy) of a periodic forest with their region maps."""

    def __init__(self, B: int, lmax: int, leaves, device="cuda"):
        import torch
        self.B, self.lmax = B, lmax
        self.leaves = _leaf_order(leaves)
        self.level = np.array([l for l, _, _ in self.leaves], dtype=np.int32)
        self.ix = np.array([x for _, x, _ in self.leaves], dtype=np.int32)
        self.iy = np.array([y for _, _, y in self.leaves], dtype=np.int32)
        self.map = af.forest_build_map(B, lmax, self.level, self.ix, self.iy)
        self.offsets = [af.forest_map_offset(B, l) for l in range(lmax + 2)]
        t = lambda a: torch.from_numpy(a).to(device)
        self.d_level, self.d_ix, self.d_iy, self.d_map = t(self.level), t(self.ix), t(self.iy), t(self.map)
        self.c = af.forest_struct(len(self.leaves), B, lmax, self.d_level, self.d_ix, self.d_iy, self.d_map)

    @property
    def nleaf(self) -> int:
        return len(self.leaves)

    @property
    def levels(self):
        return sorted(set(self.level.tolist()))

    def region(self, l: int, x: int, y: int) -> int:
        """Leaf index of region (l, x, y) (periodic) if it is a leaf, else -1."""
        side = self.B << l
        return int(self.map[self.offsets[l] + (y % side) * side + (x % side)])

    def level_slice(self, l: int) -> slice:
        idx = np.nonzero(self.level == l)[0]
        return slice(int(idx[0]), int(idx[-1]) + 1) if len(idx) else slice(0, 0)

    def neighbours(self, idx) -> np.ndarray:
        """Same-level neighbour of each leaf in idx (W, E, S, N, SW, SE, NW, NE) or -1."""
        dirs = [(-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (1, -1), (-1, 1), (1, 1)]
        out = np.full((len(idx), 8), -1, dtype=np.int32)
        for r, p in enumerate(idx):
            l, x, y = self.leaves[p]
            for d, (sx, sy) in enumerate(dirs):
                out[r, d] = self.region(l, x + sx, y + sy)
        return out


def regrid_leaves(forest: Forest, tags, lmin: int):
    """New leaf set: leaves tagged 1 below lmax are split, complete families of
    four leaves tagged -1 above lmin are merged unless the merged leaf would
    sit next to a leaf two levels finer, then leaves are split until no leaf
    has a face or corner neighbour region holding a leaf two or more levels
    finer (2:1 balance).  The same rules as the oracle's, implemented on
    per-level occupancy grids."""
    B, lmax = forest.B, forest.lmax
    # occ[l]: level-l region grid, 1 where a leaf of level exactly l sits
    occ = [np.zeros((B << l, B << l), dtype=np.int8) for l in range(lmax + 1)]
    tag = {}
    for (l, x, y), t in zip(forest.leaves, tags):
        occ[l][y, x] = 1
        tag[(l, x, y)] = int(t)

    def split(l, x, y):
        occ[l][y, x] = 0
        occ[l + 1][2 * y:2 * y + 2, 2 * x:2 * x + 2] = 1

    for (l, x, y), t in list(tag.items()):
        if t == 1 and l < lmax:
            split(l, x, y)

    def finer_than(l, x, y, d):
        """True if the level-l region (x, y) contains a leaf of level >= l + d."""
        for m in range(l + d, lmax + 1):
            s = 1 << (m - l)
            if occ[m][y * s:(y + 1) * s, x * s:(x + 1) * s].any():
                return True
        return False

    def unbalanced(l, x, y):
        side = B << l
        for sy in (-1, 0, 1):
            for sx in (-1, 0, 1):
                if (sx or sy) and finer_than(l, (x + sx) % side, (y + sy) % side, 2):
                    return True
        return False

    families = {}
    for (l, x, y), t in tag.items():
        if t == -1 and l > lmin:
            families.setdefault((l - 1, x // 2, y // 2), []).append((l, x, y))
    for (pl, px, py) in sorted(families):
        kids = families[(pl, px, py)]
        if len(kids) != 4 or not all(occ[l][y, x] for (l, x, y) in kids):
            continue
        for (l, x, y) in kids:
            occ[l][y, x] = 0
        occ[pl][py, px] = 1
        if unbalanced(pl, px, py):
            occ[pl][py, px] = 0
            for (l, x, y) in kids:
                occ[l][y, x] = 1
    changed = True
    while changed:
        changed = False
        for l in range(lmax + 1):
            ys, xs = np.nonzero(occ[l])
            for y, x in sorted(zip(ys.tolist(), xs.tolist())):
                if occ[l][y, x] and unbalanced(l, x, y):
                    split(l, x, y)
                    changed = True
    out = []
    for l in range(lmax + 1):
        ys, xs = np.nonzero(occ[l])
        out += [(l, int(x), int(y)) for y, x in zip(ys, xs)]
    return _leaf_order(out)


class AMRRun:
    """Adaptive run: subcycled steps (Section 3.2), reflux, ghost exchange, regrid."""

    def __init__(self, cfg: af.Config, B: int, lmax: int, leaves, state, lo, hi, dt0: float, device="cuda"):
        import torch
        self.cfg, self.B, self.lmax, self.device = cfg, B, lmax, device
        self.lo, self.hi = lo, hi
        self.dx0 = (hi[0] - lo[0]) / (B * cfg.n)
        self.dy0 = (hi[1] - lo[1]) / (B * cfg.n)
        self.dt0 = dt0
        self.dtype = torch.float64 if cfg.prec == af.F64 else torch.float32
        self.words = af.patch_words(cfg.n, cfg.ncomp)
        self.forest = Forest(B, lmax, leaves, device)
        order = {leaf: k for k, leaf in enumerate(leaves)}
        st = np.asarray(state).reshape(len(leaves), -1)[[order[leaf] for leaf in self.forest.leaves]]
        self.a = torch.as_tensor(st).to(device=device, dtype=self.dtype).contiguous()
        self._setup()
        self.fill(self.all_levels, self.all_levels)

    # ------------------------------------------------------------ plumbing
    @property
    def all_levels(self) -> int:
        return (1 << (self.lmax + 1)) - 1

    def _setup(self):
        import torch
        F = self.forest
        self.b = self.a.clone()
        self.freg = torch.zeros((F.nleaf, 4, self.cfg.ncomp, self.cfg.n), dtype=torch.float64, device=self.device)
        self.work = {}
        for l in F.levels:
            sl = F.level_slice(l)
            idx = np.arange(sl.start, sl.stop)
            w = af.build_step_work(self.cfg, idx, np.full(len(idx), l, np.int32), F.neighbours(idx))
            self.work[l] = (torch.from_numpy(w).to(self.device), len(w) // 64, sl)
        self.scratch = torch.zeros(max(1, af.mass_scratch_bytes(F.nleaf, self.cfg.ncomp) // 8),
                                   dtype=torch.float64, device=self.device)
        self.mass_out = torch.zeros(self.cfg.ncomp, dtype=torch.float64, device=self.device)

    def fill(self, dst: int, src: int, flags: int = 0):
        af.fill_ghosts(self.cfg, self.forest.c, dst, src, flags, self.a)

    # -------------------------------------------------------------- steps
    def advance(self, l: int):
        """One step of dt_l on every leaf of level l."""
        work, nwork, sl = self.work[l]
        af.patch_step(self.cfg, work, nwork, self.a, self.b, self.dt0, self.dx0, self.dy0, self.freg)
        self.a[sl].copy_(self.b[sl])

    def coarse_step(self):
        """Advance all levels by the step of the coarsest level present,
        finest level first; at every time where two or more levels are
        synchronised: conservative fix, then ghost exchange among them."""
        levels = self.forest.levels
        lmin, lmx = levels[0], levels[-1]
        for s in range(1 << (lmx - lmin)):
            for l in range(lmx, lmin - 1, -1):
                if l in self.work and s % (1 << (lmx - l)) == 0:
                    self.advance(l)
            sync = 0
            for l in range(lmin, lmx + 1):
                if (s + 1) % (1 << (lmx - l)) == 0:
                    sync |= 1 << l
            if bin(sync).count("1") > 1:
                af.reflux(self.cfg, self.forest.c, sync, self.dx0, self.dy0, self.freg, self.a)
                self.fill(sync, sync)

    # ---------------------------------------------------- tags and regrid
    def tags(self, comp: int, kind: int, refine_thr: float, coarsen_thr: float):
        import torch
        t = torch.zeros(self.forest.nleaf, dtype=torch.int8, device=self.device)
        ind = torch.zeros(self.forest.nleaf, dtype=torch.float64, device=self.device)
        af.tag(self.cfg, self.forest.c, self.a, comp, kind, self.dx0, self.dy0, refine_thr, coarsen_thr, t, ind)
        return t.cpu().numpy(), ind.cpu().numpy()

    def regrid(self, tags, lmin: int) -> bool:
        import torch
        new = regrid_leaves(self.forest, tags, lmin)
        if new == self.forest.leaves:
            return False
        old_forest, old_state = self.forest, self.a
        self.forest = Forest(self.B, self.lmax, new, self.device)
        self.a = torch.empty((self.forest.nleaf, self.words), dtype=self.dtype, device=self.device)
        af.transfer(self.cfg, old_forest.c, old_state, self.forest.c, self.a)
        self._keep = old_forest  # device arrays of the old forest stay alive until the copy ran
        self._setup()
        self.fill(self.all_levels, self.all_levels)
        return True

    def mass(self):
        af.mass(self.cfg, self.forest.c, self.a, self.dx0, self.dy0, self.scratch, self.mass_out)
        return self.mass_out.cpu().numpy()

    def state_in_order(self, leaves):
        """Host copy of the state with leaves in the given order."""
        idx = {leaf: k for k, leaf in enumerate(self.forest.leaves)}
        host = self.a.double().cpu().numpy()
        return host[[idx[leaf] for leaf in leaves]]
