"""Oracle AMR driver (test infrastructure): forest, subcycling, reflux, regrid.

Plain and sequential, written from Section 3 of the paper:
  * ghost data come from the leaf covering each ghost entry (orc_fill_amr);
  * a level advances with a same-level ghost copy before every step, and the
    interior plus first ghost layer of each of its leaves are advanced
    (orc_step_patch);
  * subcycling: level l+1 takes two steps of dt_l / 2 per step of level l;
    levels are advanced finest first; whenever levels are time-synchronised
    the conservative fix (orc_reflux_amr) is applied and then ghost data
    are exchanged between them (Section 3.2);
  * regrid: indicator per leaf (orc_tag), refine tagged leaves, coarsen
    families of four whose members all ask for it, keep the 2:1 balance,
    transfer the data (coarse -> fine interpolation / fine -> coarse
    averaging, Section 3.1).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import ADVECTION, VarCfg, _dp, cfg, lib, max_threads


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


class OracleForest:
    def __init__(self, eq: int, n: int, B: int, lmax: int, leaves, lo, hi, dt0: float, a=0.0, b=0.0, c=1.0,
                 state=None, field=None, t0: float = 0.0):
        """field: None (constant velocity a, b, or acoustics) or a velocity
        field of orc_step_patch_var (variable-velocity advection)."""
        self.field, self.time = field, float(t0)
        self.eq, self.n, self.B, self.lmax = eq, n, B, lmax
        self.ncomp = 1 if eq == ADVECTION else 3
        self.lo, self.hi = lo, hi
        self.dx0 = (hi[0] - lo[0]) / (B * n)
        self.dy0 = (hi[1] - lo[1]) / (B * n)
        self.dt0 = dt0
        self.a, self.b, self.c = a, b, c
        self.set_leaves(leaves)
        self.state = np.ascontiguousarray(state, dtype=np.float64).reshape(len(leaves), -1).copy()
        self.freg = np.zeros((len(leaves), 4 * self.ncomp * n))

    def set_leaves(self, leaves):
        self.leaves = list(leaves)
        self.level = np.array([l for l, _, _ in self.leaves], dtype=np.int32)
        self.ix = np.array([x for _, x, _ in self.leaves], dtype=np.int32)
        self.iy = np.array([y for _, _, y in self.leaves], dtype=np.int32)

    @property
    def levels(self):
        return sorted(set(self.level.tolist()))

    def cfg_level(self, l, dt=None):
        s = 2.0 ** -l
        return cfg(self.eq, self.n, self.dx0 * s, self.dy0 * s, self.dt0 * s if dt is None else dt, self.a,
                   self.b, self.c)

    # ---------------------------------------------------------------- pieces
    def fill(self, dst_mask: int, src_mask: int, same_only: bool):
        out = np.empty_like(self.state)
        lib().orc_fill_amr(self.n, self.ncomp, len(self.leaves), _ip(self.level), _ip(self.ix), _ip(self.iy),
                           self.B, self.lmax, dst_mask, src_mask, 1 if same_only else 0,
                           _dp(self.state), _dp(out))
        self.state = out

    def advance(self, l: int, t: float = 0.0, dt=None):
        """One step of dt (default dt_l) from time t on every leaf of level l
        (same-level copy first); each leaf's step is orc_step_patch (or
        orc_step_patch_var) on its own lattice, the leaves in parallel."""
        self.fill(1 << l, 1 << l, True)
        cf = self.cfg_level(l, dt)
        idx = np.ascontiguousarray(np.nonzero(self.level == l)[0], dtype=np.int32)
        if len(idx) == 0:
            return
        x0 = np.ascontiguousarray(self.lo[0] + self.ix[idx] * self.n * cf.dx, dtype=np.float64)
        y0 = np.ascontiguousarray(self.lo[1] + self.iy[idx] * self.n * cf.dy, dtype=np.float64)
        var = None if self.field is None else C.byref(VarCfg(self.n, self.field, cf.dx, cf.dy, cf.dt, 0.0, 0.0, t))
        lib().orc_step_patches(C.byref(cf), var, _dp(x0), _dp(y0), len(idx), _ip(idx), self.state.shape[1],
                               _dp(self.state), _dp(self.freg), self.freg.shape[1], max_threads())

    def reflux(self, sync_mask: int):
        lib().orc_reflux_amr(self.n, self.ncomp, len(self.leaves), _ip(self.level), _ip(self.ix), _ip(self.iy),
                             self.B, self.lmax, sync_mask, self.dx0, self.dy0, _dp(self.freg), _dp(self.state))

    def sync_fill(self, sync_mask: int):
        self.fill(sync_mask, sync_mask, False)

    def coarse_step(self, subcycle: bool = True):
        """Advance every level by dt of the coarsest level present (Section
        3.2, 'Subcycling'), finest level first.  subcycle=False: global time
        stepping, every level takes the finest level's dt, and all levels are
        synchronised (conservative fix, ghost exchange) after every step --
        the runs 'without subcycling' of Section 4.3."""
        levels = self.levels
        lmin, lmx = levels[0], levels[-1]
        S = 1 << (lmx - lmin)
        t0, dtf = self.time, self.dt0 / (1 << lmx)
        if not subcycle:
            every = sum(1 << l for l in levels)
            for s in range(S):
                for l in range(lmx, lmin - 1, -1):
                    if l in levels:
                        self.advance(l, t0 + s * dtf, dt=dtf)
                if len(levels) > 1:
                    self.reflux(every)
                    self.sync_fill(every)
            self.time = t0 + self.dt0 / (1 << lmin)
            return
        for s in range(S):
            for l in range(lmx, lmin - 1, -1):
                if l in levels and s % (1 << (lmx - l)) == 0:
                    self.advance(l, t0 + s * dtf)
            t = s + 1
            sync = 0
            for l in range(lmin, lmx + 1):
                if t % (1 << (lmx - l)) == 0:
                    sync |= 1 << l
            if bin(sync).count("1") > 1:
                self.reflux(sync)
                self.sync_fill(sync)
        self.time = t0 + self.dt0 / (1 << lmin)

    # ----------------------------------------------------------------- tags
    def tags(self, comp: int, kind: int, refine_thr: float, coarsen_thr: float):
        t = np.zeros(len(self.leaves), dtype=np.int8)
        ind = np.zeros(len(self.leaves))
        lib().orc_tag(self.n, self.ncomp, len(self.leaves), _ip(self.level), _dp(self.state), comp, kind,
                      self.dx0, self.dy0, refine_thr, coarsen_thr, t.ctypes.data_as(C.POINTER(C.c_int8)), _dp(ind))
        return t, ind

    def mass(self):
        out = np.zeros(self.ncomp)
        lib().orc_mass(self.n, self.ncomp, len(self.leaves), _ip(self.level), _dp(self.state), self.dx0,
                       self.dy0, _dp(out))
        return out

    # --------------------------------------------------------------- regrid
    def regrid(self, tags, lmin: int):
        """New forest from the tags (new_leaves), data transferred from the old
        one (orc_transfer), then a full ghost exchange."""
        new = new_leaves(self.leaves, tags, self.B, lmin, self.lmax)
        if new == self.leaves:
            return False
        ol, ox, oy, ost = self.level, self.ix, self.iy, self.state
        self.set_leaves(new)
        st = np.zeros((len(new), ost.shape[1]))
        lib().orc_transfer(self.n, self.ncomp, self.B, self.lmax, len(ol), _ip(ol), _ip(ox), _ip(oy), _dp(ost),
                           len(new), _ip(self.level), _ip(self.ix), _ip(self.iy), _dp(st))
        self.state = st
        self.freg = np.zeros((len(new), 4 * self.ncomp * self.n))
        self.sync_fill((1 << (self.lmax + 1)) - 1)
        return True


def new_leaves(leaves, tags, B: int, lmin: int, lmax: int):
    """Refine leaves tagged 1 (below lmax), coarsen complete families of four
    leaves tagged -1 (above lmin) unless that breaks the 2:1 balance, then
    split leaves until the forest is 2:1 balanced across faces and corners.
    Pinned by brute-force invariants on random forests (tiling, balance,
    refinement and coarsening rules; test_oracle_tag_regrid.py)."""
    cur = set(leaves)
    tag = {leaf: int(t) for leaf, t in zip(leaves, tags)}
    refine = {leaf for leaf in leaves if tag[leaf] == 1 and leaf[0] < lmax}
    out = set(cur)
    for (l, x, y) in refine:
        out.remove((l, x, y))
        out |= {(l + 1, 2 * x + a, 2 * y + b) for a in (0, 1) for b in (0, 1)}
    parents = {}
    for (l, x, y) in leaves:
        if l > lmin and tag[(l, x, y)] == -1:
            parents.setdefault((l - 1, x // 2, y // 2), []).append((l, x, y))
    for (pl, px, py), kids in sorted(parents.items()):
        if len(kids) != 4 or any(k not in out for k in kids):
            continue
        trial = (out - set(kids)) | {(pl, px, py)}
        if _violates(trial, (pl, px, py), B, lmax):
            continue
        out = trial
    changed = True
    while changed:
        changed = False
        for leaf in sorted(out):
            if _violates(out, leaf, B, lmax):
                l, x, y = leaf
                out.remove(leaf)
                out |= {(l + 1, 2 * x + a, 2 * y + b) for a in (0, 1) for b in (0, 1)}
                changed = True
    return sorted(out, key=lambda t: (t[0], t[2], t[1]))


def _violates(leafset, leaf, B, lmax):
    l, ix, iy = leaf
    side = B << l
    for sy in (-1, 0, 1):
        for sx in (-1, 0, 1):
            if sx == 0 and sy == 0:
                continue
            nx, ny = (ix + sx) % side, (iy + sy) % side
            for lv in range(l + 2, lmax + 1):
                s = 1 << (lv - l)
                for dy in range(s):
                    for dx in range(s):
                        if (lv, nx * s + dx, ny * s + dy) in leafset:
                            return True
    return False
