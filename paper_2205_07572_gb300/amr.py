"""Host driver of the adaptive Active Flux method (Section 3) on the GPU.

The forest (a periodic B x B brick of quadtrees), its device description, the
work lists of af_patch_step and the subcycling schedule live here; every
arithmetic step -- the patch step, the ghost exchange, the conservative fix,
the regrid transfer, the indicator and the mass totals -- is a call into
libaf.so, and so are the forest's neighbour tables and the regrid decision
(af_forest_neighbours, af_forest_regrid).

Leaves are kept sorted by level (then row-major), so the patches of one level
are a contiguous slice of the state array, and the levels that advance at one
time of the subcycled schedule (all levels finer than some level) are a
contiguous suffix of it.

Three ways to run the same schedule:
  "batched"   the state is a pair of arrays with a current one per level
              (af_state_pair): at each time of the schedule ONE af_patch_step
              launch advances every level due, with no copies; a whole
              coarse step can be captured once in a CUDA graph and replayed;
  "per_level" one launch per level into a scratch array, then the level's
              slice is copied back;
  "per_patch" one launch per patch (the patch-by-patch loop of a CPU solver),
              then the level's slice is copied back.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import af

_IP = C.POINTER(C.c_int32)


def _ip(a):
    return a.ctypes.data_as(_IP)


def _leaf_order(leaves):
    return sorted(leaves, key=lambda t: (t[0], t[2], t[1]))


class Forest:
    """Leaves (level, ix, iy) of a periodic forest with their region maps and
    same-level neighbour table.  `leaves` is a list of tuples or, with
    arrays=(level, ix, iy), three integer arrays (any order)."""

    def __init__(self, B: int, lmax: int, leaves=None, device="cuda", arrays=None):
        import torch
        self.B, self.lmax = B, lmax
        if arrays is None:
            arr = np.asarray(list(leaves), dtype=np.int32).reshape(-1, 3)
            lv, x, y = arr[:, 0], arr[:, 1], arr[:, 2]
        else:
            lv, x, y = (np.asarray(a, dtype=np.int32) for a in arrays)
        # by level, then row, then column (the native regrid already writes
        # that order, which one pass over the packed keys confirms)
        if (B << lmax) < (1 << 21):
            key = (lv.astype(np.int64) << 42) | (y.astype(np.int64) << 21) | x.astype(np.int64)
            if len(key) > 1 and not bool(np.all(key[1:] > key[:-1])):
                order = np.argsort(key, kind="stable")
                lv, x, y = lv[order], x[order], y[order]
        else:
            order = np.lexsort((x, y, lv))
            lv, x, y = lv[order], x[order], y[order]
        self.level = np.ascontiguousarray(lv)
        self.ix = np.ascontiguousarray(x)
        self.iy = np.ascontiguousarray(y)
        self._leaves = None
        self.map = af.forest_build_map(B, lmax, self.level, self.ix, self.iy)
        self.offsets = [af.forest_map_offset(B, l) for l in range(lmax + 2)]
        self.nbr = forest_neighbours(B, lmax, self.level, self.ix, self.iy, self.map)
        t = lambda a: torch.from_numpy(a).to(device, non_blocking=True)
        self.d_level, self.d_ix, self.d_iy, self.d_map = t(self.level), t(self.ix), t(self.iy), t(self.map)
        self.c = af.forest_struct(self.nleaf, B, lmax, self.d_level, self.d_ix, self.d_iy, self.d_map)

    @property
    def leaves(self):
        """The leaves as (level, ix, iy) tuples in storage order."""
        if self._leaves is None:
            self._leaves = list(zip(self.level.tolist(), self.ix.tolist(), self.iy.tolist()))
        return self._leaves

    def same_leaves(self, level, ix, iy) -> bool:
        """True if the arrays hold exactly this forest's leaves (any order)."""
        if len(level) != self.nleaf:
            return False
        o = np.lexsort((ix, iy, level))
        return (np.array_equal(np.asarray(level)[o], self.level) and np.array_equal(np.asarray(ix)[o], self.ix)
                and np.array_equal(np.asarray(iy)[o], self.iy))

    @property
    def nleaf(self) -> int:
        return len(self.level)

    @property
    def levels(self):
        return np.unique(self.level).tolist()

    def region(self, l: int, x: int, y: int) -> int:
        """Leaf index of region (l, x, y) (periodic) if it is a leaf, else -1."""
        side = self.B << l
        q = int(self.map[self.offsets[l] + (y % side) * side + (x % side)])
        return q if q >= 0 else -1

    def level_slice(self, l: int) -> slice:
        lo = int(np.searchsorted(self.level, l, side="left"))
        hi = int(np.searchsorted(self.level, l, side="right"))
        return slice(lo, hi)

    def neighbours(self, idx) -> np.ndarray:
        """Same-level neighbour of each leaf in idx (W, E, S, N, SW, SE, NW, NE) or -1."""
        return self.nbr[np.asarray(list(idx), dtype=np.int64)]

    def cells(self, n: int) -> np.ndarray:
        """Interior cells per level (index = level)."""
        return np.bincount(self.level, minlength=self.lmax + 1) * n * n


_EXTRA = [
    ("af_forest_neighbours", C.c_int, [C.c_int32, C.c_int32, C.c_int32, _IP, _IP, _IP, _IP, _IP]),
    ("af_forest_regrid", C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _IP, _IP, _IP, C.c_void_p,
                                   C.c_int32, _IP, _IP, _IP, _IP]),
]


def _lib():
    L = af.lib()
    for name, res, args in _EXTRA:
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    return L


def forest_neighbours(B, lmax, level, ix, iy, fmap) -> np.ndarray:
    n = len(level)
    out = np.full((n, 8), -1, dtype=np.int32)
    af._check(_lib().af_forest_neighbours(n, B, lmax, _ip(level), _ip(ix), _ip(iy), _ip(fmap), _ip(out)),
              "af_forest_neighbours")
    return out


def regrid_arrays(forest: Forest, tags, lmin: int):
    """New leaf set from per-leaf tags (af_forest_regrid) as arrays (level,
    ix, iy): leaves tagged 1 below lmax are split, complete families of four
    leaves tagged -1 above lmin are merged unless the merged leaf would sit
    next to a leaf two levels finer, then leaves are split until the forest
    is 2:1 balanced."""
    tags = np.ascontiguousarray(tags, dtype=np.int8)
    L = _lib()
    cnt = C.c_int32(0)
    args = (forest.nleaf, forest.B, lmin, forest.lmax, _ip(forest.level), _ip(forest.ix), _ip(forest.iy),
            tags.ctypes.data)
    # at most four leaves per leaf before balancing; try that capacity first
    cap = 4 * forest.nleaf + 64
    lv, x, y = (np.empty(cap, dtype=np.int32) for _ in range(3))
    st = L.af_forest_regrid(*args, cap, _ip(lv), _ip(x), _ip(y), C.byref(cnt))
    m = cnt.value
    if st != 0 and m > cap:  # a larger forest after balancing: ask again with the size it reported
        lv, x, y = (np.empty(m, dtype=np.int32) for _ in range(3))
        st = L.af_forest_regrid(*args, m, _ip(lv), _ip(x), _ip(y), C.byref(cnt))
    af._check(st, "af_forest_regrid")
    return lv[:m], x[:m], y[:m]


def regrid_leaves(forest: Forest, tags, lmin: int):
    """regrid_arrays as a list of (level, ix, iy) tuples."""
    lv, x, y = regrid_arrays(forest, tags, lmin)
    return list(zip(lv.tolist(), x.tolist(), y.tolist()))


MODES = ("batched", "per_level", "per_patch")


class AMRRun:
    """Adaptive run: subcycled steps (Section 3.2), reflux, ghost exchange, regrid."""

    def __init__(self, cfg: af.Config, B: int, lmax: int, leaves, state, lo, hi, dt0: float, device="cuda",
                 mode: str = "batched", graphs: bool = False, tiling=None, planned_fill: bool = True,
                 ext_tiling=None, field=None):
        import torch
        if mode not in MODES:
            raise ValueError(f"mode must be one of {MODES}")
        self.cfg, self.B, self.lmax, self.device = cfg, B, lmax, device
        # field: None, or a velocity field of af_patch_step_var (variable-
        # velocity advection); the swirl depends on time, which a captured
        # graph would freeze, so it runs without graphs
        self.field = field
        self.mode = mode
        self.use_graphs = bool(graphs) and mode == "batched" and field != af.FIELD_SWIRL
        self.planned_fill = planned_fill
        self.lo, self.hi = lo, hi
        self.dx0 = (hi[0] - lo[0]) / (B * cfg.n)
        self.dy0 = (hi[1] - lo[1]) / (B * cfg.n)
        self.dt0 = dt0
        self.tiling = af.default_tiling(cfg) if tiling is None else int(tiling)
        # batched mode: leaves with a non-same-level neighbour advance their
        # first ghost layer too ((n+2)^2 cells); they may use their own tiling
        self.ext_tiling = None if (ext_tiling is None or mode != "batched") else int(ext_tiling)
        self.dtype = torch.float64 if cfg.prec == af.F64 else torch.float32
        self.words = af.patch_words(cfg.n, cfg.ncomp)
        self.forest = Forest(B, lmax, leaves, device)
        order = {leaf: k for k, leaf in enumerate(_leaf_order(leaves))}
        st = np.asarray(state).reshape(len(leaves), -1)[[order[leaf] for leaf in self.forest.leaves]]
        # three state buffers of growing capacity: the current pair and the
        # one a regrid transfers into (so a regrid allocates nothing large)
        self._pool = [None, None, None]
        self._ia, self._ib = 0, 1
        self.a = self._buffer(0, self.forest.nleaf)
        self.a.copy_(torch.as_tensor(st).to(dtype=self.dtype))
        self.parity = 0
        self.time = 0.0
        self._setup()
        self.fill(self.all_levels, self.all_levels)

    # ------------------------------------------------------------ plumbing
    @property
    def all_levels(self) -> int:
        return (1 << (self.lmax + 1)) - 1

    @property
    def pair(self) -> af.StatePair:
        return af.state_pair(self.a, self.b, self.parity)

    def _buffer(self, i: int, nleaf: int):
        """View [nleaf, words] of pool buffer i, grown (by a quarter beyond
        the request) if it is too small."""
        import torch
        need = max(1, nleaf) * self.words
        buf = self._pool[i]
        if buf is None or buf.numel() < need:
            buf = torch.empty(need + need // 4, dtype=self.dtype, device=self.device)
            self._pool[i] = buf
        return buf[:nleaf * self.words].view(nleaf, self.words)

    def _setup(self):
        import torch
        F = self.forest
        self.b = self._buffer(self._ib, F.nleaf)
        if self.mode == "batched":
            self.b.zero_()
        else:
            self.b.copy_(self.a)
        self.freg = torch.zeros((F.nleaf, 4, self.cfg.ncomp, self.cfg.n), dtype=torch.float64, device=self.device)
        # work items are in leaf order, so every level's items are contiguous
        self.set_tiling(self.tiling)
        self.scratch = torch.zeros(max(1, af.mass_scratch_bytes(F.nleaf, self.cfg.ncomp) // 8),
                                   dtype=torch.float64, device=self.device)
        self.mass_out = torch.zeros(self.cfg.ncomp, dtype=torch.float64, device=self.device)
        self.graphs = {}
        self.d_nbr = torch.from_numpy(F.nbr).to(self.device)
        if self.planned_fill and str(self.device) != "cpu":
            self.plan = af.ghost_plan(self.cfg, F.c, 0, self.device)
        else:
            self.plan = None

    def set_tiling(self, tiling: int):
        """Rebuild the work list for another compiled tiling (drops captured graphs)."""
        import torch
        self.tiling = int(tiling)
        F = self.forest
        ext = (F.nbr < 0).any(axis=1) if F.nleaf else np.zeros(0, bool)
        if self.ext_tiling is None:
            groups = [(np.arange(F.nleaf), self.tiling)]
        else:
            groups = [(np.nonzero(~ext)[0], self.tiling), (np.nonzero(ext)[0], self.ext_tiling)]
        # one work list per group, each in leaf order (levels contiguous)
        self.work_groups = []
        w0 = None
        for idx, til in groups:
            w = af.build_step_work(self.cfg, idx, F.level[idx], F.nbr[idx], tiling=til, ix=F.ix[idx], iy=F.iy[idx])
            w0 = w if w0 is None else w0
            nw = len(w) // 64
            wl = w.view(np.int32).reshape(nw, 16)[:, 1] if nw else np.zeros(0, np.int32)
            starts = [int(np.searchsorted(wl, l, side="left")) for l in range(self.lmax + 2)]
            self.work_groups.append((torch.from_numpy(w).to(self.device), nw, starts, til))
        self.work_all, nwork, self.work_start, _ = self.work_groups[0]
        self.nwork = nwork
        if self.mode == "per_patch":
            wi = w0.view(np.int32).reshape(nwork, 16) if nwork else np.zeros((0, 16), np.int32)
            p = np.arange(F.nleaf)
            self.patch_work = list(zip(np.searchsorted(wi[:, 0], p, side="left").tolist(),
                                       np.searchsorted(wi[:, 0], p, side="right").tolist()))
        self.graphs = {}

    def fill(self, dst: int, src: int, flags: int = 0, stream=None):
        if self.plan is not None and dst == src and not (flags & af.FILL_ALL_PATCHES):
            plan, n_a, n_b = self.plan
            # levels finer than any present are empty: adding them makes the
            # set upward closed without changing what is exchanged
            levels = dst | (self.all_levels & ~((1 << dst.bit_length()) - 1))
            af.fill_ghosts_planned(self.cfg, self.forest.c, levels, flags, plan, n_a, n_b, self.pair, stream)
        elif self.mode == "batched":
            af.fill_ghosts_pair(self.cfg, self.forest.c, dst, src, flags, self.pair, stream)
        else:
            af.fill_ghosts(self.cfg, self.forest.c, dst, src, flags, self.a, stream)

    def _work_ptr(self, start: int) -> int:
        return self.work_all.data_ptr() + 64 * start

    # -------------------------------------------------------------- steps
    def advance_from(self, lstar: int, stream=None, t: float = 0.0):
        """One step of dt_l from time t on every leaf of every level l >= lstar
        (the levels due at one time of the subcycled schedule)."""
        if self.mode == "batched":
            for work, nw, starts, til in self.work_groups:
                s = starts[lstar]
                if nw > s:
                    if self.field is None:
                        af.patch_step_pair(self.cfg, til, work.data_ptr() + 64 * s, nw - s, self.pair, self.dt0,
                                           self.dx0, self.dy0, self.freg, stream)
                    else:
                        af.patch_step_var(self.cfg, til, work.data_ptr() + 64 * s, nw - s, self.pair,
                                          af.velocity(self.field, self.lo, self.hi, t), self.dt0, self.dx0,
                                          self.dy0, self.freg, stream)
            self.parity ^= self.all_levels & ~((1 << lstar) - 1)
            return
        for l in range(self.lmax, lstar - 1, -1):
            self.advance(l, stream)

    def advance(self, l: int, stream=None):
        """One step of dt_l on every leaf of level l (per_level / per_patch)."""
        assert self.mode != "batched"
        assert self.field is None, "variable-velocity runs use the batched mode"
        s, e = self.work_start[l], self.work_start[l + 1]
        if e == s:
            return
        sl = self.forest.level_slice(l)
        if self.mode == "per_level":
            af.patch_step(self.cfg, self._work_ptr(s), e - s, self.a, self.b, self.dt0, self.dx0, self.dy0,
                          self.freg, stream, tiling=self.tiling)
        else:
            for p in range(sl.start, sl.stop):
                ps, pe = self.patch_work[p]
                af.patch_step(self.cfg, self._work_ptr(ps), pe - ps, self.a, self.b, self.dt0, self.dx0, self.dy0,
                              self.freg, stream, tiling=self.tiling)
        self.a[sl].copy_(self.b[sl])

    def _schedule(self, stream=None):
        """Finest level first; at every time where two or more levels are
        synchronised: conservative fix, then ghost exchange among them."""
        levels = self.forest.levels
        lmin, lmx = levels[0], levels[-1]
        t0, dtf = self.time, self.dt0 / (1 << lmx)
        for s in range(1 << (lmx - lmin)):
            due = [l for l in levels if s % (1 << (lmx - l)) == 0]
            self.advance_from(min(due), stream, t0 + s * dtf)
            sync = 0
            for l in range(lmin, lmx + 1):
                if (s + 1) % (1 << (lmx - l)) == 0:
                    sync |= 1 << l
            if bin(sync).count("1") > 1:
                if self.mode == "batched":
                    af.reflux_pair(self.cfg, self.forest.c, sync, self.dx0, self.dy0, self.freg, self.pair, stream)
                else:
                    af.reflux(self.cfg, self.forest.c, sync, self.dx0, self.dy0, self.freg, self.a, stream)
                self.fill(sync, sync, stream=stream)

    def coarse_dt(self) -> float:
        """Time step of the coarsest level present (one coarse step)."""
        return self.dt0 / (1 << self.forest.levels[0])

    def coarse_step(self):
        """Advance all levels by the step of the coarsest level present."""
        dtc = self.coarse_dt()
        if not self.use_graphs:
            self._schedule()
            self.time += dtc
            return
        import torch
        key = self.parity
        g = self.graphs.get(key)
        if g is None:
            # first coarse step from this parity runs eagerly (warm-up: kernel
            # attributes and weight tables are set up outside the capture);
            # the next one from the same parity is captured
            if key not in self.graphs:
                self.graphs[key] = None
                self._schedule()
                self.time += dtc
                return
            g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            p0 = self.parity
            with torch.cuda.graph(g, stream=side):
                self._schedule()
            torch.cuda.current_stream().wait_stream(side)
            self.graphs[key] = (g, self.parity)
            self.parity = p0  # capture did not run anything
        g, p1 = self.graphs[key]
        g.replay()
        self.parity = p1
        self.time += dtc

    def cell_updates_per_coarse_step(self) -> int:
        levels = self.forest.levels
        lmin = levels[0]
        cells = self.forest.cells(self.cfg.n)
        return int(sum(int(cells[l]) << (l - lmin) for l in levels))

    def launches_per_coarse_step(self) -> int:
        """Kernels of this library launched by one coarse step."""
        levels = self.forest.levels
        lmin, lmx = levels[0], levels[-1]
        n = 0
        for s in range(1 << (lmx - lmin)):
            due = [l for l in levels if s % (1 << (lmx - l)) == 0]
            if self.mode == "batched":
                n += sum(1 for _, nw, starts, _ in self.work_groups if nw > starts[min(due)])
            elif self.mode == "per_level":
                n += len(due)
            else:
                n += sum(self.forest.level_slice(l).stop - self.forest.level_slice(l).start for l in due)
            sync = sum(1 for l in range(lmin, lmx + 1) if (s + 1) % (1 << (lmx - l)) == 0)
            if sync > 1:
                n += 1 + (2 if self.plan is not None else 3)   # reflux + exchange passes
        return n

    # ---------------------------------------------------- tags and regrid
    def tags(self, comp: int, kind: int, refine_thr: float, coarsen_thr: float):
        import torch
        t = torch.zeros(self.forest.nleaf, dtype=torch.int8, device=self.device)
        ind = torch.zeros(self.forest.nleaf, dtype=torch.float64, device=self.device)
        af.tag_pair(self.cfg, self.forest.c, self.pair, comp, kind, self.dx0, self.dy0, refine_thr, coarsen_thr,
                    t, ind)
        ind = ind.cpu().numpy()  # one synchronisation: the tags are in place by then
        return t.cpu().numpy(), ind

    def regrid(self, tags, lmin: int) -> bool:
        """Regrid from per-leaf tags (af_forest_regrid), move the state to the
        new forest (af_transfer) and exchange its ghosts; False if the forest
        is unchanged."""
        lv, x, y = regrid_arrays(self.forest, tags, lmin)
        if self.forest.same_leaves(lv, x, y):
            return False
        old_forest, old_pair, old_bufs = self.forest, self.pair, (self.a, self.b)
        self.forest = Forest(self.B, self.lmax, device=self.device, arrays=(lv, x, y))
        # the new state goes to the pool buffer the old pair does not use; the
        # old current array's buffer then holds the new second array (zeroed
        # by _setup after the transfer, in stream order)
        ic = 3 - self._ia - self._ib
        self.a = self._buffer(ic, self.forest.nleaf)
        af.transfer_pair(self.cfg, old_forest.c, old_pair, self.forest.c, self.a)
        self._keep = (old_forest, old_bufs)  # the old arrays stay alive until the copy ran
        self._ia, self._ib = ic, self._ia
        self.parity = 0
        self._setup()
        self.fill(self.all_levels, self.all_levels)
        return True

    def cnn_inputs(self, thr: float):
        """Learned tagger inputs of every leaf (BF16 storage, int16 tensor)."""
        import torch
        S = self.cfg.n + 4
        x = torch.empty((self.forest.nleaf, self.cfg.ncomp, S, S), dtype=torch.int16, device=self.device)
        af.cnn_inputs(self.cfg, self.forest.c, self.pair, self.d_nbr, self.dx0, thr, x)
        return x

    def tags_learned(self, tagger, comp: int, kind: int, refine_thr: float, coarsen_thr: float, cmin: float):
        """Tags from the learned tagger with the plain criterion (af_tag) as
        fallback where the network is not confident; returns (tags, number of
        fallbacks)."""
        import torch
        nl = self.forest.nleaf
        plain = torch.zeros(nl, dtype=torch.int8, device=self.device)
        af.tag_pair(self.cfg, self.forest.c, self.pair, comp, kind, self.dx0, self.dy0, refine_thr, coarsen_thr,
                    plain, None)
        x = self.cnn_inputs(refine_thr)
        logit, _ = tagger.infer(x, self.forest.d_level)
        tags = torch.zeros(nl, dtype=torch.int8, device=self.device)
        nf = torch.zeros(1, dtype=torch.int32, device=self.device)
        af.cnn_tags(nl, logit, plain, cmin, tags, nf)
        return tags.cpu().numpy(), int(nf.item())

    def mass(self):
        af.mass_pair(self.cfg, self.forest.c, self.pair, self.dx0, self.dy0, self.scratch, self.mass_out)
        return self.mass_out.cpu().numpy()

    def current(self):
        """Device tensor with every leaf's current values (a copy when levels
        are split between the two arrays)."""
        if self.parity == 0:
            return self.a
        out = self.a.clone()
        for l in self.forest.levels:
            if (self.parity >> l) & 1:
                sl = self.forest.level_slice(l)
                out[sl] = self.b[sl]
        return out

    def state_in_order(self, leaves):
        """Host copy of the state with leaves in the given order."""
        idx = {leaf: k for k, leaf in enumerate(self.forest.leaves)}
        host = self.current().double().cpu().numpy()
        return host[[idx[leaf] for leaf in leaves]]
