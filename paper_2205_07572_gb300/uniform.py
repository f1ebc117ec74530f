"""Host driver of a uniform, periodic array of same-level patches.

Holds two device state buffers and the device work list; every step is one
af_patch_step call (the same-level ghost copy is fused into the kernel's halo
load, Section 3.1 case 3), after which the buffers swap.  Host orchestration
only: all arithmetic runs in libaf.so.
"""
from __future__ import annotations

import numpy as np

from . import af


def periodic_neighbours(px: int, py: int) -> np.ndarray:
    """[px*py, 8] neighbour indices (W, E, S, N, SW, SE, NW, NE) on a torus."""
    dirs = [(-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (1, -1), (-1, 1), (1, 1)]
    out = np.zeros((px * py, 8), dtype=np.int32)
    for p in range(px * py):
        ix, iy = p % px, p // px
        for k, (sx, sy) in enumerate(dirs):
            out[p, k] = ((iy + sy) % py) * px + (ix + sx) % px
    return out


class UniformRun:
    """px x py patches of n x n cells, periodic, advanced by af_patch_step."""

    def __init__(self, cfg: af.Config, px: int, py: int, dx: float, dy: float, dt: float, device="cuda",
                 state=None, flux_reg: bool = False, tiling=None, field=None, lo=(0.0, 0.0), t0: float = 0.0):
        """field: None (constant velocity cfg.a, cfg.b or acoustics) or
        af.FIELD_SOLID_BODY / af.FIELD_SWIRL (variable-velocity advection on
        the box with lower-left corner lo, starting at time t0)."""
        import torch
        self.cfg, self.px, self.py = cfg, px, py
        self.field, self.lo, self.t = field, (float(lo[0]), float(lo[1])), float(t0)
        self.dx, self.dy, self.dt = dx, dy, dt
        self.npatch = px * py
        self.words = af.patch_words(cfg.n, cfg.ncomp)
        dtype = torch.float64 if cfg.prec == af.F64 else torch.float32
        self.a = torch.zeros((self.npatch, self.words), dtype=dtype, device=device)
        if state is not None:
            self.a.copy_(torch.as_tensor(np.asarray(state).reshape(self.npatch, self.words)).to(dtype))
        self.b = self.a.clone()
        self.nbr = periodic_neighbours(px, py)
        self.device = device
        self.set_tiling(tiling)
        self.freg = (torch.zeros((self.npatch, 4, cfg.ncomp, cfg.n), dtype=torch.float64, device=device)
                     if flux_reg else None)

    def set_tiling(self, tiling=None):
        """Rebuild the work list for a compiled tiling (None: the default)."""
        import torch
        self.tiling = af.default_tiling(self.cfg) if tiling is None else int(tiling)
        p = np.arange(self.npatch)
        w = af.build_step_work(self.cfg, p, nbr=self.nbr, tiling=self.tiling, ix=p % self.px, iy=p // self.px)
        self.nwork = len(w) // 64
        self.work = torch.from_numpy(w).to(self.device)
        self._graph = None  # captured pair of steps (advance); depends on the work list

    def step(self, stream=None):
        if self.field is None:
            af.patch_step(self.cfg, self.work, self.nwork, self.a, self.b, self.dt, self.dx, self.dy,
                          self.freg, stream, tiling=self.tiling)
        else:
            n = self.cfg.n
            hi = (self.lo[0] + self.px * n * self.dx, self.lo[1] + self.py * n * self.dy)
            af.patch_step_var(self.cfg, self.tiling, self.work, self.nwork, af.state_pair(self.a, self.b, 0),
                              af.velocity(self.field, self.lo, hi, self.t), self.dt, self.dx, self.dy, self.freg,
                              stream)
        self.t += self.dt
        self.a, self.b = self.b, self.a

    def advance(self, steps: int, graphs: bool = True):
        """`steps` constant-velocity steps.  With graphs, pairs of steps
        (a -> b -> a, so the buffers end where they started) replay one CUDA
        graph captured the first time (after one eager pair, which sets up the
        kernel attributes outside the capture).  The graph reads the buffer
        that was current at its capture: when the state is in the other one,
        one eager step brings it back first; an odd last step runs eagerly.
        The same launches as `steps` calls of step(), without the host cost of
        one call per step."""
        import torch
        if self.field is not None or not graphs:
            for _ in range(steps):
                self.step()
            return
        k = 0
        # the graph bakes in the step's arguments: capture again if any changed
        key = (self.dt, self.dx, self.dy, None if self.freg is None else self.freg.data_ptr(),
               self.a.data_ptr(), self.b.data_ptr(), self.tiling)
        if self._graph is not None and self._graph[2] != key and self._graph[2] != self._swapped(key):
            self._graph = None
        if self._graph is None and steps >= 4:
            self.step()
            self.step()
            k = 2
            g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            a0, b0, t0 = self.a, self.b, self.t
            with torch.cuda.graph(g, stream=side):
                self.step()
                self.step()
            torch.cuda.current_stream().wait_stream(side)
            self.a, self.b, self.t = a0, b0, t0  # the capture ran nothing
            self._graph = (g, a0, key)
        if self._graph is not None:
            g, a0, _ = self._graph
            if self.a is not a0 and steps - k >= 3:
                self.step()
                k += 1
            while self.a is a0 and steps - k >= 2:
                g.replay()
                self.t += 2 * self.dt
                k += 2
        for _ in range(steps - k):
            self.step()

    @staticmethod
    def _swapped(key):
        """The graph key with the two state buffers exchanged (after an odd
        number of steps)."""
        return key[:4] + (key[5], key[4]) + key[6:]

    def _band_setup(self, bands: int):
        """Work lists of `bands` bands of patch rows, and three streams."""
        import torch
        key = (self.tiling, bands)
        if getattr(self, "_bands_key", None) != key:
            edges = [round(k * self.py / bands) for k in range(bands + 1)]
            self._bands = []
            for b in range(bands):
                p = np.arange(edges[b] * self.px, edges[b + 1] * self.px)
                w = af.build_step_work(self.cfg, p, nbr=self.nbr[p], tiling=self.tiling)
                self._bands.append((int(p[0]), int(p[-1]) + 1, torch.from_numpy(w).to(self.device), len(w) // 64))
            self._streams = [torch.cuda.Stream() for _ in range(3)]
            self._bands_key = key

    def step_host(self, host, bands: int = 16):
        """One step of a state kept in (pinned) host memory, updated in place:
        [npatch, words] like the device arrays.  The grid is split into bands
        of patch rows; each band is copied in, advanced and copied back on
        three streams, so the two copy directions and the step overlap.  A
        band is advanced once it and the neighbouring bands (periodically)
        are on the device.  Everything is enqueued behind, and joined back
        into, the current stream; the caller synchronises."""
        import torch
        if self.field is not None:
            raise ValueError("step_host runs constant-velocity steps")
        bands = max(1, min(int(bands), self.py))
        self._band_setup(bands)
        s_in, s_cmp, s_out = self._streams
        cur = torch.cuda.current_stream()
        for st in self._streams:
            st.wait_stream(cur)
        uploaded = []
        for p0, p1, _, _ in self._bands:
            with torch.cuda.stream(s_in):
                self.a[p0:p1].copy_(host[p0:p1], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s_in)
            uploaded.append(ev)
        order = list(range(1, bands)) + [0]
        for b in order:
            for nb in {(b - 1) % bands, b, (b + 1) % bands}:
                s_cmp.wait_event(uploaded[nb])
            p0, p1, work, nwork = self._bands[b]
            af.patch_step(self.cfg, work, nwork, self.a, self.b, self.dt, self.dx, self.dy, self.freg, s_cmp,
                          tiling=self.tiling)
            done = torch.cuda.Event()
            done.record(s_cmp)
            s_out.wait_event(done)
            with torch.cuda.stream(s_out):
                host[p0:p1].copy_(self.b[p0:p1], non_blocking=True)
        cur.wait_stream(s_out)
        cur.wait_stream(s_cmp)
        self.t += self.dt

    def step_host_owned(self, host, bands: int = 16):
        """step_host for a state kept in host memory in the compact owned
        layout ([npatch, ncomp * 4 * n * n], af_pack_owned's): only the
        patches' own degrees of freedom cross the host link, 74 % of the
        lattice words for 32 x 32 patches.  The bands are copied in back to
        back on one stream; on the compute stream each is unpacked into the
        device state once it has arrived, advanced once it and its
        neighbouring bands are unpacked, and packed; a third stream copies it
        back.  Ghost rings stay on the device and are never needed (every
        patch reads its halo from its neighbours)."""
        import torch
        if self.field is not None:
            raise ValueError("step_host_owned runs constant-velocity steps")
        bands = max(1, min(int(bands), self.py))
        self._band_setup(bands)
        words = af.owned_words(self.cfg.n, self.cfg.ncomp)
        if getattr(self, "_own_bufs", None) is None or self._own_bufs[0].shape != (self.npatch, words):
            self._own_bufs = (torch.empty((self.npatch, words), dtype=self.a.dtype, device=self.device),
                              torch.empty((self.npatch, words), dtype=self.a.dtype, device=self.device))
        own_in, own_out = self._own_bufs
        s_in, s_cmp, s_out = self._streams
        cur = torch.cuda.current_stream()
        for st in self._streams:
            st.wait_stream(cur)
        uploaded = []
        for p0, p1, _, _ in self._bands:  # copies only: the link stays busy
            with torch.cuda.stream(s_in):
                own_in[p0:p1].copy_(host[p0:p1], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s_in)
            uploaded.append(ev)
        order = list(range(1, bands)) + [0]
        unpacked = set()
        for b in order:
            for nb in sorted({(b - 1) % bands, b, (b + 1) % bands} - unpacked):
                q0, q1 = self._bands[nb][:2]
                s_cmp.wait_event(uploaded[nb])
                af.unpack_owned(self.cfg, q1 - q0, own_in[q0:q1], self.a[q0:q1], s_cmp)
                unpacked.add(nb)
            p0, p1, work, nwork = self._bands[b]
            af.patch_step(self.cfg, work, nwork, self.a, self.b, self.dt, self.dx, self.dy, self.freg, s_cmp,
                          tiling=self.tiling)
            af.pack_owned(self.cfg, p1 - p0, self.b[p0:p1], own_out[p0:p1], s_cmp)
            done = torch.cuda.Event()
            done.record(s_cmp)
            s_out.wait_event(done)
            with torch.cuda.stream(s_out):
                host[p0:p1].copy_(own_out[p0:p1], non_blocking=True)
        cur.wait_stream(s_out)
        cur.wait_stream(s_cmp)
        self.t += self.dt

    @property
    def state(self):
        return self.a
