"""Seeded synthetic inputs for the Active Flux patch step.

This module only *generates data*: initial conditions, exact solutions of the
two linear PDEs (used as test references), cell averages of those functions by
Gauss-Legendre quadrature, random degree-of-freedom fields, and the packing of
all of it into the patch-state layout.  It contains none of the method's
arithmetic (no reconstruction, evolution, flux or update) and is the only module
shared by the CPU oracle's tests and the CUDA path.

State layout (the interface contract of the library, Section 2 of the paper,
degrees of freedom of Figure 1):

    state[patch][comp][plane][plane_stride]

plane 0 = cell average Q_{i,j}, plane 1 = left-edge midpoint Q_{i-1/2,j},
plane 2 = lower-left corner Q_{i-1/2,j-1/2}, plane 3 = bottom-edge midpoint
Q_{i,j-1/2}.  Each plane holds a (M+1) x (M+1) row-major lattice (x fastest),
M = N + 2g, g = 2 ghost layers (Section 3.2); lattice index (I, J) = (i+g, j+g)
for cell (i, j), i, j in [-g, N+g].  The plane stride is (M+1)^2 rounded up to
a multiple of 8 elements so every plane starts 32-byte aligned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

G = 2
AVG, XMID, CORNER, YMID = 0, 1, 2, 3


@dataclass(frozen=True)
class Layout:
    n: int            # interior cells per patch side
    ncomp: int        # 1 (advection) or 3 (acoustics: p, u, v)

    @property
    def g(self) -> int:
        return G

    @property
    def m(self) -> int:
        return self.n + 2 * G

    @property
    def w(self) -> int:
        return self.m + 1

    @property
    def plane(self) -> int:
        return (self.w * self.w + 7) // 8 * 8

    @property
    def patch_words(self) -> int:
        return self.ncomp * 4 * self.plane

    def empty(self, npatch: int, fill=np.nan, dtype=np.float64) -> np.ndarray:
        return np.full((npatch, self.ncomp, 4, self.plane), fill, dtype=dtype)

    def lattice(self, arr: np.ndarray) -> np.ndarray:
        """View [..., plane_stride] as [..., W, W] (row J, column I)."""
        return arr[..., : self.w * self.w].reshape(arr.shape[:-1] + (self.w, self.w))


# ---------------------------------------------------------------- quadrature
def gauss_legendre(nq: int):
    x, w = np.polynomial.legendre.leggauss(nq)
    return x, w


def cell_averages(f, xc: np.ndarray, yc: np.ndarray, dx: float, dy: float, nq: int = 5) -> np.ndarray:
    """Average of f over [xc-dx/2, xc+dx/2] x [yc-dy/2, yc+dy/2] (tensor Gauss-Legendre)."""
    gx, gw = gauss_legendre(nq)
    acc = np.zeros(np.broadcast(xc, yc).shape)
    for a in range(nq):
        for b in range(nq):
            acc += gw[a] * gw[b] * f(xc + 0.5 * dx * gx[a], yc + 0.5 * dy * gx[b])
    return acc / 4.0


# ------------------------------------------------------- initial conditions
def gaussian(xc, yc, sigma):
    return lambda x, y: np.exp(-((x - xc) ** 2 + (y - yc) ** 2) / (2.0 * sigma * sigma))


def sinsin_plus_gaussian(x, y):
    """Smooth advection datum: sin(2 pi x) sin(2 pi y) + Gaussian bump (amp 1, sigma 0.05)."""
    return np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) + gaussian(0.5, 0.5, 0.05)(x, y)


def tanh_disc(x, y, x0=0.5, y0=0.5, r0=0.15, eps=0.02):
    """Smoothed disc of Section 4.1: H(r + r0) - H(r - r0), H(r) = (tanh(r/eps)+1)/2."""
    r = np.sqrt((x - x0) ** 2 + (y - y0) ** 2)
    h = lambda s: 0.5 * (np.tanh(s / eps) + 1.0)
    return h(r + r0) - h(r - r0)


def vortex_velocity(xc=0.5, yc=0.5):
    """Stationary vortex of Section 4.6 (speed 5r, 2-5r, 0 with kinks at r = 0.2, 0.4)."""
    def speed_over_r(x, y):
        r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2)
        s = np.where(r <= 0.2, 5.0 * r, np.where(r <= 0.4, 2.0 - 5.0 * r, 0.0))
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(r > 0, s / np.where(r > 0, r, 1.0), 5.0)
    u = lambda x, y: -(y - yc) * speed_over_r(x, y)
    v = lambda x, y: (x - xc) * speed_over_r(x, y)
    return u, v


def pulse_plus_vortex():
    """Acoustic datum: Gaussian pressure pulse (sigma 0.05) at the centre + stationary vortex."""
    u, v = vortex_velocity()
    return [gaussian(0.5, 0.5, 0.05), u, v]


def lukacova_exact(t: float, c: float = 1.0):
    """Closed-form acoustic solution of Section 4.5.1 on [-1,1]^2 (periodic)."""
    tp = 2 * np.pi
    p = lambda x, y: -np.cos(tp * c * t) * (np.sin(tp * x) + np.sin(tp * y)) / c
    u = lambda x, y: np.sin(tp * c * t) * np.cos(tp * x) / c
    v = lambda x, y: np.sin(tp * c * t) * np.cos(tp * y) / c
    return [p, u, v]


def translated(f, a: float, b: float, t: float, lo=(0.0, 0.0), hi=(1.0, 1.0)):
    """Exact advection solution q(x,y,t) = q0(x - a t, y - b t) on a periodic box."""
    lx, ly = hi[0] - lo[0], hi[1] - lo[1]

    def g(x, y):
        xs = lo[0] + np.mod(x - a * t - lo[0], lx)
        ys = lo[1] + np.mod(y - b * t - lo[1], ly)
        return f(xs, ys)
    return g


def ring_wave(x, y):
    """Ring-shaped high-frequency pressure wave exp(-(r-0.25)^2/0.001) cos(80 pi r)."""
    r = np.sqrt(x * x + y * y)
    return np.exp(-((r - 0.25) ** 2) / 0.001) * np.cos(80 * np.pi * r)


def ring_wave_at(r0: float, width: float = 0.001, k: float = 80.0):
    """Ring wave exp(-(r-r0)^2/width) cos(k pi r) around the origin."""
    def f(x, y):
        r = np.sqrt(x * x + y * y)
        return np.exp(-((r - r0) ** 2) / width) * np.cos(k * np.pi * r)
    return f


def per_unit_tree(f, origin=(0.0, 0.0)):
    """f repeated in every unit tree [ox + k, ox + k + 1) x [oy + m, oy + m + 1)
    (k, m integers) of a brick, each copy the values f takes on the tree at
    the origin: g(x, y) = f(ox + frac(x - ox), oy + frac(y - oy))."""
    ox, oy = origin

    def g(x, y):
        return f(ox + np.mod(x - ox, 1.0), oy + np.mod(y - oy, 1.0))
    return g


def swirl_gaussians(x, y):
    """Two Gaussians exp(-100 |x - c|^2) at (0.5, 0.25) and (0.5, 0.75) (Section 4.3)."""
    return np.exp(-100.0 * ((x - 0.5) ** 2 + (y - 0.25) ** 2)) + np.exp(-100.0 * ((x - 0.5) ** 2 + (y - 0.75) ** 2))


def wave_packet(x, y):
    """exp(-r^2/0.01) cos(60 pi x), centred at (0.5, 0.5)."""
    r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2
    return np.exp(-r2 / 0.01) * np.cos(60 * np.pi * x)


# ------------------------------------------------------------ state packing
@dataclass(frozen=True)
class UniformGrid:
    """px x py same-level patches of n x n cells tiling [x0,x1] x [y0,y1]."""
    layout: Layout
    px: int
    py: int
    lo: tuple = (0.0, 0.0)
    hi: tuple = (1.0, 1.0)

    @property
    def npatch(self) -> int:
        return self.px * self.py

    @property
    def dx(self) -> float:
        return (self.hi[0] - self.lo[0]) / (self.px * self.layout.n)

    @property
    def dy(self) -> float:
        return (self.hi[1] - self.lo[1]) / (self.py * self.layout.n)

    def patch_origin(self, p: int):
        ix, iy = p % self.px, p // self.px
        n = self.layout.n
        return self.lo[0] + ix * n * self.dx, self.lo[1] + iy * n * self.dy

    def periodic_neighbours(self) -> np.ndarray:
        """[npatch, 8] same-level neighbour indices, order W, E, S, N, SW, SE, NW, NE."""
        dirs = [(-1, 0), (1, 0), (0, -1), (0, 1), (-1, -1), (1, -1), (-1, 1), (1, 1)]
        out = np.zeros((self.npatch, 8), dtype=np.int32)
        for p in range(self.npatch):
            ix, iy = p % self.px, p // self.px
            for k, (sx, sy) in enumerate(dirs):
                out[p, k] = ((iy + sy) % self.py) * self.px + (ix + sx) % self.px
        return out

    def state(self, funcs, nq: int = 5, ghosts: bool = False, dtype=np.float64,
              periodic: bool = True) -> np.ndarray:
        """Pack cell averages and point values of funcs (one callable per component).

        Interior-owned entries (lattice indices [g, g+N) in both directions) are
        always filled; the ghost ring is filled from the (periodically wrapped)
        analytic functions if ghosts=True, otherwise set to NaN.
        """
        lay = self.layout
        assert len(funcs) == lay.ncomp
        n, g, w = lay.n, G, lay.w
        dx, dy = self.dx, self.dy
        st = lay.empty(self.npatch, dtype=np.float64)
        lat = lay.lattice(st)
        idx = np.arange(w) - g                 # cell / node-line index i for lattice I
        own = (idx >= 0) & (idx < n)
        lx, ly = self.hi[0] - self.lo[0], self.hi[1] - self.lo[1]

        def wrapx(x):
            return self.lo[0] + np.mod(x - self.lo[0], lx) if periodic else x

        def wrapy(y):
            return self.lo[1] + np.mod(y - self.lo[1], ly) if periodic else y

        for p in range(self.npatch):
            ox, oy = self.patch_origin(p)
            xl = ox + idx * dx                     # node lines x_{i-1/2}
            yl = oy + idx * dy
            xc = xl + 0.5 * dx                     # cell centres
            yc = yl + 0.5 * dy
            X_l, Y_l = np.meshgrid(xl, yl)         # [J, I]
            X_c, Y_c = np.meshgrid(xc, yc)
            for c, f in enumerate(funcs):
                wf = lambda x, y, f=f: f(wrapx(x), wrapy(y))
                lat[p, c, AVG] = cell_averages(wf, X_c, Y_c, dx, dy, nq)
                lat[p, c, XMID] = wf(X_l, Y_c)
                lat[p, c, CORNER] = wf(X_l, Y_l)
                lat[p, c, YMID] = wf(X_c, Y_l)
            if not ghosts:
                mask = ~(own[None, :] & own[:, None])
                lat[p][:, :, mask] = np.nan
        return st.astype(dtype)

    def interior_averages(self, st: np.ndarray, comp: int) -> np.ndarray:
        """Global [py*N, px*N] array of interior cell averages of one component."""
        lay = self.layout
        n, g = lay.n, G
        lat = lay.lattice(st)
        out = np.zeros((self.py * n, self.px * n))
        for p in range(self.npatch):
            ix, iy = p % self.px, p // self.px
            out[iy * n:(iy + 1) * n, ix * n:(ix + 1) * n] = lat[p, comp, AVG, g:g + n, g:g + n]
        return out

    def exact_averages(self, f, nq: int = 5) -> np.ndarray:
        n = self.layout.n
        xc = self.lo[0] + (np.arange(self.px * n) + 0.5) * self.dx
        yc = self.lo[1] + (np.arange(self.py * n) + 0.5) * self.dy
        X, Y = np.meshgrid(xc, yc)
        return cell_averages(f, X, Y, self.dx, self.dy, nq)

    def l1_error(self, st: np.ndarray, comp: int, f, nq: int = 5) -> float:
        """sum |Q - Q_exact| dx dy over interior cell averages."""
        d = self.interior_averages(st, comp) - self.exact_averages(f, nq)
        return float(np.abs(d).sum() * self.dx * self.dy)


def random_state(layout: Layout, npatch: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Uniform(-1, 1) values in every entry of every plane (all DOFs independent)."""
    rng = np.random.default_rng(seed)
    st = rng.uniform(-1.0, 1.0, size=(npatch, layout.ncomp, 4, layout.plane))
    return st.astype(dtype)


def cfl_dt(eq: str, cfl: float, dx: float, dy: float, a=1.0, b=0.0, c=1.0) -> float:
    """Largest dt with the given CFL number (Eq. cfl-adv / Eq. cfl-acoustics form)."""
    if eq == "advection":
        return cfl / max(abs(a) / dx, abs(b) / dy)
    return cfl / max(c / dx, c / dy)


def steps_to(t_end: float, dt_max: float):
    """Land exactly on t_end: n = ceil(T / dt_max), dt = T / n."""
    n = int(math.ceil(t_end / dt_max - 1e-12))
    return n, t_end / n


def pack_owned(grid: UniformGrid, owned: np.ndarray, dtype=np.float64) -> np.ndarray:
    """Scatter global owned DOFs owned[comp][plane][py*N][px*N] into a patch state.

    Entry [c][k][J][I] of `owned` is the DOF of plane k owned by global cell
    (I, J); ghost entries of the result are NaN.
    """
    lay = grid.layout
    n, g = lay.n, G
    st = lay.empty(grid.npatch)
    lat = lay.lattice(st)
    for p in range(grid.npatch):
        ix, iy = p % grid.px, p // grid.px
        lat[p, :, :, g:g + n, g:g + n] = owned[:, :, iy * n:(iy + 1) * n, ix * n:(ix + 1) * n]
    return st.astype(dtype)


def unpack_owned(grid: UniformGrid, st: np.ndarray) -> np.ndarray:
    """Inverse of pack_owned: gather interior-owned entries into global arrays."""
    lay = grid.layout
    n, g = lay.n, G
    lat = lay.lattice(st)
    out = np.zeros((lay.ncomp, 4, grid.py * n, grid.px * n), dtype=st.dtype)
    for p in range(grid.npatch):
        ix, iy = p % grid.px, p // grid.px
        out[:, :, iy * n:(iy + 1) * n, ix * n:(ix + 1) * n] = lat[p, :, :, g:g + n, g:g + n]
    return out


def random_owned(grid: UniformGrid, seed: int) -> np.ndarray:
    """Uniform(-1, 1) global owned DOFs for every component and plane."""
    rng = np.random.default_rng(seed)
    n = grid.layout.n
    return rng.uniform(-1.0, 1.0, size=(grid.layout.ncomp, 4, grid.py * n, grid.px * n))


def periodic_state(grid: UniformGrid, funcs, nq: int = 2, dtype=np.float64) -> np.ndarray:
    """Vectorised packing for a periodic grid: every entry (ghost ring
    included) holds the value of the periodically wrapped functions.  Used for
    large synthetic inputs."""
    lay = grid.layout
    n, g, w = lay.n, G, lay.w
    PX, PY = grid.px * n, grid.py * n
    kx = np.arange(-g, PX + g + 1)
    ky = np.arange(-g, PY + g + 1)
    lx, ly = grid.hi[0] - grid.lo[0], grid.hi[1] - grid.lo[1]
    wrap_x = lambda x: grid.lo[0] + np.mod(x - grid.lo[0], lx)
    wrap_y = lambda y: grid.lo[1] + np.mod(y - grid.lo[1], ly)
    xl = grid.lo[0] + kx * grid.dx
    yl = grid.lo[1] + ky * grid.dy
    xc, yc = xl + 0.5 * grid.dx, yl + 0.5 * grid.dy
    st = np.empty((grid.npatch, lay.ncomp, 4, lay.plane), dtype=dtype)
    st[..., w * w:] = 0
    lat = lay.lattice(st).reshape(grid.py, grid.px, lay.ncomp, 4, w, w)
    for c, f in enumerate(funcs):
        wf = lambda x, y, f=f: f(wrap_x(x), wrap_y(y))
        planes = [
            cell_averages(wf, xc[None, :], yc[:, None], grid.dx, grid.dy, nq),
            wf(xl[None, :], yc[:, None]),
            wf(xl[None, :], yl[:, None]),
            wf(xc[None, :], yl[:, None]),
        ]
        for k, arr in enumerate(planes):
            arr = np.ascontiguousarray(arr, dtype=dtype)
            s0, s1 = arr.strides
            win = np.lib.stride_tricks.as_strided(arr, shape=(grid.py, grid.px, w, w),
                                                  strides=(n * s0, n * s1, s0, s1))
            lat[:, :, c, k] = win
    return st


# ------------------------------------------------------------ forest inputs
def _region_has_level(leafset, l, ix, iy, lmin_needed, lmax):
    """True if the level-l region (ix, iy) holds a leaf of level >= lmin_needed."""
    for lv in range(max(lmin_needed, l + 1), lmax + 1):
        s = 1 << (lv - l)
        for dy in range(s):
            for dx in range(s):
                if (lv, ix * s + dx, iy * s + dy) in leafset:
                    return True
    return False


def balanced_forest(B: int, lmin: int, lmax: int, refine) -> list:
    """Leaves (level, ix, iy) of a periodic forest over a B x B brick.

    Starts from all level-lmin patches, refines every leaf for which
    refine(level, ix, iy) is true (up to lmax), then enforces the 2:1 balance
    across faces and corners (a leaf whose neighbour region at its own level
    holds a leaf two or more levels finer is split).  Leaves are returned
    sorted by level, then row-major.  Input generator for tests and benchmarks.
    """
    leaves = {(lmin, ix, iy) for iy in range(B << lmin) for ix in range(B << lmin)}
    changed = True
    while changed:
        changed = False
        for (l, ix, iy) in sorted(leaves):
            if l < lmax and refine(l, ix, iy):
                leaves.remove((l, ix, iy))
                leaves |= {(l + 1, 2 * ix + a, 2 * iy + b) for a in (0, 1) for b in (0, 1)}
                changed = True
    changed = True
    while changed:
        changed = False
        for (l, ix, iy) in sorted(leaves):
            side = B << l
            bad = False
            for sy in (-1, 0, 1):
                for sx in (-1, 0, 1):
                    if sx == 0 and sy == 0:
                        continue
                    if _region_has_level(leaves, l, (ix + sx) % side, (iy + sy) % side, l + 2, lmax):
                        bad = True
            if bad:
                leaves.remove((l, ix, iy))
                leaves |= {(l + 1, 2 * ix + a, 2 * iy + b) for a in (0, 1) for b in (0, 1)}
                changed = True
    return sorted(leaves, key=lambda t: (t[0], t[2], t[1]))


def diagonal_refine(width: float = 0.0):
    """Refine patches that touch the diagonal y = x of the unit brick."""
    def pred(l, ix, iy):
        return abs(ix - iy) <= 0 + width
    return pred


def forest_state(n: int, ncomp: int, B: int, lmax: int, leaves, funcs, lo=(0.0, 0.0), hi=(1.0, 1.0),
                 nq: int = 3, dtype=np.float64) -> np.ndarray:
    """Pack the initial data of every leaf (all entries, ghosts from the
    periodically wrapped functions)."""
    lay = Layout(n, ncomp)
    out = np.empty((len(leaves), ncomp, 4, lay.plane))
    for k, (l, ix, iy) in enumerate(leaves):
        side = B << l
        w = (hi[0] - lo[0]) / side
        h = (hi[1] - lo[1]) / side
        g1 = UniformGrid(lay, 1, 1, (lo[0] + ix * w, lo[1] + iy * h), (lo[0] + (ix + 1) * w, lo[1] + (iy + 1) * h))
        lx, ly = hi[0] - lo[0], hi[1] - lo[1]
        wrapped = [lambda x, y, f=f: f(lo[0] + np.mod(x - lo[0], lx), lo[1] + np.mod(y - lo[1], ly)) for f in funcs]
        out[k] = g1.state(wrapped, nq=nq, ghosts=True, periodic=False)[0]
    return out.astype(dtype)


def forest_state_fast(n: int, ncomp: int, B: int, level, ix, iy, funcs, lo=(0.0, 0.0), hi=(1.0, 1.0),
                      nq: int = 2, dtype=np.float64, chunk: int = 2048) -> np.ndarray:
    """Vectorised forest_state for large forests: leaves given as arrays, in
    that order; every entry (ghost ring included) holds the periodically
    wrapped functions' values (cell averages by nq x nq Gauss-Legendre)."""
    lay = Layout(n, ncomp)
    level, ix, iy = (np.asarray(a, dtype=np.int64) for a in (level, ix, iy))
    P, w = len(level), lay.w
    out = np.zeros((P, ncomp, 4, lay.plane), dtype=dtype)
    lat = lay.lattice(out)
    lx, ly = hi[0] - lo[0], hi[1] - lo[1]
    idx = np.arange(w) - G
    wraps = [lambda x, y, f=f: f(lo[0] + np.mod(x - lo[0], lx), lo[1] + np.mod(y - lo[1], ly)) for f in funcs]
    for s in range(0, P, chunk):
        e = min(P, s + chunk)
        side = (B << level[s:e]).astype(np.float64)
        dx, dy = lx / (side * n), ly / (side * n)                      # [p]
        ox, oy = lo[0] + ix[s:e] * n * dx, lo[1] + iy[s:e] * n * dy
        xl = ox[:, None] + idx[None, :] * dx[:, None]                   # [p, I]
        yl = oy[:, None] + idx[None, :] * dy[:, None]                   # [p, J]
        xc, yc = xl + 0.5 * dx[:, None], yl + 0.5 * dy[:, None]
        XL, YL = xl[:, None, :], yl[:, :, None]                         # [p, J, I]
        XC, YC = xc[:, None, :], yc[:, :, None]
        DX, DY = dx[:, None, None], dy[:, None, None]
        for c, f in enumerate(wraps):
            lat[s:e, c, AVG] = cell_averages(f, XC, YC, DX, DY, nq)
            lat[s:e, c, XMID] = f(XL, YC)
            lat[s:e, c, CORNER] = f(XL, YL)
            lat[s:e, c, YMID] = f(XC, YL)
    return out


def refine_band(B: int, lo, hi, inside):
    """Refinement predicate on arrays: a level-l region (ix, iy) of the B x B
    brick over [lo, hi] is refined if inside(x, y) holds at any of its 5 x 5
    sample points (corners, edges and interior)."""
    def pred(l, ix, iy):
        side = B << np.asarray(l)
        w, h = (hi[0] - lo[0]) / side, (hi[1] - lo[1]) / side
        t = np.linspace(0.0, 1.0, 5)
        x = lo[0] + (np.asarray(ix)[..., None, None] + t[None, :]) * np.asarray(w)[..., None, None]
        y = lo[1] + (np.asarray(iy)[..., None, None] + t[:, None]) * np.asarray(h)[..., None, None]
        return inside(x, y).any(axis=(-1, -2))
    return pred
