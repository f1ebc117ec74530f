"""Thin Python binding of libaf.so (include/af.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module converts
arguments (torch tensors -> device pointers, numpy arrays -> host pointers,
torch streams -> cudaStream_t) and raises AFError on a non-zero status.
There is no fallback: if libaf.so is missing the first call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaf.so")

ADVECTION, ACOUSTICS = 0, 1
F64, F32 = 0, 1


class AFError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)}" if what else status_string(status))


class Config(C.Structure):
    _fields_ = [("eq", C.c_int32), ("prec", C.c_int32), ("n", C.c_int32), ("ncomp", C.c_int32),
                ("a", C.c_double), ("b", C.c_double), ("c", C.c_double)]


class Work(C.Structure):
    _fields_ = [("patch", C.c_int32), ("level", C.c_int32), ("nbr", C.c_int32 * 8),
                ("x0", C.c_int16), ("x1", C.c_int16), ("y0", C.c_int16), ("y1", C.c_int16),
                ("flags", C.c_int32), ("ix", C.c_int32), ("iy", C.c_int32), ("pad_", C.c_int32)]


assert C.sizeof(Work) == 64

_lib = None
_VP, _DP, _IP = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)


def lib():
    """Load libaf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2205_07572_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        L.af_status_string.restype = C.c_char_p
        L.af_status_string.argtypes = [C.c_int]
        L.af_plane_stride.restype = C.c_int64
        L.af_plane_stride.argtypes = [C.c_int32]
        L.af_patch_words.restype = C.c_int64
        L.af_patch_words.argtypes = [C.c_int32, C.c_int32]
        L.af_build_step_work.restype = C.c_int
        L.af_build_step_work.argtypes = [C.POINTER(Config), C.c_int32, _IP, _IP, _IP, C.POINTER(Work),
                                         C.c_int32, _IP]
        L.af_patch_step.restype = C.c_int
        L.af_patch_step.argtypes = [C.POINTER(Config), C.c_int32, _VP, _VP, _VP, C.c_double, C.c_double,
                                    C.c_double, _VP, _VP]
        L.af_build_step_work_tiled.restype = C.c_int
        L.af_build_step_work_tiled.argtypes = [C.POINTER(Config), C.c_int32, C.c_int32, _IP, _IP, _IP,
                                               C.POINTER(Work), C.c_int32, _IP]
        L.af_patch_step_tiled.restype = C.c_int
        L.af_patch_step_tiled.argtypes = [C.POINTER(Config), C.c_int32, C.c_int32, _VP, _VP, _VP, C.c_double,
                                          C.c_double, C.c_double, _VP, _VP]
        L.af_step_tilings.restype = C.c_int32
        L.af_step_tilings.argtypes = [C.c_void_p, C.c_int32]
        L.af_step_default_tiling.restype = C.c_int32
        L.af_step_default_tiling.argtypes = [C.POINTER(Config)]
        L.af_build_step_work_at.restype = C.c_int
        L.af_build_step_work_at.argtypes = [C.POINTER(Config), C.c_int32, C.c_int32, _IP, _IP, _IP, _IP, _IP,
                                            C.POINTER(Work), C.c_int32, _IP]
        _register_more(L)
        _lib = L
    return _lib


def _register_more(L):
    """Signatures of the entry points added beside the step (fill, reflux, tag)."""
    for name, res, args in _EXTRA:
        if hasattr(L, name):
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args


_EXTRA: list = []


def status_string(s: int) -> str:
    return lib().af_status_string(int(s)).decode()


def _check(st: int, what: str):
    if st != 0:
        raise AFError(st, what)


def ptr(x):
    """Device/host address of a torch tensor, numpy array or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def config(eq: int, prec: int, n: int, a: float = 0.0, b: float = 0.0, c: float = 1.0) -> Config:
    return Config(eq, prec, n, 1 if eq == ADVECTION else 3, a, b, c)


def plane_stride(n: int) -> int:
    return int(lib().af_plane_stride(n))


def patch_words(n: int, ncomp: int) -> int:
    return int(lib().af_patch_words(n, ncomp))


class Tiling(C.Structure):
    _fields_ = [("tile_x", C.c_int32), ("tile_y", C.c_int32), ("threads", C.c_int32), ("persistent", C.c_int32)]


def step_tilings():
    """Compiled tilings of af_patch_step: list of (tile_x, tile_y, threads, persistent)."""
    L = lib()
    n = L.af_step_tilings(None, 0)
    buf = (Tiling * n)()
    L.af_step_tilings(buf, n)
    return [(t.tile_x, t.tile_y, t.threads, t.persistent) for t in buf]


def default_tiling(cfg: Config) -> int:
    return int(lib().af_step_default_tiling(C.byref(cfg)))


def build_step_work(cfg: Config, patches, levels=None, nbr=None, tiling=None, ix=None, iy=None) -> np.ndarray:
    """Host work list of af_patch_step as a uint8 array (64 bytes per entry);
    ix, iy (patch positions) are needed by patch_step_var only."""
    patches = np.ascontiguousarray(patches, dtype=np.int32)
    lv = None if levels is None else np.ascontiguousarray(levels, dtype=np.int32)
    nb = None if nbr is None else np.ascontiguousarray(nbr, dtype=np.int32).reshape(-1)
    px = None if ix is None else np.ascontiguousarray(ix, dtype=np.int32)
    py = None if iy is None else np.ascontiguousarray(iy, dtype=np.int32)
    npatch = len(patches)
    L = lib()
    k = default_tiling(cfg) if tiling is None else int(tiling)
    cnt = C.c_int32(0)
    ip = lambda a: None if a is None else a.ctypes.data_as(_IP)
    # a first guess of the capacity (four tiles per patch), then the count the
    # library reports if that was too small
    cap = 4 * npatch + 8
    for _ in range(2):
        buf = np.empty(64 * cap, dtype=np.uint8)
        st = L.af_build_step_work_at(C.byref(cfg), k, npatch, ip(patches), ip(lv), ip(px), ip(py), ip(nb),
                                     buf.ctypes.data_as(C.POINTER(Work)), cap, C.byref(cnt))
        if st == 0 or cnt.value <= cap:
            break
        cap = cnt.value
    _check(st, "af_build_step_work")
    return buf[:64 * cnt.value].copy() if cnt.value < cap else buf


def patch_step(cfg: Config, work, nwork: int, state_in, state_out, dt0: float, dx0: float, dy0: float,
               flux_reg=None, stream=None, tiling=None) -> None:
    if tiling is None:
        st = lib().af_patch_step(C.byref(cfg), int(nwork), ptr(work), ptr(state_in), ptr(state_out),
                                 float(dt0), float(dx0), float(dy0), ptr(flux_reg), stream_handle(stream))
    else:
        st = lib().af_patch_step_tiled(C.byref(cfg), int(tiling), int(nwork), ptr(work), ptr(state_in),
                                       ptr(state_out), float(dt0), float(dx0), float(dy0), ptr(flux_reg),
                                       stream_handle(stream))
    _check(st, "af_patch_step")


# ------------------------------------------------------------------- forest
FILL_SAME_LEVEL_ONLY = 1
FILL_ALL_PATCHES = 2


class ForestC(C.Structure):
    _fields_ = [("nleaf", C.c_int32), ("B", C.c_int32), ("lmax", C.c_int32), ("pad_", C.c_int32),
                ("d_level", C.c_void_p), ("d_ix", C.c_void_p), ("d_iy", C.c_void_p), ("d_map", C.c_void_p)]


_FP = C.POINTER(ForestC)
_EXTRA += [
    ("af_forest_map_offset", C.c_int64, [C.c_int32, C.c_int32]),
    ("af_forest_build_map", C.c_int, [C.c_int32, C.c_int32, C.c_int32, _IP, _IP, _IP, _IP]),
    ("af_fill_ghosts", C.c_int, [C.POINTER(Config), _FP, C.c_uint32, C.c_uint32, C.c_int32, _VP, _VP]),
    ("af_transfer", C.c_int, [C.POINTER(Config), _FP, _VP, _FP, _VP, _VP]),
    ("af_reflux", C.c_int, [C.POINTER(Config), _FP, C.c_uint32, C.c_double, C.c_double, _VP, _VP, _VP]),
    ("af_tag", C.c_int, [C.POINTER(Config), _FP, _VP, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                         C.c_double, _VP, _VP, _VP]),
    ("af_mass_scratch_bytes", C.c_int64, [C.c_int32, C.c_int32]),
    ("af_mass", C.c_int, [C.POINTER(Config), _FP, _VP, C.c_double, C.c_double, _VP, _VP, _VP]),
]
if _lib is not None:
    _register_more(_lib)


def forest_map_offset(B: int, level: int) -> int:
    return int(lib().af_forest_map_offset(B, level))


def forest_build_map(B: int, lmax: int, level, ix, iy) -> np.ndarray:
    level = np.ascontiguousarray(level, dtype=np.int32)
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    out = np.empty(forest_map_offset(B, lmax + 1), dtype=np.int32)
    ip = lambda a: a.ctypes.data_as(_IP)
    _check(lib().af_forest_build_map(len(level), B, lmax, ip(level), ip(ix), ip(iy), ip(out)), "af_forest_build_map")
    return out


def forest_struct(nleaf: int, B: int, lmax: int, d_level, d_ix, d_iy, d_map) -> ForestC:
    return ForestC(nleaf, B, lmax, 0, ptr(d_level), ptr(d_ix), ptr(d_iy), ptr(d_map))


def fill_ghosts(cfg: Config, forest: ForestC, dst_levels: int, src_levels: int, flags: int, state, stream=None):
    _check(lib().af_fill_ghosts(C.byref(cfg), C.byref(forest), dst_levels, src_levels, flags, ptr(state),
                                stream_handle(stream)), "af_fill_ghosts")


def transfer(cfg: Config, old: ForestC, d_old, new: ForestC, d_new, stream=None):
    _check(lib().af_transfer(C.byref(cfg), C.byref(old), ptr(d_old), C.byref(new), ptr(d_new),
                             stream_handle(stream)), "af_transfer")


def reflux(cfg: Config, forest: ForestC, sync_levels: int, dx0: float, dy0: float, flux_reg, state, stream=None):
    _check(lib().af_reflux(C.byref(cfg), C.byref(forest), sync_levels, dx0, dy0, ptr(flux_reg), ptr(state),
                           stream_handle(stream)), "af_reflux")


def tag(cfg: Config, forest: ForestC, state, comp: int, kind: int, dx0: float, dy0: float, refine_thr: float,
        coarsen_thr: float, tags, indicator=None, stream=None):
    _check(lib().af_tag(C.byref(cfg), C.byref(forest), ptr(state), comp, kind, dx0, dy0, refine_thr, coarsen_thr,
                        ptr(tags), ptr(indicator), stream_handle(stream)), "af_tag")


def mass_scratch_bytes(nleaf: int, ncomp: int) -> int:
    return int(lib().af_mass_scratch_bytes(nleaf, ncomp))


def mass(cfg: Config, forest: ForestC, state, dx0: float, dy0: float, scratch, out, stream=None):
    _check(lib().af_mass(C.byref(cfg), C.byref(forest), ptr(state), dx0, dy0, ptr(scratch), ptr(out),
                         stream_handle(stream)), "af_mass")


_EXTRA += [("af_mass_noalloc", C.c_int, [C.POINTER(Config), _FP, _VP, C.c_double, C.c_double, _VP, _VP])]
if _lib is not None:
    _register_more(_lib)


def mass_noalloc(cfg: Config, forest: ForestC, state, dx0: float, dy0: float, out, stream=None):
    """af_mass with the library's fixed scratch array (no allocation)."""
    _check(lib().af_mass_noalloc(C.byref(cfg), C.byref(forest), ptr(state), dx0, dy0, ptr(out),
                                 stream_handle(stream)), "af_mass_noalloc")


# --------------------------------------------------------------- state pairs
class StatePair(C.Structure):
    """af_state_pair: level l's current values are in buf[(parity >> l) & 1]."""
    _fields_ = [("buf", C.c_void_p * 2), ("parity", C.c_uint32), ("pad_", C.c_uint32)]


_SP = C.POINTER(StatePair)
_EXTRA += [
    ("af_patch_step_pair", C.c_int, [C.POINTER(Config), C.c_int32, C.c_int32, _VP, _SP, C.c_double, C.c_double,
                                     C.c_double, _VP, _VP]),
    ("af_fill_ghosts_pair", C.c_int, [C.POINTER(Config), _FP, C.c_uint32, C.c_uint32, C.c_int32, _SP, _VP]),
    ("af_transfer_pair", C.c_int, [C.POINTER(Config), _FP, _SP, _FP, _VP, _VP]),
    ("af_reflux_pair", C.c_int, [C.POINTER(Config), _FP, C.c_uint32, C.c_double, C.c_double, _VP, _SP, _VP]),
    ("af_tag_pair", C.c_int, [C.POINTER(Config), _FP, _SP, C.c_int32, C.c_int32, C.c_double, C.c_double,
                              C.c_double, C.c_double, _VP, _VP, _VP]),
    ("af_mass_pair", C.c_int, [C.POINTER(Config), _FP, _SP, C.c_double, C.c_double, _VP, _VP, _VP]),
]
if _lib is not None:
    _register_more(_lib)


def state_pair(buf0, buf1, parity: int) -> StatePair:
    p = StatePair()
    p.buf[0] = ptr(buf0)
    p.buf[1] = ptr(buf1)
    p.parity = int(parity) & 0xFFFFFFFF
    return p


def patch_step_pair(cfg: Config, tiling: int, work, nwork: int, pair: StatePair, dt0: float, dx0: float, dy0: float,
                    flux_reg=None, stream=None) -> None:
    _check(lib().af_patch_step_pair(C.byref(cfg), int(tiling), int(nwork), ptr(work), C.byref(pair), float(dt0),
                                    float(dx0), float(dy0), ptr(flux_reg), stream_handle(stream)),
           "af_patch_step_pair")


def fill_ghosts_pair(cfg: Config, forest: ForestC, dst_levels: int, src_levels: int, flags: int, pair: StatePair,
                     stream=None):
    _check(lib().af_fill_ghosts_pair(C.byref(cfg), C.byref(forest), dst_levels, src_levels, flags, C.byref(pair),
                                     stream_handle(stream)), "af_fill_ghosts_pair")


def transfer_pair(cfg: Config, old: ForestC, old_pair: StatePair, new: ForestC, d_new, stream=None):
    _check(lib().af_transfer_pair(C.byref(cfg), C.byref(old), C.byref(old_pair), C.byref(new), ptr(d_new),
                                  stream_handle(stream)), "af_transfer_pair")


def reflux_pair(cfg: Config, forest: ForestC, sync_levels: int, dx0: float, dy0: float, flux_reg, pair: StatePair,
                stream=None):
    _check(lib().af_reflux_pair(C.byref(cfg), C.byref(forest), sync_levels, dx0, dy0, ptr(flux_reg),
                                C.byref(pair), stream_handle(stream)), "af_reflux_pair")


def tag_pair(cfg: Config, forest: ForestC, pair: StatePair, comp: int, kind: int, dx0: float, dy0: float,
             refine_thr: float, coarsen_thr: float, tags, indicator=None, stream=None):
    _check(lib().af_tag_pair(C.byref(cfg), C.byref(forest), C.byref(pair), comp, kind, dx0, dy0, refine_thr,
                             coarsen_thr, ptr(tags), ptr(indicator), stream_handle(stream)), "af_tag_pair")


def mass_pair(cfg: Config, forest: ForestC, pair: StatePair, dx0: float, dy0: float, scratch, out, stream=None):
    _check(lib().af_mass_pair(C.byref(cfg), C.byref(forest), C.byref(pair), dx0, dy0, ptr(scratch), ptr(out),
                              stream_handle(stream)), "af_mass_pair")


# --------------------------------------------------------------- ghost plan
GHOST_ENTRY_BYTES = 16
_EXTRA += [
    ("af_ghost_plan_count", C.c_int, [C.POINTER(Config), _FP, C.c_int32, _VP, _VP]),
    ("af_ghost_plan_build", C.c_int, [C.POINTER(Config), _FP, C.c_int32, _VP, C.c_int64, C.c_int64, _VP, _VP]),
    ("af_fill_ghosts_planned", C.c_int, [C.POINTER(Config), _FP, C.c_uint32, C.c_int32, _VP, C.c_int64, C.c_int64,
                                         _SP, _VP]),
]
if _lib is not None:
    _register_more(_lib)


def ghost_plan(cfg: Config, forest: ForestC, flags: int = 0, device="cuda", stream=None):
    """Build the ghost plan of a forest: returns (plan tensor, n_a, n_b).
    Reads the two counts back to the host (one stream synchronisation)."""
    import torch
    counts = torch.zeros(2, dtype=torch.int64, device=device)
    _check(lib().af_ghost_plan_count(C.byref(cfg), C.byref(forest), flags, ptr(counts), stream_handle(stream)),
           "af_ghost_plan_count")
    n_a, n_b = (int(v) for v in counts.cpu().tolist())
    plan = torch.empty(max(1, (n_a + n_b) * GHOST_ENTRY_BYTES // 8), dtype=torch.int64, device=device)
    scratch = torch.empty(4, dtype=torch.int64, device=device)
    _check(lib().af_ghost_plan_build(C.byref(cfg), C.byref(forest), flags, ptr(plan), n_a, n_b, ptr(scratch),
                                     stream_handle(stream)), "af_ghost_plan_build")
    if int(scratch[2].item()) != 0:
        raise AFError(1, "af_ghost_plan_build: counts too small")
    return plan, n_a, n_b


def fill_ghosts_planned(cfg: Config, forest: ForestC, levels: int, flags: int, plan, n_a: int, n_b: int,
                        pair: StatePair, stream=None):
    _check(lib().af_fill_ghosts_planned(C.byref(cfg), C.byref(forest), levels, flags, ptr(plan), n_a, n_b,
                                        C.byref(pair), stream_handle(stream)), "af_fill_ghosts_planned")


# ------------------------------------------------------- learned tagger
_EXTRA += [
    ("af_cnn_param_count", C.c_int64, [C.c_int32]),
    ("af_cnn_inputs", C.c_int, [C.POINTER(Config), _FP, _SP, _VP, C.c_double, C.c_double, _VP, _VP]),
    ("af_cnn_forward", C.c_int, [C.c_int32, C.c_int32, C.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("af_cnn_partial_floats", C.c_int64, [C.c_int32, C.c_int32]),
    ("af_cnn_backward", C.c_int, [C.c_int32, C.c_int32, C.c_int32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP,
                                  C.c_double, _VP, C.c_int32, _VP, _VP]),
    ("af_cnn_adam", C.c_int, [C.c_int64, _VP, _VP, _VP, _VP, C.c_int32, C.c_double, C.c_double, C.c_double,
                              C.c_double, _VP]),
    ("af_cnn_tags", C.c_int, [C.c_int32, _VP, _VP, C.c_double, _VP, _VP, _VP]),
]
if _lib is not None:
    _register_more(_lib)


def cnn_param_count(ncomp: int) -> int:
    return int(lib().af_cnn_param_count(ncomp))


def cnn_inputs(cfg: Config, forest: ForestC, pair: StatePair, nbr, dx0: float, thr: float, x, stream=None):
    _check(lib().af_cnn_inputs(C.byref(cfg), C.byref(forest), C.byref(pair), ptr(nbr), dx0, thr, ptr(x),
                               stream_handle(stream)), "af_cnn_inputs")


def cnn_forward(ncomp: int, n: int, nsample: int, x, level, params, logit, m, arg, stream=None):
    _check(lib().af_cnn_forward(ncomp, n, nsample, ptr(x), ptr(level), ptr(params), ptr(logit), ptr(m), ptr(arg),
                                stream_handle(stream)), "af_cnn_forward")


def cnn_partial_floats(ncomp: int, nblocks: int) -> int:
    return int(lib().af_cnn_partial_floats(ncomp, nblocks))


def cnn_backward(ncomp: int, n: int, nsample: int, x, level, params, logit, m, arg, label, weight,
                 weight_sum: float, partial, nblocks: int, grad, stream=None):
    _check(lib().af_cnn_backward(ncomp, n, nsample, ptr(x), ptr(level), ptr(params), ptr(logit), ptr(m), ptr(arg),
                                 ptr(label), ptr(weight), float(weight_sum), ptr(partial), nblocks, ptr(grad),
                                 stream_handle(stream)), "af_cnn_backward")


def cnn_adam(nparam: int, params, m, v, grad, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().af_cnn_adam(nparam, ptr(params), ptr(m), ptr(v), ptr(grad), step, lr, beta1, beta2, eps,
                             stream_handle(stream)), "af_cnn_adam")


def cnn_tags(nleaf: int, logit, plain, cmin: float, tags, nfallback, stream=None):
    _check(lib().af_cnn_tags(nleaf, ptr(logit), ptr(plain), cmin, ptr(tags), ptr(nfallback),
                             stream_handle(stream)), "af_cnn_tags")



# ------------------------------------------------- variable-velocity advection
FIELD_SOLID_BODY, FIELD_SWIRL = 0, 1


class Velocity(C.Structure):
    _fields_ = [("field", C.c_int32), ("pad_", C.c_int32), ("x_lo", C.c_double), ("y_lo", C.c_double),
                ("x_hi", C.c_double), ("y_hi", C.c_double), ("t", C.c_double)]


_EXTRA += [("af_patch_step_var", C.c_int, [C.POINTER(Config), C.c_int32, C.c_int32, _VP, _SP, C.POINTER(Velocity),
                                           C.c_double, C.c_double, C.c_double, _VP, _VP])]
if _lib is not None:
    _register_more(_lib)


def velocity(field: int, lo, hi, t: float) -> Velocity:
    return Velocity(field, 0, float(lo[0]), float(lo[1]), float(hi[0]), float(hi[1]), float(t))


def patch_step_var(cfg: Config, tiling: int, work, nwork: int, pair: StatePair, vel: Velocity, dt0: float,
                   dx0: float, dy0: float, flux_reg=None, stream=None) -> None:
    _check(lib().af_patch_step_var(C.byref(cfg), int(tiling), int(nwork), ptr(work), C.byref(pair), C.byref(vel),
                                   float(dt0), float(dx0), float(dy0), ptr(flux_reg), stream_handle(stream)),
           "af_patch_step_var")


_EXTRA += [("af_step_wait_timeouts", C.c_int, [C.POINTER(C.c_uint32), C.c_int32])]
if _lib is not None:
    _register_more(_lib)


WORK_SKIP_BULK_COPY = 2  # af_work.flags bit: failure injection, the tile's bulk copies are not issued


def step_wait_timeouts(reset: bool = False) -> int:
    """Tiles whose bounded wait on a bulk copy gave up (synchronises)."""
    v = C.c_uint32(0)
    _check(lib().af_step_wait_timeouts(C.byref(v), 1 if reset else 0), "af_step_wait_timeouts")
    return int(v.value)


_EXTRA += [("af_pack_owned", C.c_int, [C.POINTER(Config), C.c_int32, _VP, _VP, _VP]),
           ("af_unpack_owned", C.c_int, [C.POINTER(Config), C.c_int32, _VP, _VP, _VP])]
if _lib is not None:
    _register_more(_lib)


def owned_words(n: int, ncomp: int) -> int:
    """Elements of one patch in the compact owned layout: ncomp * 4 * n * n."""
    return ncomp * 4 * n * n


def pack_owned(cfg: Config, npatch: int, state, owned, stream=None) -> None:
    """af_pack_owned: lattice state -> compact [patch][comp][plane][n][n]."""
    _check(lib().af_pack_owned(C.byref(cfg), int(npatch), ptr(state), ptr(owned), stream_handle(stream)),
           "af_pack_owned")


def unpack_owned(cfg: Config, npatch: int, owned, state, stream=None) -> None:
    """af_unpack_owned: compact owned entries -> lattice state (ghosts untouched)."""
    _check(lib().af_unpack_owned(C.byref(cfg), int(npatch), ptr(owned), ptr(state), stream_handle(stream)),
           "af_unpack_owned")


_EXTRA += [("af_fma_probe_threads", C.c_int32, []),
           ("af_fma_throughput", C.c_int, [C.c_int32, C.c_int32, C.c_int32, _VP, _VP])]
if _lib is not None:
    _register_more(_lib)


def fma_throughput(prec: int, blocks: int, iters: int, sink, stream=None) -> None:
    """af_fma_throughput: 2 * 8 * iters * blocks * 256 flops of FMA chains."""
    _check(lib().af_fma_throughput(int(prec), int(blocks), int(iters), ptr(sink), stream_handle(stream)),
           "af_fma_throughput")
