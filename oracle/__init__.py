"""FP64 CPU oracle of the Active Flux method (arXiv 2205.07572) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and the oracle never imports the product.
The C source ``af_oracle.c`` is compiled with plain gcc into ``liboracle.so``
next to it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "af_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ADVECTION, ACOUSTICS = 0, 1
CORNER, XMID, YMID = 0, 1, 2   # node types of orc_node_evolve


class Cfg(C.Structure):
    _fields_ = [("eq", C.c_int32), ("n", C.c_int32), ("ncomp", C.c_int32), ("pad_", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("dt", C.c_double),
                ("a", C.c_double), ("b", C.c_double), ("c", C.c_double)]


SOLID_BODY, SWIRL = 0, 1   # velocity fields of the variable-velocity advection


class VarCfg(C.Structure):
    """Variable-velocity advection (Sections 4.2, 4.3): field, mesh widths,
    time step, position of the patch's node line 0, time t^n."""
    _fields_ = [("n", C.c_int32), ("field", C.c_int32), ("dx", C.c_double), ("dy", C.c_double),
                ("dt", C.c_double), ("x0", C.c_double), ("y0", C.c_double), ("t", C.c_double)]


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O2 -fopenmp).  Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        L.orc_plane_stride.restype = C.c_long
        L.orc_plane_stride.argtypes = [C.c_int]
        L.orc_recon_eval.restype = C.c_double
        L.orc_recon_eval.argtypes = [C.c_int, C.c_int, dp, C.c_int, C.c_int, C.c_int,
                                     C.c_double, C.c_double, C.c_int, C.c_int, C.c_double, C.c_double]
        L.orc_node_evolve.restype = None
        L.orc_node_evolve.argtypes = [C.POINTER(Cfg), dp, C.c_int, C.c_int, C.c_int, C.c_double, dp]
        L.orc_step_patch.restype = None
        L.orc_step_patch.argtypes = [C.POINTER(Cfg), dp, dp, dp]
        L.orc_fill_periodic.restype = None
        L.orc_fill_periodic.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp]
        L.orc_run_uniform.restype = None
        L.orc_run_uniform.argtypes = [C.POINTER(Cfg), C.c_int, C.c_int, C.c_int, dp, dp, C.c_int]
        L.orc_max_threads.restype = C.c_int
        ip = C.POINTER(C.c_int32)
        L.orc_fill_amr.restype = None
        L.orc_fill_amr.argtypes = [C.c_int, C.c_int, C.c_int, ip, ip, ip, C.c_int, C.c_int, C.c_uint32,
                                   C.c_uint32, C.c_int, dp, dp]
        L.orc_reflux_amr.restype = None
        L.orc_reflux_amr.argtypes = [C.c_int, C.c_int, C.c_int, ip, ip, ip, C.c_int, C.c_int, C.c_uint32,
                                     C.c_double, C.c_double, dp, dp]
        L.orc_tag.restype = None
        L.orc_tag.argtypes = [C.c_int, C.c_int, C.c_int, ip, dp, C.c_int, C.c_int, C.c_double, C.c_double,
                              C.c_double, C.c_double, C.POINTER(C.c_int8), dp]
        L.orc_mass.restype = None
        L.orc_mass.argtypes = [C.c_int, C.c_int, C.c_int, ip, dp, C.c_double, C.c_double, dp]
        L.orc_transfer.restype = None
        L.orc_transfer.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, ip, ip, ip, dp, C.c_int, ip, ip,
                                   ip, dp]
        vp = C.POINTER(VarCfg)
        L.orc_var_velocity.restype = None
        L.orc_var_velocity.argtypes = [vp, C.c_double, C.c_double, C.c_double, dp]
        L.orc_var_foot.restype = None
        L.orc_var_foot.argtypes = [vp, C.c_double, C.c_double, C.c_double, dp]
        L.orc_node_evolve_var.restype = C.c_double
        L.orc_node_evolve_var.argtypes = [vp, dp, C.c_int, C.c_int, C.c_int, C.c_double]
        L.orc_step_patch_var.restype = None
        L.orc_step_patch_var.argtypes = [vp, dp, dp, dp]
        L.orc_run_uniform_var.restype = None
        L.orc_run_uniform_var.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, dp, dp, C.c_int]
        L.orc_step_patches.restype = None
        L.orc_step_patches.argtypes = [C.POINTER(Cfg), vp, dp, dp, C.c_int, ip, C.c_long, dp, dp, C.c_long, C.c_int]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def cfg(eq: int, n: int, dx: float, dy: float, dt: float, a=0.0, b=0.0, c=1.0) -> Cfg:
    return Cfg(eq, n, 1 if eq == ADVECTION else 3, 0, dx, dy, dt, a, b, c)


def recon_eval(n, ncomp, patch, comp, i, j, xi, eta, mx=0, my=0, dx=1.0, dy=1.0) -> float:
    patch = np.ascontiguousarray(patch, dtype=np.float64)
    return lib().orc_recon_eval(n, ncomp, _dp(patch), comp, i, j, xi, eta, mx, my, dx, dy)


def node_evolve(cf: Cfg, patch, node_type: int, i: int, j: int, tau: float) -> np.ndarray:
    patch = np.ascontiguousarray(patch, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_node_evolve(C.byref(cf), _dp(patch), node_type, i, j, tau, _dp(out))
    return out[: cf.ncomp]


def step_patch(cf: Cfg, patch, freg=None) -> np.ndarray:
    patch = np.ascontiguousarray(patch, dtype=np.float64)
    out = np.empty_like(patch)
    fr = None if freg is None else _dp(freg)
    lib().orc_step_patch(C.byref(cf), _dp(patch), _dp(out), fr)
    return out


def fill_periodic(n: int, ncomp: int, px: int, py: int, state: np.ndarray) -> None:
    lib().orc_fill_periodic(n, ncomp, px, py, _dp(state))


def run_uniform(cf: Cfg, px: int, py: int, nsteps: int, state: np.ndarray, nthreads: int = 0) -> np.ndarray:
    """Advance a periodic px x py patch array nsteps steps (returns a new array)."""
    st = np.ascontiguousarray(state, dtype=np.float64).copy()
    tmp = np.empty_like(st)
    nt = nthreads if nthreads > 0 else max_threads()
    lib().orc_run_uniform(C.byref(cf), px, py, nsteps, _dp(st), _dp(tmp), nt)
    return st


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ------------------------------------------------ variable-velocity advection
def var_velocity(vc: VarCfg, x: float, y: float, t: float) -> np.ndarray:
    out = np.zeros(2)
    lib().orc_var_velocity(C.byref(vc), x, y, t, _dp(out))
    return out


def var_foot(vc: VarCfg, x: float, y: float, tau: float) -> np.ndarray:
    out = np.zeros(2)
    lib().orc_var_foot(C.byref(vc), x, y, tau, _dp(out))
    return out


def node_evolve_var(vc: VarCfg, patch, node_type: int, i: int, j: int, tau: float) -> float:
    patch = np.ascontiguousarray(patch, dtype=np.float64)
    return float(lib().orc_node_evolve_var(C.byref(vc), _dp(patch), node_type, i, j, tau))


def step_patch_var(vc: VarCfg, patch, freg=None) -> np.ndarray:
    patch = np.ascontiguousarray(patch, dtype=np.float64)
    out = np.empty_like(patch)
    lib().orc_step_patch_var(C.byref(vc), _dp(patch), _dp(out), None if freg is None else _dp(freg))
    return out


def run_uniform_var(vc: VarCfg, px: int, py: int, lo, nsteps: int, state: np.ndarray, nthreads: int = 0):
    """Advance a periodic px x py patch array nsteps steps from time vc.t
    (returns the new array; vc.t is advanced)."""
    st = np.ascontiguousarray(state, dtype=np.float64).copy()
    tmp = np.empty_like(st)
    nt = nthreads if nthreads > 0 else max_threads()
    lib().orc_run_uniform_var(C.byref(vc), px, py, float(lo[0]), float(lo[1]), nsteps, _dp(st), _dp(tmp), nt)
    return st
