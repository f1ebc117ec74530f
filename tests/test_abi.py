"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and rejects bad arguments on the host before touching the GPU."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def af():
    from paper_2205_07572_gb300 import af as _af, build
    build.build()
    return _af


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(af_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(af):
    L = af.lib()
    names = _declared()
    assert "af_patch_step" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_layout_sizes(af):
    for n in (8, 16, 32, 64):
        w = n + 5
        assert af.plane_stride(n) == (w * w + 7) // 8 * 8
        assert af.patch_words(n, 3) == 12 * af.plane_stride(n)


def test_work_builder_tiles(af):
    cfg = af.config(af.ACOUSTICS, af.F32, 32)
    nbr = np.zeros((3, 8), np.int32)
    w = np.frombuffer(af.build_step_work(cfg, [0, 1, 2], nbr=nbr).tobytes(), dtype=np.int16).reshape(-1, 32)
    assert len(w) == 3                       # interior patches: one 32^2 tile each
    assert (w[:, 20:24] == [0, 32, 0, 32]).all()
    nbr[1, 5] = -1                           # patch 1 misses its SE neighbour
    w = np.frombuffer(af.build_step_work(cfg, [0, 1, 2], nbr=nbr).tobytes(), dtype=np.int16).reshape(-1, 32)
    assert len(w) == 1 + 4 + 1               # extended patch: [-1, 33) in 2 x 2 tiles
    ext = w[1:5, 20:24]
    assert ext[:, 0].min() == -1 and ext[:, 1].max() == 33
    cfg64 = af.config(af.ADVECTION, af.F64, 64)
    w = af.build_step_work(cfg64, [0])
    assert len(w) // 64 == 9                 # [-1, 65) -> 3 x 3 tiles of 22


def test_work_builder_more_tiles_than_its_first_capacity_guess(af):
    """build_step_work guesses four work items per patch, then asks again
    with the count the library reports: 64-cell patches in 32 x 8 tiles take
    16 items each (27 when extended), all of them returned."""
    k = af.step_tilings().index((32, 8, 128, 0))
    cfg = af.config(af.ACOUSTICS, af.F32, 64)
    nbr = np.zeros((5, 8), np.int32)
    nbr[2, 0] = -1
    w = af.build_step_work(cfg, np.arange(5), nbr=nbr, tiling=k)
    items = np.frombuffer(w.tobytes(), dtype=np.int32).reshape(-1, 16)
    assert len(items) == 4 * 16 + 27
    assert np.array_equal(np.bincount(items[:, 0], minlength=5), [16, 16, 27, 16, 16])


def test_host_side_errors(af):
    cfg = af.config(af.ACOUSTICS, af.F64, 16, c=1.0)
    buf_a, buf_b, work = 1 << 20, 2 << 20, 3 << 20  # fake, aligned, never dereferenced
    dx = 1.0 / 16
    with pytest.raises(af.AFError) as e:
        af.patch_step(cfg, work, 1, buf_a, buf_b, 0.6 * dx, dx, dx, stream=0)
    assert e.value.status == 2               # AF_ERR_CFL (Eq. cfl-acoustics)
    with pytest.raises(af.AFError) as e:
        af.patch_step(cfg, work, 1, buf_a, buf_a, 0.4 * dx, dx, dx, stream=0)
    assert e.value.status == 1               # in == out
    with pytest.raises(af.AFError) as e:
        af.patch_step(cfg, work, 1, buf_a + 8, buf_b, 0.4 * dx, dx, dx, stream=0)
    assert e.value.status == 3               # misaligned state
    bad = af.config(af.ACOUSTICS, af.F64, 16, c=1.0)
    bad.ncomp = 1
    with pytest.raises(af.AFError):
        af.patch_step(bad, work, 1, buf_a, buf_b, 0.4 * dx, dx, dx, stream=0)
    adv = af.config(af.ADVECTION, af.F32, 16, a=1.0, b=0.5)
    with pytest.raises(af.AFError) as e:
        af.patch_step(adv, work, 1, buf_a, buf_b, 1.1 * dx, dx, dx, stream=0)
    assert e.value.status == 2               # Eq. cfl-adv
    af.patch_step(adv, work, 0, buf_a, buf_b, 0.5 * dx, dx, dx, stream=0)  # nothing to do: OK
    # the persistent (two-window) tiling is withdrawn: refused before any launch
    kp = [i for i, t in enumerate(af.step_tilings()) if t[3] == 1][0]
    with pytest.raises(af.AFError) as e:
        af.patch_step(adv, work, 1, buf_a, buf_b, 0.5 * dx, dx, dx, stream=0, tiling=kp)
    assert e.value.status == 6               # AF_ERR_UNIMPLEMENTED


def test_work_items_carry_patch_positions(af):
    cfg = af.config(af.ADVECTION, af.F64, 16)
    w = af.build_step_work(cfg, [0, 1, 2], levels=[1, 1, 2], ix=[3, 1, 7], iy=[0, 2, 5])
    items = np.frombuffer(w.tobytes(), dtype=np.int32).reshape(-1, 16)
    # af_work: patch, level, nbr[8], x0/x1, y0/y1 (int16 pairs), flags, ix, iy, pad
    assert items[:, 0].tolist() == [0, 1, 2]
    assert items[:, 13].tolist() == [3, 1, 7] and items[:, 14].tolist() == [0, 2, 5]
    plain = np.frombuffer(af.build_step_work(cfg, [0]).tobytes(), dtype=np.int32).reshape(-1, 16)
    assert plain[0, 13] == 0 and plain[0, 14] == 0


def test_variable_velocity_host_side_errors(af):
    """af_patch_step_var refuses on the host: a foot farther than one mesh
    width (AF_ERR_CFL, with the speed bounded over the domain and its ghost
    layers), aliased arrays, acoustics, unknown fields."""
    cfg = af.config(af.ADVECTION, af.F64, 16)
    buf_a, buf_b, work = 1 << 20, 2 << 20, 3 << 20   # fake, aligned, never dereferenced
    dx = 2.0 / 64
    solid = af.velocity(af.FIELD_SOLID_BODY, (-1, -1), (1, 1), 0.0)
    pair = af.state_pair(buf_a, buf_b, 0)
    with pytest.raises(af.AFError) as e:      # pi * (1 + 3 dx) * dt > dx
        af.patch_step_var(cfg, 0, work, 1, pair, solid, 0.32 * dx, dx, dx, stream=0)
    assert e.value.status == 2
    with pytest.raises(af.AFError) as e:
        af.patch_step_var(cfg, 0, work, 1, af.state_pair(buf_a, buf_a, 0), solid, 0.2 * dx, dx, dx, stream=0)
    assert e.value.status == 1
    swirl = af.velocity(af.FIELD_SWIRL, (0, 0), (1, 1), 0.3)
    with pytest.raises(af.AFError) as e:      # |v| <= 1
        af.patch_step_var(cfg, 0, work, 1, pair, swirl, 1.01 * dx, dx, dx, stream=0)
    assert e.value.status == 2
    bad = af.velocity(7, (0, 0), (1, 1), 0.0)
    with pytest.raises(af.AFError):
        af.patch_step_var(cfg, 0, work, 1, pair, bad, 0.2 * dx, dx, dx, stream=0)
    acu = af.config(af.ACOUSTICS, af.F64, 16, c=1.0)
    with pytest.raises(af.AFError):
        af.patch_step_var(acu, 0, work, 1, pair, swirl, 0.2 * dx, dx, dx, stream=0)
    af.patch_step_var(cfg, 0, work, 0, pair, swirl, 0.2 * dx, dx, dx, stream=0)   # nothing to do: OK


def test_owned_layout_host_side_errors(af):
    """af_pack_owned / af_unpack_owned refuse bad arguments on the host."""
    cfg = af.config(af.ACOUSTICS, af.F32, 32, c=1.0)
    state, owned = 1 << 20, 2 << 20                   # fake, aligned, never dereferenced
    af.pack_owned(cfg, 0, state, owned, stream=0)     # nothing to do: OK
    with pytest.raises(af.AFError) as e:
        af.pack_owned(cfg, 1, state, state, stream=0)
    assert e.value.status == 1                        # same array twice
    with pytest.raises(af.AFError) as e:
        af.unpack_owned(cfg, 1, None, state, stream=0)
    assert e.value.status == 1
    with pytest.raises(af.AFError) as e:
        af.pack_owned(cfg, 1, state + 8, owned, stream=0)
    assert e.value.status == 3                        # state not 32-byte aligned
    with pytest.raises(af.AFError) as e:
        af.unpack_owned(cfg, 1, owned + 2, state, stream=0)
    assert e.value.status == 3                        # owned not aligned to float
    bad = af.config(af.ACOUSTICS, af.F32, 32, c=1.0)
    bad.ncomp = 1
    with pytest.raises(af.AFError):
        af.pack_owned(bad, 1, state, owned, stream=0)
    assert af.owned_words(32, 3) == 12 * 32 * 32


def test_probe_and_counter_host_side_errors(af):
    """af_fma_throughput and af_step_wait_timeouts refuse bad arguments on
    the host, before any device call."""
    import ctypes
    L = af.lib()
    sink = 1 << 20                                     # fake, aligned, never dereferenced
    assert L.af_fma_throughput(7, 1, 1, ctypes.c_void_p(sink), None) == 1       # unknown precision
    assert L.af_fma_throughput(af.F32, 0, 1, ctypes.c_void_p(sink), None) == 1  # no blocks
    assert L.af_fma_throughput(af.F32, 1, 0, ctypes.c_void_p(sink), None) == 1  # no iterations
    assert L.af_fma_throughput(af.F32, 1, 1, None, None) == 1                   # no sink
    assert L.af_fma_throughput(af.F64, 1, 1, ctypes.c_void_p(sink + 4), None) == 3  # misaligned FP64 sink
    assert L.af_step_wait_timeouts(None, 0) == 1
    assert L.af_fma_probe_threads() == 256 * 8


def test_mass_noalloc_host_side_errors_and_capacity(af):
    """af_mass_noalloc refuses, on the host, what af_mass refuses: a missing
    state or result, a misaligned state (AF_ERR_LAYOUT, as af_mass's
    check), a misaligned result.  Its fixed array holds 1024 partial sums
    (af.h): af_mass needs at most 256 per component for any leaf count, so
    three components always fit."""
    import ctypes
    cfg = af.config(af.ACOUSTICS, af.F64, 16, c=1.0)
    fake = 1 << 20                                     # fake, aligned, never dereferenced
    F = af.forest_struct(300, 1, 5, fake, fake, fake, fake)
    L = af.lib()

    def call(state, out):
        return L.af_mass_noalloc(ctypes.byref(cfg), ctypes.byref(F), ctypes.c_void_p(state), 1 / 16, 1 / 16,
                                 ctypes.c_void_p(out), None)

    assert call(0, fake) == 1                          # no state
    assert call(fake, 0) == 1                          # no result
    assert call(fake + 8, fake) == 3                   # state not 32-byte aligned
    assert call(fake, fake + 4) == 3                   # result not 8-byte aligned
    for nleaf in (1, 255, 256, 300, 1 << 20, (1 << 31) - 1):
        assert af.mass_scratch_bytes(nleaf, 3) <= 1024 * 8
    assert af.mass_scratch_bytes(1 << 20, 3) == 256 * 3 * 8
