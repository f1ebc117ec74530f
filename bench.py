#!/usr/bin/env python3
"""Benchmark of the Active Flux patch step on GB300.

Workload (one bench step = one Active Flux time step of the whole grid, i.e.
one af_patch_step launch over every patch):
  2-D acoustics (p, u, v), c = 1, periodic unit square, Gaussian pressure pulse
  (sigma 0.05) at the centre plus the stationary vortex, CFL 0.4, patches of
  32 x 32 cells with 2 ghost layers.  The grid is 4096 x 4096 cells
  (128 x 128 patches): the same patch shape as the 512 x 512 / 16 x 16-patch
  configuration, scaled so the state (1.1 GB FP32, 2.2 GB FP64 per copy) is
  larger than the 129 MB L2 and every step streams from HBM.

Metric: interior cell updates per second (all three components).  Reported
for the FP32 patch stencil (`value`) and the FP64 stencil (`fp64`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only other implementation of
the method here) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS = 32
P_SIDE = 128
CFL = 0.4
BYTES_PER_CELL = {"f32": 3 * 8 * 4, "f64": 3 * 8 * 8}   # 3 comps x (4 read + 4 written) words
WORKLOAD = ("acoustics c=1, periodic unit square, 4096x4096 cells as 128x128 patches of 32x32 "
            "(2 ghost layers), Gaussian pulse sigma 0.05 + stationary vortex, CFL 0.4")
METRIC = "cell updates/sec (Active Flux patch step, acoustics, 32x32 patches)"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# --------------------------------------------------------------------- peaks
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = None
    src = "fallback"
    if os.path.exists(path):
        try:
            d = json.load(open(path))

            def find(o, key):
                if isinstance(o, dict):
                    for k, v in o.items():
                        if k == key and isinstance(v, (int, float)):
                            return float(v)
                        r = find(v, key)
                        if r is not None:
                            return r
                return None
            hbm = find(d, "hbm_gbs")
            if hbm is not None:
                src = "measured"
        except Exception:
            hbm = None
    if hbm is None:
        hbm = 6800.0
    return hbm, src


# ------------------------------------------------------------------- traffic
PROFILE = os.path.join(ROOT, "profiles", "step_kernel_f32_acoustics_4096x4096.md")
KERNEL_SOURCES = ["paper_2205_07572_gb300/csrc/af_step_kernels.cuh", "paper_2205_07572_gb300/csrc/af_internal.h",
                  "paper_2205_07572_gb300/csrc/af_step_f32_n32.cu"]


def kernel_source_hash() -> str:
    """First 16 hex digits of the SHA-256 of the step kernel's sources."""
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(tiling: dict, path: str = PROFILE):
    """DRAM bytes (read + write) per launch of the timed tiling, from the
    committed ncu summary's `traffic:` record, or None when the summary
    covers another tiling or the kernel's sources changed since the capture
    (their hash differs).  Returns (bytes or None, description)."""
    import re
    try:
        txt = open(path).read()
    except OSError:
        return None, "no ncu summary"
    m = re.search(r"traffic: tiling=(\d+)x(\d+)x(\d+) bytes_per_launch=(\d+) source_hash=([0-9a-f]+)", txt)
    if not m:
        return None, "no traffic record in the ncu summary"
    tmx, tmy, nt, nbytes, hsh = int(m[1]), int(m[2]), int(m[3]), int(m[4]), m[5]
    rel = os.path.relpath(path, ROOT)
    if (tuple(tiling["tile"]) != (tmx, tmy) or tiling["threads"] != nt or tiling["persistent"]):
        return None, f"{rel} covers the {tmx}x{tmy}/{nt} tiling, not the timed one"
    if hsh != kernel_source_hash():
        return None, f"stale: the kernel sources changed since the capture in {rel}"
    return float(nbytes), f"ncu dram__bytes_read.sum + dram__bytes_write.sum, {rel}"


# -------------------------------------------------------------------- clocks
def smi_device(dev: int) -> str:
    """nvidia-smi's selector (-i) for CUDA device `dev` of this process.
    CUDA numbers the devices it can see, so under CUDA_VISIBLE_DEVICES its
    index is not nvidia-smi's: select by the device's UUID, else by the
    CUDA_VISIBLE_DEVICES entry the index maps to."""
    try:
        import torch
        u = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    except Exception:
        u = None
    if u is not None and str(u):
        s = str(u)
        return s if s.startswith(("GPU-", "MIG-")) else "GPU-" + s
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ent = [e.strip() for e in vis.split(",") if e.strip()]
        if 0 <= dev < len(ent):
            return ent[dev]
    return str(dev)


class ClockSampler:
    def __init__(self, gpu: str):
        """gpu: nvidia-smi's selector of the timed device (smi_device)."""
        self.f = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- setup
def initial_state(prec: str):
    import synth as S
    grid = S.UniformGrid(S.Layout(N_CELLS, 3), P_SIDE, P_SIDE)
    st = S.periodic_state(grid, S.pulse_plus_vortex(), nq=2,
                          dtype=np.float32 if prec == "f32" else np.float64)
    return grid, st


def _busy(run, seconds: float):
    """Untimed steps for about `seconds` (keeps the GPU under the bench load
    while the clocks are sampled)."""
    import torch
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        for _ in range(8):
            run.step()
        torch.cuda.synchronize()


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time per step (replicas: every rank advances its own
    copy of the workload, so the job takes as long as its slowest rank)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput of `world` replicas over the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


def run_ours(prec: str, steps: int, warmup: int, rank: int, world: int, dist):
    import torch
    from paper_2205_07572_gb300 import af
    from paper_2205_07572_gb300.uniform import UniformRun
    grid, st = initial_state(prec)
    dt = CFL * grid.dx
    cfg = af.config(af.ACOUSTICS, af.F32 if prec == "f32" else af.F64, N_CELLS, c=1.0)
    run = UniformRun(cfg, P_SIDE, P_SIDE, grid.dx, grid.dy, dt, state=st)
    # autotune the tile shape on this workload (outside the timed region)
    from paper_2205_07572_gb300 import tune
    best, table = tune.tune(run, steps=3 if prec == "f64" else 10, warmup=1)
    stream = torch.cuda.current_stream()
    # The timed region is far shorter than nvidia-smi's sampling interval, so
    # the clocks are sampled over a window of the same step loop around it
    # (about 0.3 s of untimed steps before the warm-up and after the timed steps).
    smi_sel = smi_device(torch.cuda.current_device())
    clocks = ClockSampler(smi_sel)
    _busy(run, 0.3)
    for _ in range(warmup):
        run.step()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev0, ev1 = marks[0], marks[-1]
    ev0.record(stream)
    for k in range(steps):
        run.step()
        marks[k + 1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    each = sorted(marks[k].elapsed_time(marks[k + 1]) for k in range(steps))
    _busy(run, 0.3)
    ck = clocks.stop()
    ck["window"] = "same step loop, ~0.3 s before the warm-up to ~0.3 s after the timed steps"
    ck["device"] = smi_sel
    ms = max_over_ranks(ev0.elapsed_time(ev1) / steps, dist, "cuda")
    cells = grid.npatch * N_CELLS * N_CELLS
    # sanity: the state stays finite
    assert torch.isfinite(run.state).all().item()
    tilings = af.step_tilings()
    return {"ms": ms, "cells": cells, "clocks": ck, "nwork": run.nwork, "run": run,
            "ms_median": each[len(each) // 2], "ms_best": each[0],
            "tiling": {"index": best, "tile": tilings[best][:2], "threads": tilings[best][2],
                       "persistent": bool(tilings[best][3]),
                       "tuned_ms": {str(tilings[k]): round(v, 4) for k, v in table.items()}}}


def run_e2e(prec: str, steps: int, warmup: int, tiling=None, bands: int = 32, layout: str = "owned"):
    """Same step through the public API with the state kept in pinned HOST
    memory: every step copies it host->device, runs af_patch_step, and copies
    the result back (host<->device copies inside the timed region), in bands
    of patch rows so that the copies in, the step and the copies out overlap.
    layout "owned": the host holds only the patches' own degrees of freedom
    ([patch][comp][plane][n][n], UniformRun.step_host_owned: unpacked into and
    packed out of the device state by af_unpack_owned / af_pack_owned);
    "lattice": the host holds the device layout, ghost rings and padding
    included (UniformRun.step_host)."""
    import torch
    import synth as S
    from paper_2205_07572_gb300 import af
    grid, st = initial_state(prec)
    dt = CFL * grid.dx
    cfg = af.config(af.ACOUSTICS, af.F32 if prec == "f32" else af.F64, N_CELLS, c=1.0)
    from paper_2205_07572_gb300.uniform import UniformRun
    run = UniformRun(cfg, P_SIDE, P_SIDE, grid.dx, grid.dy, dt, state=None, tiling=tiling)
    lat = st.reshape(run.a.shape)
    if layout == "owned":
        g, n = S.G, N_CELLS
        own = S.Layout(n, 3).lattice(lat.reshape(grid.npatch, 3, 4, -1))[..., g:g + n, g:g + n]
        host = torch.from_numpy(np.ascontiguousarray(own).reshape(grid.npatch, -1)).pin_memory()
        step = run.step_host_owned
    else:
        host = torch.from_numpy(lat).pin_memory()
        step = run.step_host
    stream = torch.cuda.current_stream()

    def one():
        step(host, bands)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        one()
    ev1.record(stream)
    torch.cuda.synchronize()
    assert torch.isfinite(host).all().item()
    ms = ev0.elapsed_time(ev1) / steps
    nbytes = host.numel() * host.element_size()
    cells = grid.npatch * N_CELLS * N_CELLS
    return {"value": cells / (ms * 1e-3), "unit": "cell updates/s", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "ms_per_step": ms, "bands": bands, "host_layout": layout,
            "link_gbs": 2 * nbytes / (ms * 1e-3) / 1e9}


def link_peak(nbytes: int, reps: int = 5):
    """Host-link copy rates for a state of `nbytes` in pinned host memory:
    host->device alone, device->host alone, and both at once on two streams
    (the pattern of the end-to-end step).  Best of `reps`, GB/s."""
    import torch
    h_in = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    h_out = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d_a = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d_b = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s_up, s_dn = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(up: bool, dn: bool) -> float:
        best = float("inf")
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if up:
                with torch.cuda.stream(s_up):
                    d_a.copy_(h_in, non_blocking=True)
            if dn:
                with torch.cuda.stream(s_dn):
                    h_out.copy_(d_b, non_blocking=True)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        return (int(up) + int(dn)) * nbytes / best / 1e9

    out = {"h2d_gbs": timed(True, False), "d2h_gbs": timed(False, True), "both_gbs": timed(True, True),
           "bytes_each_way": nbytes, "how": "pinned host <-> device copies (torch copy_), best of %d" % reps}
    del h_in, h_out, d_a, d_b
    return out


def literal_config2(prec: str, steps: int):
    """The 512 x 512-cell (16 x 16 patches of 32^2) configuration itself: its
    17-34 MB state is L2-resident, so this is reported beside the HBM-scaled
    workload, not as the headline.  The rate is the whole T = 0.5 run (640
    steps) replayed from a CUDA graph, on the tiling tuned for this grid; the
    per-call eager rate is given beside it."""
    import torch
    import synth as S
    from paper_2205_07572_gb300 import af
    from paper_2205_07572_gb300.uniform import UniformRun
    from paper_2205_07572_gb300 import tune
    grid = S.UniformGrid(S.Layout(N_CELLS, 3), 16, 16)
    st = np.nan_to_num(grid.state(S.pulse_plus_vortex(), nq=3))
    dt = CFL * grid.dx
    cfg = af.config(af.ACOUSTICS, af.F32 if prec == "f32" else af.F64, N_CELLS, c=1.0)
    run = UniformRun(cfg, 16, 16, grid.dx, grid.dy, dt, state=st)
    # this grid is about one wave of CTAs: its own tiling, and the whole
    # T = 0.5 run (640 steps) replayed from a CUDA graph of two steps
    best, tried = tune.tune(run, steps=20, warmup=3)
    for _ in range(5):
        run.step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        run.step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    run.advance(4)  # capture (after an eager pair) and one replay
    torch.cuda.synchronize()
    nrun = 640
    ev0.record(stream)
    run.advance(nrun)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_run = ev0.elapsed_time(ev1)
    cells = grid.npatch * N_CELLS * N_CELLS
    return {"value": cells * nrun / (ms_run * 1e-3), "ms_per_step": ms_run / nrun, "steps_T0.5": nrun,
            "run_ms_T0.5": ms_run, "graphs": True, "tiling": af.step_tilings()[best],
            "tuned_ms": {str(af.step_tilings()[k]): round(v, 4) for k, v in tried.items()},
            "eager": {"value": cells / (ms * 1e-3), "ms_per_step": ms}}


# ------------------------------------------------------- adaptive workloads
# Quadtree AMR with 16 x 16-cell patches and subcycling.  One AMR bench step
# is one coarse step: every level advanced to the next time of the coarsest
# level (level l takes 2^(l - lmin) steps), with the conservative fix and the
# ghost exchange at every synchronised time.
AMR_CASES = {
    "advection_levels2-6": dict(
        eq=0, B=1, lmin=2, lmax=6, lo=(0.0, 0.0), hi=(1.0, 1.0), a=1.0, b=1.0, per_patch=True,
        desc=("advection a=(1,1), periodic unit square, wave packet exp(-r^2/0.01) cos(60 pi x), levels 2-6, "
              "16x16-cell patches, gradient tagging (refine >= 4, coarsen < 1), CFL 0.4"),
        tag=(0, 1, 4.0, 1.0)),
    "acoustics_levels3-7": dict(
        eq=1, B=3, lmin=3, lmax=7, lo=(-1.5, -1.5), hi=(1.5, 1.5), a=0.0, b=0.0, per_patch=True,
        desc=("acoustics c=1, periodic [-1.5,1.5]^2 (3x3 brick), ring wave exp(-(r-0.25)^2/0.001) cos(80 pi r), "
              "u=v=0, levels 3-7, 16x16-cell patches, gradient tagging on p (refine >= 4, coarsen < 1), CFL 0.4"),
        tag=(0, 1, 4.0, 1.0)),
    # the configurations' stated patch counts: the same data repeated in every
    # unit tree of a brick (one packet per tree of a 2x2 brick: 1k-5k leaves;
    # one ring per tree of the 3x3 brick: tens of thousands of leaves)
    "advection_levels2-6_2x2_packets": dict(
        eq=0, B=2, lmin=2, lmax=6, lo=(0.0, 0.0), hi=(2.0, 2.0), a=1.0, b=1.0, per_patch=False,
        per_tree=(0.0, 0.0),
        desc=("advection a=(1,1), periodic [0,2]^2 (2x2 brick), the wave packet exp(-r^2/0.01) cos(60 pi x) in "
              "each unit tree, levels 2-6, 16x16-cell patches, gradient tagging (refine >= 4, coarsen < 1), "
              "CFL 0.4"),
        tag=(0, 1, 4.0, 1.0)),
    "acoustics_levels3-7_3x3_rings": dict(
        eq=1, B=3, lmin=3, lmax=7, lo=(-1.5, -1.5), hi=(1.5, 1.5), a=0.0, b=0.0, per_patch=False,
        per_tree=(-0.5, -0.5),
        desc=("acoustics c=1, periodic [-1.5,1.5]^2 (3x3 brick), the ring wave exp(-(r-0.25)^2/0.001) "
              "cos(80 pi r) centred in each unit tree, u=v=0, levels 3-7, 16x16-cell patches, gradient tagging "
              "on p (refine >= 4, coarsen < 1), CFL 0.4"),
        tag=(0, 1, 4.0, 1.0)),
}
AMR_N = 16


def _amr_funcs(case):
    import synth as S
    c = AMR_CASES[case]
    f = S.wave_packet if c["eq"] == 0 else S.ring_wave
    if "per_tree" in c:
        f = S.per_unit_tree(f, c["per_tree"])
    if c["eq"] == 0:
        return [f]
    zero = lambda x, y: 0.0 * x
    return [f, zero, zero]


def amr_initial(case: str, device="cuda"):
    """Initial forest by the method's own adaptation: start from the uniform
    coarsest level, then tag (af_tag) and regrid (af_forest_regrid) the exact
    initial data once per level."""
    import synth as S
    from paper_2205_07572_gb300 import af
    from paper_2205_07572_gb300.amr import AMRRun, Forest, regrid_leaves
    c = AMR_CASES[case]
    B, lmin, lmax = c["B"], c["lmin"], c["lmax"]
    side = B << lmin
    leaves = [(lmin, x, y) for y in range(side) for x in range(side)]
    cfg = af.config(c["eq"], af.F64, AMR_N, c["a"], c["b"], 1.0)
    funcs = _amr_funcs(case)
    for _ in range(lmax - lmin):
        lv = np.array(leaves, dtype=np.int64).reshape(-1, 3)
        st = S.forest_state_fast(AMR_N, cfg.ncomp, B, lv[:, 0], lv[:, 1], lv[:, 2], funcs, c["lo"], c["hi"])
        run = AMRRun(cfg, B, lmax, leaves, st, c["lo"], c["hi"], 1e-9, device=device)
        comp, kind, rt, ct = c["tag"]
        tags, _ = run.tags(comp, kind, rt, ct)
        new = regrid_leaves(run.forest, np.maximum(tags, 0), lmin)
        if new == run.forest.leaves:
            break
        leaves = new
    lv = np.array(leaves, dtype=np.int64).reshape(-1, 3)
    st = S.forest_state_fast(AMR_N, cfg.ncomp, B, lv[:, 0], lv[:, 1], lv[:, 2], funcs, c["lo"], c["hi"])
    return leaves, st


def amr_time(case: str, leaves, st, prec: str, mode: str, graphs: bool, coarse_steps: int, warmup: int,
             regrid: bool = False, tiling=None, ext_tiling=None):
    """Cell updates per second of coarse steps of an adaptive run (the
    forest fixed, or regridded before every coarse step)."""
    import torch
    from paper_2205_07572_gb300 import af
    from paper_2205_07572_gb300.amr import AMRRun
    c = AMR_CASES[case]
    cfg = af.config(c["eq"], af.F32 if prec == "f32" else af.F64, AMR_N, c["a"], c["b"], 1.0)
    dx0 = (c["hi"][0] - c["lo"][0]) / (c["B"] * AMR_N)
    speed = max(abs(c["a"]), abs(c["b"])) if c["eq"] == 0 else 1.0
    dt0 = CFL * dx0 / speed
    run = AMRRun(cfg, c["B"], c["lmax"], leaves, st, c["lo"], c["hi"], dt0, mode=mode, graphs=graphs,
                 tiling=tiling, ext_tiling=ext_tiling)
    comp, kind, rt, ct = c["tag"]

    def one():
        if regrid:
            tags, _ = run.tags(comp, kind, rt, ct)
            run.regrid(tags, c["lmin"])
        cu = run.cell_updates_per_coarse_step()
        nl = run.launches_per_coarse_step()
        run.coarse_step()
        return cu, nl

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cu = nl = 0
    ev0.record(stream)
    for _ in range(coarse_steps):
        a, b = one()
        cu += a
        nl += b
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    levels = np.bincount(run.forest.level, minlength=c["lmax"] + 1).tolist()
    return {"value": cu / (ms * 1e-3), "tiling": run.tiling, "unit": "cell updates/s", "ms_per_coarse_step": ms / coarse_steps,
            "coarse_steps": coarse_steps, "cell_updates": cu, "gpu_launches": nl, "leaves": run.forest.nleaf,
            "leaves_per_level": levels}, run


def amr_l1_exact(case: str, run, t: float):
    """Sum over leaves and interior cells of |Q - Q_exact| dx_l dy_l (advection:
    the initial data translated by (a, b) t)."""
    import synth as S
    c = AMR_CASES[case]
    f = S.translated(_amr_funcs(case)[0], c["a"], c["b"], t, c["lo"], c["hi"])
    F = run.forest
    ex = S.forest_state_fast(AMR_N, 1, c["B"], F.level, F.ix, F.iy, [f], c["lo"], c["hi"], nq=4)
    lay = S.Layout(AMR_N, 1)
    got = run.current().double().cpu().numpy().reshape(F.nleaf, 1, 4, -1)
    g = lay.lattice(got)[:, 0, 0, S.G:S.G + AMR_N, S.G:S.G + AMR_N]
    e = lay.lattice(ex)[:, 0, 0, S.G:S.G + AMR_N, S.G:S.G + AMR_N]
    area = ((c["hi"][0] - c["lo"][0]) / ((c["B"] << F.level) * AMR_N)) ** 2
    return float((np.abs(g - e).sum(axis=(1, 2)) * area).sum())


def amr_l1_between(case: str, ra, rb):
    """L1 distance of the first component's averages of two runs on the same forest."""
    import synth as S
    c = AMR_CASES[case]
    F = ra.forest
    assert F.leaves == rb.forest.leaves
    lay = S.Layout(AMR_N, ra.cfg.ncomp)
    ga = lay.lattice(ra.current().double().cpu().numpy().reshape(F.nleaf, ra.cfg.ncomp, 4, -1))
    gb = lay.lattice(rb.current().double().cpu().numpy().reshape(F.nleaf, rb.cfg.ncomp, 4, -1))
    sl = (slice(None), 0, 0, slice(S.G, S.G + AMR_N), slice(S.G, S.G + AMR_N))
    area = ((c["hi"][0] - c["lo"][0]) / ((c["B"] << F.level) * AMR_N)) ** 2
    return float((np.abs(ga[sl] - gb[sl]).sum(axis=(1, 2)) * area).sum())


def amr_tune(case: str, leaves, st, prec: str):
    """Fastest compiled tiling for one coarse step of the fixed forest, then
    the fastest second tiling for the leaves that advance their ghost layer
    (AMRRun ext_tiling; None: the same tiling).  Returns (tiling, ext_tiling,
    times in ms keyed "k" or "k+e")."""
    from paper_2205_07572_gb300 import tune
    cands = tune.default_candidates()
    times = {}
    for k in cands:
        r, _ = amr_time(case, leaves, st, prec, "batched", False, 2, 1, tiling=k)
        times[(k, None)] = r["ms_per_coarse_step"]
    best = min(times, key=times.get)[0]
    for e in cands:
        if e != best:
            r, _ = amr_time(case, leaves, st, prec, "batched", False, 2, 1, tiling=best, ext_tiling=e)
            times[(best, e)] = r["ms_per_coarse_step"]
    k, e = min(times, key=times.get)
    return k, e, {(str(a) if b is None else f"{a}+{b}"): round(v, 4) for (a, b), v in times.items()}


def amr_bench(case: str, coarse_steps: int, warmup: int, per_patch: bool = True):
    """Batched FP32 (graph-replayed) vs batched FP64 vs per-level and
    per-patch FP64 launches on one adaptive workload."""
    t0 = time.perf_counter()
    leaves, st = amr_initial(case)
    out = {"workload": AMR_CASES[case]["desc"], "setup_s": None}
    out["setup_s"] = round(time.perf_counter() - t0, 1)
    c = AMR_CASES[case]
    k32, e32, out["tuned_ms_f32"] = amr_tune(case, leaves, st, "f32")
    k64, e64, out["tuned_ms_f64"] = amr_tune(case, leaves, st, "f64")
    # graphs: the first coarse step from each level parity runs eagerly, the
    # second is captured, so four warm-up steps leave only replays timed
    r32, run32 = amr_time(case, leaves, st, "f32", "batched", True, coarse_steps, max(4, warmup), tiling=k32,
                          ext_tiling=e32)
    r64, run64 = amr_time(case, leaves, st, "f64", "batched", False, coarse_steps, max(4, warmup), tiling=k64,
                          ext_tiling=e64)
    r32["ext_tiling"], r64["ext_tiling"] = e32, e64
    out["batched_graphs_f32"] = r32
    out["batched_f64"] = r64
    out["l1_f32_vs_f64"] = amr_l1_between(case, run32, run64)
    if c["eq"] == 0:
        out["l1_vs_exact"] = {"f32": amr_l1_exact(case, run32, run32.time),
                              "f64": amr_l1_exact(case, run64, run64.time), "t": run32.time}
    del run32, run64
    out["per_level_f64"], _ = amr_time(case, leaves, st, "f64", "per_level", False, max(1, coarse_steps // 2), 1)
    if per_patch:
        out["per_patch_f64"], _ = amr_time(case, leaves, st, "f64", "per_patch", False, 1, 1)
    # the method as the paper runs it: regrid before every coarse step
    nrg = max(2, coarse_steps // 2)
    rg32, g32 = amr_time(case, leaves, st, "f32", "batched", False, nrg, 1, regrid=True, tiling=k32,
                         ext_tiling=e32)
    rg64, g64 = amr_time(case, leaves, st, "f64", "batched", False, nrg, 1, regrid=True, tiling=k64,
                         ext_tiling=e64)
    out["regrid_every_coarse_step_f32"], out["regrid_every_coarse_step_f64"] = rg32, rg64
    if c["eq"] == 0:
        out["regrid_l1_vs_exact"] = {"f32": amr_l1_exact(case, g32, g32.time),
                                     "f64": amr_l1_exact(case, g64, g64.time), "t": g32.time}
    out["regrid_same_forest_f32_f64"] = g32.forest.leaves == g64.forest.leaves
    if out["regrid_same_forest_f32_f64"]:
        out["regrid_l1_f32_vs_f64"] = amr_l1_between(case, g32, g64)
    del g32, g64
    out["leaves"] = len(leaves)
    # precision and batching at equal L1 first: batched FP32 against batched
    # FP64, then against the per-level and per-patch launches
    out["speedup_batched_f32_vs_batched_f64"] = r32["value"] / r64["value"]
    out["speedup_batched_f32_vs_per_level_f64"] = r32["value"] / out["per_level_f64"]["value"]
    if per_patch:
        out["speedup_batched_f32_vs_per_patch_f64"] = r32["value"] / out["per_patch_f64"]["value"]
    return out


def amr_profile_run(steps: int, warmup: int, case: str = "acoustics_levels3-7", tile=(16, 16, 128)):
    """Batched FP32 coarse steps (no graph capture, so every kernel is its own
    launch) of one adaptive workload on its initial forest, with the compiled
    tiling `tile` (cells x, cells y, threads)."""
    import torch
    from paper_2205_07572_gb300 import af
    from paper_2205_07572_gb300.amr import AMRRun
    c = AMR_CASES[case]
    leaves, st = amr_initial(case)
    cfg = af.config(c["eq"], af.F32, AMR_N, c["a"], c["b"], 1.0)
    dx0 = (c["hi"][0] - c["lo"][0]) / (c["B"] * AMR_N)
    run = AMRRun(cfg, c["B"], c["lmax"], leaves, st, c["lo"], c["hi"], CFL * dx0, tiling=_tiling_index(*tile))
    for _ in range(warmup):
        run.coarse_step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        run.coarse_step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    cu = run.cell_updates_per_coarse_step()
    return {"workload": c["desc"], "leaves": run.forest.nleaf, "ms_per_coarse_step": ms,
            "value": cu / (ms * 1e-3), "unit": "cell updates/s", "launches_per_coarse_step":
            run.launches_per_coarse_step(), "graphs": False}


# ----------------------------------------------------------- learned tagging
def adapt_initial(cfg, B, lmin, lmax, lo, hi, funcs, tag):
    """Initial forest by the method's own adaptation (tag and regrid the exact
    initial data once per level), and its state."""
    import synth as S
    from paper_2205_07572_gb300.amr import AMRRun, regrid_leaves
    side = B << lmin
    leaves = [(lmin, x, y) for y in range(side) for x in range(side)]
    for _ in range(lmax - lmin):
        lv = np.array(leaves, dtype=np.int64).reshape(-1, 3)
        st = S.forest_state_fast(cfg.n, cfg.ncomp, B, lv[:, 0], lv[:, 1], lv[:, 2], funcs, lo, hi)
        run = AMRRun(cfg, B, lmax, leaves, st, lo, hi, 1e-9)
        t, _ = run.tags(*tag)
        new = regrid_leaves(run.forest, np.maximum(t, 0), lmin)
        if new == run.forest.leaves:
            break
        leaves = new
    lv = np.array(leaves, dtype=np.int64).reshape(-1, 3)
    return leaves, S.forest_state_fast(cfg.n, cfg.ncomp, B, lv[:, 0], lv[:, 1], lv[:, 2], funcs, lo, hi)


def _tiling_index(tmx, tmy, threads):
    from paper_2205_07572_gb300 import af
    return [t[:3] for t in af.step_tilings()].index((tmx, tmy, threads))


def pareto_front(points):
    """Points (l1, rate) not beaten by another with lower (or equal) L1 and
    higher rate, by increasing L1."""
    front = []
    for l1, rate in sorted(points):
        if not front or rate > front[-1][1]:
            front.append((l1, rate))
    return front


def rate_at(front, l1):
    """Throughput of a Pareto front at L1 error `l1`, interpolated linearly
    in log L1 and log rate between its neighbours; None outside its range.
    A front that reaches lower L1 at an equal or higher rate counts as that
    rate at every larger L1 (it could be run as is)."""
    if not front or l1 < front[0][0] * (1 - 1e-12):
        return None
    best = None
    for k, (a, ra) in enumerate(front):
        if a <= l1:
            best = ra if best is None else max(best, ra)
        if k + 1 < len(front):
            (b, rb) = front[k + 1]
            if a <= l1 <= b:
                t = (math.log(l1) - math.log(a)) / (math.log(b) - math.log(a)) if b > a else 0.0
                v = math.exp(math.log(ra) + t * (math.log(rb) - math.log(ra)))
                best = v if best is None else max(best, v)
    return best


def learned_tagging(B=3, lmin=3, lmax=7, train_radii=(0.2, 0.3), test_radius=0.25, train_steps=256,
                    t_end=None, test_steps=128, intervals=(2, 4, 8), plain_intervals=(1, 2, 4),
                    thresholds=(3.0, 4.0, 6.0), epochs=4, batch=4096, cmin=0.5, seed=0, fp64=True,
                    per_patch=True):
    """Acoustics ring wave on the 3 x 3 brick [-1.5, 1.5]^2, levels 3-7 (the
    configuration-4 forest), 16 x 16-cell patches, FP32 stencil.  For each
    regrid interval R in `intervals` a tagger is trained on runs of the method
    (plain criterion, regrid every R coarse steps) started from rings of other
    radii, to predict whether the plain criterion tags a leaf at any of the
    next R coarse steps.  On the test ring, runs to the same end time are
    compared by the L1 distance of p to a uniform run at the finest level and
    by cell updates per second (regrids and tagging included):
      plain criterion, regrid every {plain_intervals} steps, refine threshold
      in {thresholds} (coarsen below a quarter of it);
      learned tags (plain fallback below confidence cmin), regrid every R.
    The two Pareto fronts (L1, throughput) are compared at equal L1
    (interpolated).  Batched FP64 and per-patch FP64 runs of the plain
    criterion (every step, threshold 4) give the precision baselines; the
    per-patch run is timed on a few coarse steps (its arithmetic, and so its
    L1, is the batched FP64 run's)."""
    import torch
    import synth as S
    from paper_2205_07572_gb300 import af
    from paper_2205_07572_gb300.amr import AMRRun
    from paper_2205_07572_gb300.tagger import Tagger, collect, prepare, uniform_global, l1_vs_uniform
    lo, hi = (-1.5, -1.5), (1.5, 1.5)
    n = AMR_N
    cfg = af.config(af.ACOUSTICS, af.F32, n, c=1.0)
    cfg64 = af.config(af.ACOUSTICS, af.F64, n, c=1.0)
    dx0 = (hi[0] - lo[0]) / (B * n)
    dt0 = CFL * dx0
    comp, kind = 0, 1
    zero = lambda x, y: 0.0 * x
    out = {"workload": (f"acoustics ring waves exp(-(r-r0)^2/0.001) cos(80 pi r) on the {B}x{B} brick "
                        f"[-1.5,1.5]^2, levels {lmin}-{lmax}, 16x16 patches, FP32; train r0 {list(train_radii)}, "
                        f"test r0 {test_radius}; gradient criterion (refine >= thr, coarsen < thr/4)"),
           "levels": [lmin, lmax]}
    tagq = lambda thr: (comp, kind, thr, thr / 4.0)
    t16 = _tiling_index(16, 16, 128)  # the tiling the autotuner picks for these forests
    # ---- one tagger per regrid interval
    taggers, out["training"] = {}, {}
    for R in intervals:
        t0 = time.perf_counter()
        parts = []
        for r0 in train_radii:
            leaves, st = adapt_initial(cfg, B, lmin, lmax, lo, hi, [S.ring_wave_at(r0), zero, zero], tagq(4.0))
            run = AMRRun(cfg, B, lmax, leaves, st, lo, hi, dt0, tiling=t16)
            parts.append(collect(run, train_steps, tagq(4.0), lmin, 4.0, horizon=R))
            del run
        data = {k: torch.cat([p[k] for p in parts]) for k in parts[0]}
        torch.cuda.synchronize()
        collect_s = time.perf_counter() - t0
        data = prepare(data, batch, seed=seed)
        tg = Tagger(3, n, seed=seed)
        ev0 = tg.evaluate(data)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        tg.fit(data, epochs=epochs, batch=batch)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t1
        taggers[R] = tg
        out["training"][str(R)] = {"samples": int(data["level"].numel()),
                                   "positive_fraction": data["positives"] / int(data["level"].numel()),
                                   "collect_s": round(collect_s, 2), "train_s": round(train_s, 3),
                                   "train_samples_per_s": epochs * (int(data["level"].numel()) // batch) * batch
                                   / train_s, "before": ev0, "after": tg.evaluate(data)}
        del data, parts
    funcs = [S.ring_wave_at(test_radius), zero, zero]
    leaves, st = adapt_initial(cfg, B, lmin, lmax, lo, hi, funcs, tagq(4.0))
    out["initial_leaves"] = len(leaves)
    T = t_end if t_end is not None else test_steps * dt0 / (1 << lmin)
    # how well each tagger predicts the plain criterion on the test ring
    out["test_eval"] = {}
    for R, tg in taggers.items():
        run = AMRRun(cfg, B, lmax, leaves, st, lo, hi, dt0, tiling=t16)
        test = prepare(collect(run, min(test_steps, 64), tagq(4.0), lmin, 4.0, horizon=R), batch, seed=seed + 1)
        out["test_eval"][str(R)] = tg.evaluate(test)
        del run, test

    def tagged_run(c, tagger, every, thr, mode="batched"):
        run = AMRRun(c, B, lmax, leaves, st, lo, hi, dt0, mode=mode, tiling=t16)
        leaves_sum = cu = falls = regrids = steps = 0
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        while run.time < T - 1e-12:
            if steps % every == 0:
                if tagger is not None:
                    tags, nf = run.tags_learned(tagger, *tagq(thr), cmin)
                    falls += nf
                else:
                    tags, _ = run.tags(*tagq(thr))
                regrids += 1
                run.regrid(tags, lmin)
            leaves_sum += run.forest.nleaf
            cu += run.cell_updates_per_coarse_step()
            run.coarse_step()
            steps += 1
        torch.cuda.synchronize()
        el = time.perf_counter() - t2
        r = {"regrids": regrids, "coarse_steps": steps, "mean_leaves": leaves_sum / steps, "cell_updates": cu,
             "cell_updates_per_s": cu / el, "wall_s": round(el, 4), "t": run.time}
        if tagger is not None:
            r["fallback_fraction"] = falls / max(1, leaves_sum)
        return r, run

    # reference: uniform finest level to T
    side = B << lmax
    ref_leaves = [(lmax, x, y) for y in range(side) for x in range(side)]
    lv = np.array(ref_leaves, dtype=np.int64)
    rst = S.forest_state_fast(n, 3, B, lv[:, 0], lv[:, 1], lv[:, 2], funcs, lo, hi)
    ref = AMRRun(cfg, B, lmax, ref_leaves, rst, lo, hi, dt0, graphs=True, tiling=_tiling_index(16, 16, 128))
    del rst
    while ref.time < T - 1e-12:
        ref.coarse_step()
    out["reference"] = {"leaves": len(ref_leaves), "t": ref.time, "precision": "f32"}
    g = uniform_global(ref, 0)
    del ref
    runs = {}
    for every in plain_intervals:
        for thr in thresholds:
            r, run = tagged_run(cfg, None, every, thr)
            r["l1_p_vs_uniform"] = l1_vs_uniform(run, g, 0)
            runs[f"plain_every_{every}_thr_{thr:g}"] = r
            del run
    for R, tg in taggers.items():
        r, run = tagged_run(cfg, tg, R, 4.0)
        r["l1_p_vs_uniform"] = l1_vs_uniform(run, g, 0)
        runs[f"learned_every_{R}"] = r
        del run
    if fp64:
        r, run = tagged_run(cfg64, None, 1, 4.0)
        r["l1_p_vs_uniform"] = l1_vs_uniform(run, g, 0)
        runs["plain_every_1_thr_4_f64_batched"] = r
        del run
    out["runs"] = runs
    for v in runs.values():
        assert abs(v["t"] - T) < 1e-9, (v["t"], T)
    plain_front = pareto_front([(v["l1_p_vs_uniform"], v["cell_updates_per_s"]) for k, v in runs.items()
                                if k.startswith("plain") and "f64" not in k])
    learned_front = pareto_front([(v["l1_p_vs_uniform"], v["cell_updates_per_s"]) for k, v in runs.items()
                                  if k.startswith("learned")])
    out["pareto"] = {"plain_f32": plain_front, "learned_f32": learned_front}
    # equal L1: at every point of either front, the other front's rate
    matched = []
    for l1, _ in plain_front + learned_front:
        rp, rl = rate_at(plain_front, l1), rate_at(learned_front, l1)
        if rp is not None and rl is not None:
            matched.append({"l1": l1, "learned": rl, "plain": rp, "learned_over_plain": rl / rp})
    out["equal_l1"] = sorted(matched, key=lambda m: m["l1"])
    base = runs["plain_every_1_thr_4"]
    out["equal_l1_at_plain_every_step"] = {
        "l1": base["l1_p_vs_uniform"], "plain": base["cell_updates_per_s"],
        "learned": rate_at(learned_front, base["l1_p_vs_uniform"])}
    if fp64:
        b64 = runs["plain_every_1_thr_4_f64_batched"]
        out["fp64_batched_every_step"] = {"l1": b64["l1_p_vs_uniform"], "rate": b64["cell_updates_per_s"],
                                          "learned_f32_at_that_l1": rate_at(learned_front, b64["l1_p_vs_uniform"]),
                                          "plain_f32_at_that_l1": rate_at(plain_front, b64["l1_p_vs_uniform"])}
    if per_patch:
        run = AMRRun(cfg64, B, lmax, leaves, st, lo, hi, dt0, mode="per_patch")
        run.coarse_step()
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        cu = 0
        for _ in range(2):
            cu += run.cell_updates_per_coarse_step()
            run.coarse_step()
        torch.cuda.synchronize()
        out["fp64_per_patch"] = {"rate": cu / (time.perf_counter() - t3), "coarse_steps_timed": 2,
                                 "l1": "as fp64_batched_every_step (same arithmetic, one launch per patch)"}
        del run
    # inference cost (inputs + forward) on the initial forest of the test ring, and the forward alone on a
    # large batch, against the measured BF16 tensor peak
    tg = taggers[intervals[len(intervals) // 2]]
    run = AMRRun(cfg, B, lmax, leaves, st, lo, hi, dt0)
    x = run.cnn_inputs(4.0)
    fwd = tg.outputs(run.forest.nleaf)[:2]
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tg.infer(x, run.forest.d_level, fwd)
    e0.record(stream)
    for _ in range(10):
        run.cnn_inputs(4.0)
        tg.infer(x, run.forest.d_level, fwd)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 10
    flop = 2 * 32 * ((n + 2) ** 2 * 3 * 9 + n * n * 32 * 9)      # per patch: both convolutions
    reps = max(1, 65536 // run.forest.nleaf)
    xb = x.repeat(reps, 1, 1, 1).contiguous()
    lb = run.forest.d_level.repeat(reps).contiguous()
    fb = tg.outputs(int(lb.numel()))[:2]
    tg.infer(xb, lb, fb)
    e0.record(stream)
    for _ in range(10):
        tg.infer(xb, lb, fb)
    e1.record(stream)
    torch.cuda.synchronize()
    msb = e0.elapsed_time(e1) / 10
    peak = bf16_peak()
    out["inference"] = {"leaves": run.forest.nleaf, "ms_inputs_and_forward": ms,
                        "tflops_inputs_and_forward": run.forest.nleaf * flop / (ms * 1e-3) / 1e12,
                        "batch": int(lb.numel()), "ms_forward": msb,
                        "tflops_forward": int(lb.numel()) * flop / (msb * 1e-3) / 1e12,
                        "peak_tflops": peak[0], "peak_source": peak[1],
                        "flop_per_patch": flop}
    out["inference"]["frac_forward"] = out["inference"]["tflops_forward"] / peak[0]
    return out


def tagger_kernels(nsample: int = 65536, steps: int = 20, warmup: int = 3, C: int = 3, N: int = 16,
                   batch: int = 4096):
    """The tagger's kernels alone on synthetic BF16 inputs (normal, seed 0):
    af_cnn_forward on nsample patches, with the maxima's positions (the
    training forward) and without (inference), and a training step (forward,
    backward, Adam) on `batch`; TFLOP/s of the two convolutions against the
    measured BF16 tensor peak."""
    import torch
    from paper_2205_07572_gb300.tagger import Tagger
    g = torch.Generator(device="cpu").manual_seed(0)
    xf = torch.randn((nsample, C, N + 4, N + 4), generator=g) * 2.0
    x = (xf.to(torch.bfloat16).view(torch.int16)).cuda()
    level = torch.randint(0, 8, (nsample,), generator=g, dtype=torch.int32).cuda()
    tg = Tagger(C, N, seed=0)
    out = tg.outputs(nsample)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        tg.forward(x, level, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        tg.forward(x, level, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    inf_out = out[:2]
    for _ in range(warmup):
        tg.infer(x, level, inf_out)
    e0.record(stream)
    for _ in range(steps):
        tg.infer(x, level, inf_out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_i = e0.elapsed_time(e1) / steps
    flop = 2 * 32 * ((N + 2) ** 2 * C * 9 + N * N * 32 * 9)
    peak = bf16_peak()
    label = (torch.rand(batch, generator=g) > 0.5).float().cuda()
    weight = torch.ones(batch).cuda()
    xb, lb = x[:batch].contiguous(), level[:batch].contiguous()
    fb = tg.outputs(batch)
    for _ in range(warmup):
        tg.train_step(xb, lb, label, weight, float(batch), 1e-4, fb)
    e0.record(stream)
    for _ in range(steps):
        tg.train_step(xb, lb, label, weight, float(batch), 1e-4, fb)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_t = e0.elapsed_time(e1) / steps
    tf = nsample * flop / (ms * 1e-3) / 1e12
    tf_i = nsample * flop / (ms_i * 1e-3) / 1e12
    return {"shape": {"ncomp": C, "n": N, "channels": 32}, "forward": {
                "samples": nsample, "ms": ms, "samples_per_s": nsample / (ms * 1e-3), "flop_per_sample": flop,
                "tflops": tf, "peak_tflops": peak[0], "peak_source": peak[1], "frac": tf / peak[0]},
            "inference": {"samples": nsample, "ms": ms_i, "samples_per_s": nsample / (ms_i * 1e-3),
                          "tflops": tf_i, "frac": tf_i / peak[0]},
            "train_step": {"batch": batch, "ms": ms_t, "samples_per_s": batch / (ms_t * 1e-3)}}


def bf16_peak():
    """Measured dense BF16 tensor peak (burst), TFLOP/s, and its source."""
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        if isinstance(d.get("bf16_tflops"), (int, float)):
            return float(d["bf16_tflops"]), "measured (MEASURED_PEAKS.json bf16_tflops, burst)"
    except Exception:
        pass
    return 1900.0, "fallback"


# ------------------------------------------------ variable-velocity advection
TABLE3 = {4: 5.722927e-06, 5: 7.268088e-07}   # Section 4.3, Table 3 (uniform, t = 1)


def var_velocity_bench(steps: int = 20):
    """Swirl (Section 4.3, constant-preserving flux, RK4 back-tracing), 16x16
    patches on the periodic unit square: the paper's Table 3 runs (levels 4
    and 5, two Gaussians, t = 1, CFL 0.5) on the GPU with their L1 errors, and
    the FP32 / FP64 step rate on 4096^2 cells; solid-body rotation rate too."""
    import torch
    import synth as S
    from paper_2205_07572_gb300 import af
    from paper_2205_07572_gb300.uniform import UniformRun
    out = {"workload": "swirl: stream function sin^2 sin^2 cos(pi t)/pi, 16x16 patches, periodic unit square; "
                       "solid-body rotation on [-1,1]^2"}
    n = 16
    tab = {}
    for level, px in ((4, 16), (5, 32)):
        grid = S.UniformGrid(S.Layout(n, 1), px, px)
        st = S.periodic_state(grid, [S.swirl_gaussians], nq=4)
        nsteps, dt = S.steps_to(1.0, 0.5 * grid.dx)
        res = {}
        for prec in ("f64", "f32"):
            cfg = af.config(af.ADVECTION, af.F32 if prec == "f32" else af.F64, n)
            run = UniformRun(cfg, px, px, grid.dx, grid.dy, dt, state=st, field=af.FIELD_SWIRL)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(nsteps):
                run.step()
            torch.cuda.synchronize()
            el = time.perf_counter() - t0
            host = run.state.double().cpu().numpy().reshape(st.shape)
            res[prec] = {"l1": grid.l1_error(host, 0, S.swirl_gaussians, nq=4), "wall_s": round(el, 4)}
        tab[f"level{level}_{px * n}x{px * n}"] = {**res, "paper": TABLE3[level], "steps": nsteps}
    out["table3"] = tab
    rates = {}
    for field, name, lo, hi, vmax in ((af.FIELD_SWIRL, "swirl", (0.0, 0.0), (1.0, 1.0), 1.0),
                                      (af.FIELD_SOLID_BODY, "solid_body", (-1.0, -1.0), (1.0, 1.0), np.pi * 1.01)):
        px = 256
        grid = S.UniformGrid(S.Layout(n, 1), px, px, lo, hi)
        f = S.swirl_gaussians if field == af.FIELD_SWIRL else S.gaussian(0.3, 0.2, 0.1)
        st = S.periodic_state(grid, [f], nq=2, dtype=np.float32)
        for prec in ("f32", "f64"):
            cfg = af.config(af.ADVECTION, af.F32 if prec == "f32" else af.F64, n)
            run = UniformRun(cfg, px, px, grid.dx, grid.dy, 0.45 * grid.dx / vmax, state=st, field=field, lo=lo)
            stream = torch.cuda.current_stream()
            # the default tiling or one n x n tile per patch (bulk-staged): the faster
            cands = sorted({af.default_tiling(cfg), [t[:2] for t in af.step_tilings()].index((n, n))})
            tmeas = {}
            for kt in cands:
                run.set_tiling(kt)
                for _ in range(2):
                    run.step()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(3):
                    run.step()
                e1.record(stream)
                torch.cuda.synchronize()
                tmeas[kt] = e0.elapsed_time(e1) / 3
            run.set_tiling(min(tmeas, key=tmeas.get))
            for _ in range(3):
                run.step()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k = steps if prec == "f32" else max(3, steps // 4)
            e0.record(stream)
            for _ in range(k):
                run.step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            cells = px * px * n * n
            bpc = 8 * (4 if prec == "f32" else 8)
            rates[f"{name}_{prec}"] = {"value": cells / (ms * 1e-3), "unit": "cell updates/s", "ms_per_step": ms,
                                       "achieved_gbs": cells * bpc / (ms * 1e-3) / 1e9, "cells": cells,
                                       "tiling": af.step_tilings()[run.tiling],
                                       "tried_ms": {str(af.step_tilings()[k]): round(v, 4) for k, v in tmeas.items()}}
    out["rates_4096x4096"] = rates
    return out


# FP32 / FP64 flops of one acoustic cell update in the implemented kernels:
# per component 76 adds for the orbit sums of the three nodes and 230
# multiply-adds for their two time combinations (T and Q^{n+1}); then the
# Simpson face sums (4 faces x 3 components x one multiply-add and one add),
# 8 flux scalings and the update (3 components x 2 differences and 2
# multiply-adds).  Node values of the tile's extra row and column, computed
# twice, are not counted.
ACOUSTIC_FLOP_PER_CELL = 3 * 76 + 230 * 2 + 4 * 3 * 3 + 8 + 3 * 6


def fma_peaks(repeats: int = 5):
    """Measured FMA rates of this GPU (af_fma_throughput: 8 independent
    chains per thread, 8 CTAs of 256 threads per SM), TFLOP/s, best of
    `repeats` CUDA-event timings."""
    import torch
    from paper_2205_07572_gb300 import af
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    blocks = sms * 8
    out = {}
    stream = torch.cuda.current_stream()
    for prec, name, dtype, iters in ((af.F32, "fp32", torch.float32, 2048), (af.F64, "fp64", torch.float64, 64)):
        sink = torch.empty(blocks * 256, dtype=dtype, device="cuda")
        af.fma_throughput(prec, blocks, 8, sink, stream)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            af.fma_throughput(prec, blocks, iters, sink, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = 2 * 8 * iters * blocks * 256 / (best * 1e-3) / 1e12
    return out


# ----------------------------------------------------------- CPU oracle arm
def oracle_sample(steps: int, budget_s: float = 15.0, nthreads=None):
    """Time the FP64 oracle on a bounded sample of the workload: an 8 x 8 block
    of the 32^2 patches treated as its own periodic grid (same patch shape,
    same datum, same CFL)."""
    import oracle as O
    import synth as S
    px = py = 8
    grid = S.UniformGrid(S.Layout(N_CELLS, 3), px, py, (0.5 - 4 * N_CELLS / 4096, 0.5 - 4 * N_CELLS / 4096),
                         (0.5 + 4 * N_CELLS / 4096, 0.5 + 4 * N_CELLS / 4096))
    st = np.nan_to_num(grid.state(S.pulse_plus_vortex(), nq=2))
    dt = CFL * grid.dx
    cf = O.cfg(O.ACOUSTICS, N_CELLS, grid.dx, grid.dy, dt, c=1.0)
    nt = O.max_threads() if nthreads is None else int(nthreads)
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        st = O.run_uniform(cf, px, py, 1, st, nthreads=nt)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    cells = px * py * N_CELLS * N_CELLS
    return {"value": cells * done / el, "unit": "cell updates/s", "cores": nt, "kind": "oracle",
            "sample": f"8x8 patches of 32^2 (65536 cells) of the same workload, {done} FP64 steps, {el:.1f} s"}


# ---------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", default="both", choices=["both", "f32", "f64"],
                    help="which stencil precision(s) to time (profiling runs use one)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the end-to-end, literal-size, adaptive-mesh and CPU-baseline measurements")
    ap.add_argument("--var-only", action="store_true", help="only the variable-velocity advection runs")
    ap.add_argument("--amr-profile", action="store_true",
                    help="only batched FP32 coarse steps of the acoustics levels 3-7 forest (for a launch list)")
    ap.add_argument("--amr-tile", type=int, nargs=3, default=[16, 16, 128], metavar=("TX", "TY", "THREADS"),
                    help="compiled tiling of --amr-profile")
    ap.add_argument("--learned-only", action="store_true",
                    help="only the learned-tagging experiment")
    ap.add_argument("--amr-only", action="store_true",
                    help="time only the adaptive-mesh workloads (one JSON object per workload)")
    ap.add_argument("--tagger-only", action="store_true",
                    help="only the learned tagger's forward and backward kernels on a synthetic batch")
    ap.add_argument("--patches", type=int, default=128,
                    help="patches per side of the uniform workload with --prec f32/f64 (profiling of a smaller case)")
    args = ap.parse_args()
    if args.prec != "both":
        globals()["P_SIDE"] = args.patches
    warm = max(3, args.warmup)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle as O
        O.build()
        # under torchrun (OMP_NUM_THREADS=1 per rank) rank 0 runs alone: it
        # takes the host's cores, as the single-process run does
        nt = max(O.max_threads(), os.cpu_count() or 1) if world > 1 else None
        per = []
        for k in range(warm + args.steps):
            r = oracle_sample(1, budget_s=60.0, nthreads=nt)
            if k >= warm:
                per.append(r)
        v = statistics.median(x["value"] for x in per)
        cpu = dict(per[0])
        cpu["value"] = v
        cpu["sample"] = cpu["sample"].replace("1 FP64 steps", "one FP64 step per bench step")
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cell updates/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": warm,
                "ms_per_step": 65536 / v * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD + " (oracle sample: 8x8 patches)", "l2": "inputs > L2 n/a (CPU)"},
                "cpu_baseline": cpu,
                "e2e": {"value": v, "unit": "cell updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    from paper_2205_07572_gb300 import build
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()

    if args.amr_only:
        if rank == 0:
            for case in AMR_CASES:
                print(json.dumps({"amr": case, **amr_bench(case, 8, 4, per_patch=AMR_CASES[case]["per_patch"])}),
                      flush=True)
        return
    if args.amr_profile:
        if rank == 0:
            print(json.dumps(amr_profile_run(args.steps, warm, tile=tuple(args.amr_tile))), flush=True)
        return
    if args.var_only:
        if rank == 0:
            print(json.dumps({"variable_velocity": var_velocity_bench()}), flush=True)
        return
    if args.learned_only:
        if rank == 0:
            print(json.dumps({"learned_tagging": learned_tagging()}), flush=True)
        return
    if args.tagger_only:
        if rank == 0:
            print(json.dumps({"tagger_kernels": tagger_kernels(steps=args.steps, warmup=warm)}), flush=True)
        return
    if args.prec != "both":
        r = run_ours(args.prec, args.steps, warm, rank, world, dist)
        if rank == 0:
            print(json.dumps({"prec": args.prec, "ms_per_step": r["ms"],
                              "value": world * r["cells"] / (r["ms"] * 1e-3), "unit": "cell updates/s",
                              "clocks": r["clocks"], "tiling": r["tiling"]}), flush=True)
        return
    r32 = run_ours("f32", args.steps, warm, rank, world, dist)
    r64 = run_ours("f64", max(3, args.steps // 4), warm, rank, world, dist)
    hbm, src = measured_peaks()
    cells = r32["cells"]
    traffic, traffic_src = profiled_traffic(r32["tiling"])
    value = job_rate(cells, world, r32["ms"])
    achieved = cells * BYTES_PER_CELL["f32"] / (r32["ms"] * 1e-3) / 1e9
    line = None
    if rank == 0:
        extras = not args.no_extras
        e2e = run_e2e("f32", max(3, args.steps // 4), 2, r32["tiling"]["index"]) if extras else None
        if e2e is not None:  # context: the host holding the device layout, ghost rings included
            lat = run_e2e("f32", max(3, args.steps // 4), 2, r32["tiling"]["index"], layout="lattice")
            e2e["lattice_layout"] = {k: lat[k] for k in ("value", "ms_per_step", "h2d_bytes_per_step",
                                                         "d2h_bytes_per_step", "link_gbs")}
            e2e["link_peak"] = link_peak(e2e["h2d_bytes_per_step"])
            e2e["link_frac"] = e2e["link_gbs"] / e2e["link_peak"]["both_gbs"]
        lit32 = literal_config2("f32", 50) if extras else None
        lit64 = literal_config2("f64", 10) if extras else None
        cpu = None if (args.no_cpu_baseline or not extras) else oracle_sample(20)
        if cpu is not None:
            one = oracle_sample(20, budget_s=5.0, nthreads=1)
            cpu["single_thread"] = {k: one[k] for k in ("value", "unit", "cores", "sample")}
        peaks = fma_peaks()
        f32_tf = cells * ACOUSTIC_FLOP_PER_CELL / (r32["ms"] * 1e-3) / 1e12
        f64_tf = cells * ACOUSTIC_FLOP_PER_CELL / (r64["ms"] * 1e-3) / 1e12
        alu = {"flop_per_cell": ACOUSTIC_FLOP_PER_CELL,
               "fp32": {"achieved": f32_tf, "peak": peaks["fp32"], "unit": "TFLOP/s", "frac": f32_tf / peaks["fp32"]},
               "fp64": {"achieved": f64_tf, "peak": peaks["fp64"], "unit": "TFLOP/s", "frac": f64_tf / peaks["fp64"]},
               "peak_source": "measured: af_fma_throughput (8 independent FMA chains per thread, best of 5)"}
        amr = {case: amr_bench(case, 8, 4, per_patch=AMR_CASES[case]["per_patch"]) for case in AMR_CASES} \
            if extras else None
        learned = learned_tagging() if extras else None
        var = var_velocity_bench() if extras else None
        v64 = world * cells / (r64["ms"] * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": "cell updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": warm, "ms_per_step": r32["ms"], "higher_is_better": True,
            "ms_per_step_median": r32["ms_median"], "ms_per_step_best": r32["ms_best"],
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "patches": P_SIDE * P_SIDE, "cells_per_step": cells,
                       "l2": "inputs larger than L2 (1.1 GB FP32 state per copy)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "tiling_f32": r32["tiling"], "tiling_f64": r64["tiling"]},
            "fp64": {"value": v64, "unit": "cell updates/s", "ms_per_step": r64["ms"],
                     "ms_per_step_median": r64["ms_median"], "ms_per_step_best": r64["ms_best"],
                     "achieved_gbs": cells * BYTES_PER_CELL["f64"] / (r64["ms"] * 1e-3) / 1e9,
                     "bound": "alu", "clocks": r64["clocks"]},
            "alu": alu,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "traffic_source": traffic_src,
                         "kernel": "step_kernel<float, acoustics>",
                         "peak_source": f"{src} HBM copy bandwidth",
                         "algorithmic_bytes_per_launch": cells * BYTES_PER_CELL["f32"]},
            "literal_512x512": {"f32": lit32, "f64": lit64, "note": "L2-resident (34 MB FP64 state)"},
            "amr": amr,
            "learned_tagging": learned,
            "variable_velocity": var,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "clocks": r32["clocks"],
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
