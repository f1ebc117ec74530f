"""Autotuner of af_patch_step's tile shape and threads per tile.

For a given run (anything with .set_tiling(k) and .step()), every compiled
tiling that the library accepts is timed with CUDA events on the current
stream over a few steps after warm-up, and the fastest is kept.  Results
are memoised per (equation, precision, patch size, patches, neighbour mode)
for the life of the process.

The default search space leaves out the persistent (two-window pipelined)
tiling: the library refuses it (two launches of it failed on the GPU, in
experimental builds, with a cause that reading the code has not found), and
it was slower on every workload measured before that.
"""
from __future__ import annotations

from . import af

_memo: dict = {}


def time_tiling(run, k: int, steps: int = 5, warmup: int = 2) -> float:
    """Milliseconds per step of `run` with tiling k (inf if not supported)."""
    import torch
    try:
        run.set_tiling(k)
        for _ in range(warmup):
            run.step()
    except af.AFError:
        return float("inf")
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        run.step()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def default_candidates():
    """Indices of the compiled tilings the autotuner tries by default: the
    one-tile-per-CTA kernels (persistent tilings excluded)."""
    return [k for k, t in enumerate(af.step_tilings()) if not t[3]]


def tune(run, key=None, steps: int = 5, warmup: int = 2, candidates=None):
    """Pick the fastest tiling for `run`; returns (best index, {index: ms})."""
    if key is not None and key in _memo:
        run.set_tiling(_memo[key][0])
        return _memo[key]
    cands = default_candidates() if candidates is None else candidates
    times = {k: time_tiling(run, k, steps, warmup) for k in cands}
    best = min(times, key=times.get)
    run.set_tiling(best)
    if key is not None:
        _memo[key] = (best, times)
    return best, times
