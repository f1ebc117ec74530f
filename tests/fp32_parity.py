"""How FP32 parity is held to 1e-5 over runs of several steps.

The bound 1e-5 (normwise relative, per component) is a bound on ONE step of
the FP32 kernels against the FP64 oracle started from the same (FP32-
representable) data.  Over K steps the rounding errors of the steps add up,
and a stable linear scheme does not amplify them, so a K-step FP32 run is
held to:
  * every step, restarted from the GPU's own FP32 state, within 1e-5 of the
    oracle's step from that state (the per-step bound itself), and
  * the whole trajectory within K x 1e-5 of the oracle's FP64 trajectory.
For adaptive runs a "step" is one coarse step (all substeps, the
conservative fix and the ghost exchanges of Section 3.2); at its end every
flux register the fix reads has been consumed and reset, so the oracle's
registers carry nothing that depends on its own earlier rounding.
"""
import copy

import numpy as np

TOL32 = 1e-5
TOL64 = 1e-12


def lockstep_amr(Fo, run, steps, compare, prec, sync):
    """Advance the oracle forest Fo and the GPU run `steps` coarse steps.
    compare(F, tol) asserts that the GPU state agrees with forest F within
    tol; sync() waits for the GPU.  FP64: the trajectories at the end, to
    1e-12.  FP32: per step from the GPU's state to 1e-5, and the trajectory
    to steps x 1e-5."""
    if prec == 0:
        for _ in range(steps):
            Fo.coarse_step()
            run.coarse_step()
        sync()
        compare(Fo, TOL64)
        return
    Ft = copy.deepcopy(Fo)
    for _ in range(steps):
        sync()
        Fo.state = np.nan_to_num(run.state_in_order(Fo.leaves)).reshape(Fo.state.shape)
        Fo.coarse_step()
        Ft.coarse_step()
        run.coarse_step()
        sync()
        compare(Fo, TOL32)
    compare(Ft, steps * TOL32)
