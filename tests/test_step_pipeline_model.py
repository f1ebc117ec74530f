"""CPU model of the bulk (TMA) staging schedule of the step kernels, walked
over whole launches to clear the suspects of a recorded GPU failure.

A variant of the bulk staging -- tiles at a patch's bottom or top skipping
the patch's own ghost rows -- once ended the first multi-tile launch of the
persistent (two-window) kernel with an unspecified launch failure; it was
removed and the cause was never found.  This model restates, from the
kernel source, the arithmetic of every bulk copy (bulk_issue: lattice
offsets g_org, g_lo, g_hi, the shared-memory destination, the byte count
and the expected-transaction count) and the two-window schedule of
step_kernel_pipe (window and mbarrier per tile, wait parities), and checks
them for the launch that failed (48 x 48 patches of 32^2 cells, 32 x 8
tiles, 9216 work items over the resident CTAs) and for the bench launch:
  * every copy lands inside its window's plane slot and reads inside its
    patch's plane, both ends 16-byte aligned, size a multiple of 16 bytes;
  * the bytes announced to the mbarrier equal the bytes issued, and stay
    below the mbarrier's transaction-count limit (2^20 - 1);
  * each wait uses the parity of the phase its copies complete;
  * a window is refilled only after the iteration that read it has ended
    (its barrier, after the proxy fence), never while it is being read.
The ghost-row-skip variant, as described, is checked the same way.  All of
it holds, so none of these explains the failure.  A second launch of the
same shape failed the same way later, in another experimental build; the
persistent tilings are now refused by the library (AF_ERR_UNIMPLEMENTED) and
the kernel is not launched until the cause is found."""
import numpy as np
import pytest

KG, PLANES = 2, 4


def plane_stride(n):
    return ((n + 2 * KG + 1) ** 2 + 7) // 8 * 8


def geo(tmx, tmy):
    wx, wy = tmx + 2 * KG + 1, tmy + 3
    return wx, (wx * wy + 12 + 3) // 4 * 4


def win_off(wx, esz):
    e = 16 // esz
    return e + ((KG - 1) * wx + KG - 1) % e


def copies(n, tmx, tmy, y0, y1, esz, skip_ghost_rows=False):
    """(window-slot offset, lattice offset, elements) of one plane's bulk copy
    of a full-width tile [0, n) x [y0, y1), as bulk_issue computes it; with
    skip_ghost_rows the copy leaves out the window rows outside [0, n)."""
    wx, wsz = geo(tmx, tmy)
    e = 16 // esz
    assert wx == n + 2 * KG + 1
    wh = y1 - y0 + 3
    g_org = (y0 - 1 + KG) * wx + (KG - 1)
    r0, r1 = 0, wh                       # window rows copied
    if skip_ghost_rows:
        r0 = 1 if y0 == 0 else 0
        r1 = wh - (y1 + 2 - n) if y1 + 2 > n else wh
    g_lo = (g_org + r0 * wx - 1) // e * e
    g_hi = (g_org - 1 + r1 * wx + e - 1) // e * e
    return win_off(wx, esz) + (g_lo - g_org), g_lo, g_hi - g_lo


def tiles(n, tmy):
    """Row bands of af_build_step_work for a patch with eight same-level
    neighbours: [0, n) cut into near-equal bands of at most tmy rows."""
    nb = -(-n // tmy)
    cuts = [round(k * n / nb) for k in range(nb + 1)]
    return list(zip(cuts[:-1], cuts[1:]))


@pytest.mark.parametrize("esz", [4, 8])
@pytest.mark.parametrize("skip", [False, True])
@pytest.mark.parametrize("n,tmx,tmy", [(32, 32, 8), (32, 32, 16), (32, 32, 32), (16, 16, 16)])
def test_bulk_copies_stay_in_bounds_and_aligned(n, tmx, tmy, skip, esz):
    wx, wsz = geo(tmx, tmy)
    plane = plane_stride(n)
    ncp = 3 * PLANES
    for y0, y1 in tiles(n, tmy):
        if (y0 * wx) % (16 // esz):
            continue                      # staged element by element, not in bulk
        dst, src, cnt = copies(n, tmx, tmy, y0, y1, esz, skip)
        assert dst >= 0 and dst + cnt <= wsz, (y0, y1, dst, cnt, wsz)
        assert src >= 0 and src + cnt <= plane, (y0, y1, src, cnt, plane)
        assert (dst * esz) % 16 == 0 and (src * esz) % 16 == 0 and (cnt * esz) % 16 == 0
        # the window entries the stencil reads, rows 0 .. wh-1 and columns
        # 0 .. n+2 of each, lie inside the slot
        wh = y1 - y0 + 3
        assert win_off(wx, esz) + (wh - 1) * wx + n + 2 < wsz
        tx = cnt * esz * ncp
        assert tx < (1 << 20) - 1


def _pipeline_schedule(nwork, grid):
    """Per CTA of step_kernel_pipe: the tiles it runs, the window each is
    staged into, the barrier it completes on and the parity waited for."""
    sched = []
    for cta in range(min(grid, nwork)):
        phase = [0, 0]
        uses = []
        t = cta
        # first tile: window 0, barrier 0
        uses.append((t, 0, 0, phase[0]))
        phase[0] ^= 1
        b = 0
        while t < nwork:
            tn = t + grid
            if tn < nwork:
                uses.append((tn, b ^ 1, b ^ 1, phase[b ^ 1]))
                phase[b ^ 1] ^= 1
            t = tn
            b ^= 1
        sched.append(uses)
    return sched


@pytest.mark.parametrize("px,grid", [(48, 152 * 3), (48, 152 * 4), (128, 152 * 3)])
def test_pipeline_windows_barriers_and_parities(px, grid):
    """The persistent kernel's schedule as its code computes it: tile k of a
    CTA is staged into window k mod 2 and completes on barrier k mod 2; the
    wait parity it uses is the number of earlier completions of that barrier
    mod 2; tile k+1 is issued at the start of iteration k, after the barrier
    that ended iteration k-1, the last reader of that window."""
    nwork = px * px * 4
    for uses in _pipeline_schedule(nwork, grid):
        done = [0, 0]
        for k, (t, win, bar, par) in enumerate(uses):
            assert win == k % 2 and bar == k % 2
            assert par == done[bar] % 2
            done[bar] += 1
            # issued in iteration k-1 (k >= 1), whose reader of window k % 2
            # was tile k-2 in iteration k-2: separated by iteration k-2's end
            if k >= 2:
                assert uses[k - 2][1] == win
