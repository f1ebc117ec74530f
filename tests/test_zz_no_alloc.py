"""af_mass_noalloc: the allocation-free variant of af_mass, for callers that
cannot allocate device memory (their own pool allocator owns the device, or
their time loop must not call cudaMalloc / cudaFree, which synchronise the
device).  Checked through the C ABI against af_mass on two calls in a row,
on a small forest (one partial sum per leaf) and on a forest of more than
256 leaves (256 blocks, several leaves per block, all three components).
Named so that pytest collects it last."""
import numpy as np
import pytest

import synth as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sorted(leaves):
    return sorted(leaves, key=lambda t: (t[0], t[2], t[1]))


@pytest.mark.parametrize("big", [False, True])
@pytest.mark.parametrize("prec", [0, 1])
def test_mass_noalloc_matches_mass_on_consecutive_calls(prec, big):
    from paper_2205_07572_gb300 import af, build
    from paper_2205_07572_gb300.amr import Forest
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 8 if big else 16
    if big:   # 3 x 3 brick, levels 2-4 along a diagonal band: several hundred leaves
        B, lmax = 3, 4
        leaves = _sorted(S.balanced_forest(B, 2, lmax, lambda l, x, y: abs(x - y) <= 1))
        assert len(leaves) > 300
    else:
        B, lmax = 1, 3
        leaves = _sorted(S.balanced_forest(1, 2, 3, lambda l, x, y: x == y))
    F = Forest(B, lmax, leaves)
    tdt = torch.float64 if prec == 0 else torch.float32
    cfg = af.config(af.ACOUSTICS, prec, n, c=1.0)
    first = S.random_state(S.Layout(n, 3), len(leaves), seed=11).reshape(len(leaves), -1) + 0.5
    second = S.random_state(S.Layout(n, 3), len(leaves), seed=12).reshape(len(leaves), -1)
    scratch = torch.zeros(af.mass_scratch_bytes(len(leaves), 3) // 8, dtype=torch.float64, device="cuda")
    for data in (first, second):
        st = torch.from_numpy(np.nan_to_num(data)).to(tdt).cuda()
        ref = torch.zeros(3, dtype=torch.float64, device="cuda")
        got = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        af.mass(cfg, F.c, st, 1 / 16, 1 / 16, scratch, ref)
        af.mass_noalloc(cfg, F.c, st, 1 / 16, 1 / 16, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.isfinite(g).all()
        assert np.abs(g - r).max() <= 1e-12 * max(1.0, np.abs(r).max())
    # a one-component problem after the three-component ones reuses the array
    cfg1 = af.config(af.ADVECTION, prec, n, 1.0, 0.5)
    one = S.random_state(S.Layout(n, 1), len(leaves), seed=3).reshape(len(leaves), -1)
    st = torch.from_numpy(np.nan_to_num(one)).to(tdt).cuda()
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    got = torch.zeros(1, dtype=torch.float64, device="cuda")
    af.mass(cfg1, F.c, st, 1 / 16, 1 / 16, scratch, ref)
    af.mass_noalloc(cfg1, F.c, st, 1 / 16, 1 / 16, got)
    torch.cuda.synchronize()
    assert abs(got.item() - ref.item()) <= 1e-12 * max(1.0, abs(ref.item()))
