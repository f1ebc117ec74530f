"""What the learned tagger gains over the plain criterion (GPU), on a small
forest (2 x 2 brick, levels 2-5): trained on runs of the method from two
ring waves, on a third ring it predicts the plain criterion's tags over the
next regrid interval; regridding every 4 coarse steps with it keeps the
solution closer to a uniform finest-level run than the plain criterion does
with the same regrids; it reaches the L1 error of the plain criterion
regridding every coarse step (the paper's practice) at a higher rate of cell
updates; and the equal-L1 comparison of the two Pareto fronts (L1 distance
against cell updates per second) is well formed."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lt():
    from paper_2205_07572_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    return bench.learned_tagging(B=2, lmin=2, lmax=5, train_radii=(0.18, 0.32), test_radius=0.25,
                                 train_steps=192, test_steps=32, intervals=(4,), plain_intervals=(1, 4),
                                 thresholds=(3.0, 4.0), epochs=10, batch=2048, fp64=False, per_patch=False)


def test_tagger_agrees_with_the_plain_criterion(lt):
    ev = lt["test_eval"]["4"]
    assert ev["accuracy"] > 0.9 and ev["recall"] > 0.8, ev


def test_learned_regrids_beat_plain_regrids_at_equal_interval(lt):
    runs = lt["runs"]
    plain, learned = runs["plain_every_4_thr_4"], runs["learned_every_4"]
    assert plain["regrids"] == learned["regrids"]
    assert learned["l1_p_vs_uniform"] < plain["l1_p_vs_uniform"], runs
    # not by refining everything: at most 25% more leaves on average
    assert learned["mean_leaves"] < 1.25 * plain["mean_leaves"], runs
    assert learned["fallback_fraction"] < 0.05


def test_equal_l1_comparison_is_consistent(lt):
    """Every run reaches the same end time; the fronts are Pareto fronts
    (L1 and rate both increasing); every matched point carries both rates."""
    import bench
    T = {round(r["t"], 12) for r in lt["runs"].values()}
    assert len(T) == 1
    for key in ("plain_f32", "learned_f32"):
        fr = lt["pareto"][key]
        assert fr and all(a[0] <= b[0] and a[1] < b[1] for a, b in zip(fr, fr[1:]))
    for m in lt["equal_l1"]:
        assert m["learned"] > 0 and m["plain"] > 0
        assert math.isclose(m["learned_over_plain"], m["learned"] / m["plain"])
        assert math.isclose(m["learned"], bench.rate_at(lt["pareto"]["learned_f32"], m["l1"]))


def test_learned_tagging_reaches_plain_l1_at_higher_throughput(lt):
    """At the L1 error of the plain criterion regridding every coarse step,
    the learned tags (regridding every 4 steps) deliver more cell updates
    per second, regrids and tagging included."""
    m = lt["equal_l1_at_plain_every_step"]
    assert m["learned"] is not None and m["learned"] > m["plain"], m
