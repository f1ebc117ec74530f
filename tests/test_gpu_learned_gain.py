"""What the learned tagger gains over the plain criterion (GPU): trained on
runs of the method from two ring waves, on a third ring it predicts the
plain criterion's tags over the next regrid interval, and regridding every
4 coarse steps with it keeps the solution closer to a uniform finest-level
run than the plain criterion does with the same regrids."""
import numpy as np
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
                                 train_steps=192, test_steps=32, horizon=4, epochs=10, batch=2048)


def test_tagger_agrees_with_the_plain_criterion(lt):
    ev = lt["test_eval"]
    assert ev["accuracy"] > 0.9 and ev["recall"] > 0.8, ev


def test_learned_regrids_beat_plain_regrids_at_equal_interval(lt):
    runs = lt["runs"]
    plain, learned = runs["plain_every_4"], runs["learned_every_4"]
    assert plain["regrids"] == learned["regrids"]
    assert learned["l1_p_vs_uniform"] < plain["l1_p_vs_uniform"], runs
    # not by refining everything: at most 25% more leaves on average
    assert learned["mean_leaves"] < 1.25 * plain["mean_leaves"], runs
    assert learned["fallback_fraction"] < 0.05
