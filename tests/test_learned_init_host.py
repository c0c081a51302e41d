"""Host logic of the learned-initialiser evaluation, on CPU: the step count
to reach the default run's optimum.  No GPU is used."""
import numpy as np

from paper_2505_00136_gb300 import learned_init as li


def test_steps_to_reach_counts_from_one_and_caps():
    h = np.array([10.0, 5.0, 2.0, 1.5, 1.0])
    assert li.steps_to_reach(h, 1.0, 0.0) == 5
    assert li.steps_to_reach(h, 1.0, 0.5) == 4            # 1.5 <= 1 + 0.5
    assert li.steps_to_reach(h, 10.0, 0.0) == 1
    assert li.steps_to_reach(h, 0.5, 1e-6) == len(h) + 1  # never reached: the cap + 1


def test_steps_to_reach_scales_the_tolerance_by_the_magnitude():
    # NLML values are often negative: the band is rtol |target| above the target
    h = np.array([-90.0, -99.0, -99.95, -100.0])
    assert li.steps_to_reach(h, -100.0, 1e-3) == 3        # -99.95 <= -100 + 0.1
    assert li.steps_to_reach(h, -100.0, 1e-4) == 4
    # overshooting below the target counts as reached
    assert li.steps_to_reach(np.array([5.0, -1.0, 3.0]), 0.0, 0.0) == 2
