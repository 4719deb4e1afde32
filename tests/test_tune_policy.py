"""The offline tuner's choice (CPU only): the fastest schedule per regime, and
the schedules each grid size offers."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_1303_6615_gb300.tune import pick, schedules_for  # noqa: E402


def test_pick_is_the_fastest():
    assert pick({2: 0.881, 3: 0.767}) == 3
    assert pick({2: 0.326, 3: 0.545}) == 2
    assert pick({1: 1.0}) == 1


def test_schedules_per_grid_size():
    assert schedules_for(3) == [1]            # N = 8: N/4 and N/2 are both 32 threads
    assert schedules_for(7) == [1, 2]         # N = 128: no lane pairs below 256
    assert schedules_for(8) == [1, 2, 3]      # N = 256: no radix-16 plan below 512
    assert schedules_for(9) == [1, 2, 3, 4]
    assert schedules_for(10) == [1, 2, 3, 4]
    assert schedules_for(11) == [1, 3, 4]     # N = 2048: N/2 would exceed 512 threads
