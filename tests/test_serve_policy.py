"""The serving loop's choice between finishing a lone request in one
arp_parareal_solve and advancing it a level per step (host logic only)."""
import pytest

from paper_1303_6615_gb300.serve import lone_solve_worthwhile


@pytest.mark.parametrize("mean_gap,since_last,level_s,remaining,expected", [
    (None, 0.0, None, 6, True),       # no arrival history yet
    (0.010, 0.0, None, 6, True),      # no lone solve measured yet
    (0.001, 0.0005, 0.0015, 6, False),  # 1000 req/s against a 9 ms solve: newcomers would wait
    (0.100, 0.010, 0.0015, 6, True),  # 10 req/s: the next request is not expected before the solve ends
    (0.001, 1.0, 0.0015, 6, True),    # the rate has dropped: a second without arrivals
    (0.009, 0.0, 0.0015, 6, False),   # a gap equal to the solve time: keep the levels interleaved
    (0.009, 0.0, 0.0015, 5, True),    # fewer levels left: the solve fits before the next arrival
])
def test_lone_solve_policy(mean_gap, since_last, level_s, remaining, expected):
    assert lone_solve_worthwhile(mean_gap, since_last, level_s, remaining) is expected
