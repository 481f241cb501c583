"""Host-side scheduling rules of the benchmark (no GPU): the fused call's group size and the
fit schedules the tuner times."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_fused_group_size_is_the_fewest_even_calls():
    assert bench.fused_group_size(50) == 13          # 13, 13, 13, 11
    assert bench.fused_group_size(8) == 8
    assert bench.fused_group_size(16) == 16
    assert bench.fused_group_size(17) == 9           # two calls: 9 + 8
    assert bench.fused_group_size(1) == 1
    for b in range(1, 65):
        g = bench.fused_group_size(b)
        calls = -(-b // g)
        assert g <= 16 and calls == -(-b // 16)      # no more calls than needed
        assert b - (calls - 1) * g >= 1              # the last call is not empty


def test_fit_phase_candidates():
    iters = [3, 4, 5, 5, 5, 6, 6, 6, 6, 7, 7, 8, 9, 12, 20]
    c = bench.fit_phase_candidates(iters)
    assert c[0] is None                              # one launch is always timed
    assert len(c) == len(set(c)) > 1
    for ph in c[1:]:
        assert list(ph) == sorted(set(ph)) and ph[-1] == 20 and ph[0] >= 1
    # every fit ends in the first phase: no schedule beyond one launch
    assert bench.fit_phase_candidates([20] * 10) == [None]
    # quantiles of [4, 5, 6] rounded up: the median 5, the rest 6 (the cap)
    assert bench.fit_phase_candidates([4, 5, 6], max_iters=6) == [None, (5, 6)]
