"""Host logic of bench.py that needs no GPU: how the timed steps are split
into launches of one captured CUDA graph."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_graph_shape_times_exactly_the_requested_steps():
    for steps in list(range(1, 260)) + [997, 1000, 1024, 4096]:
        g, runs = bench.graph_shape(steps)
        assert g * runs == steps
        assert 1 <= g <= 100
        # no larger divisor within the cap was passed over
        assert all(steps % d for d in range(g + 1, min(steps, 100) + 1))


def test_graph_shape_keeps_short_runs_in_one_graph():
    assert bench.graph_shape(20) == (20, 1)
    assert bench.graph_shape(100) == (100, 1)
    assert bench.graph_shape(250) == (50, 5)
    assert bench.graph_shape(101) == (1, 101)
