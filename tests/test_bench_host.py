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


def test_force_traffic_record_scales_by_list_entries_and_checks_the_source(tmp_path,
                                                                          monkeypatch):
    """The DRAM-traffic record is used only while the profiled kernel source is
    the current one, and it scales with the list entries of the run."""
    rec = tmp_path / "profiles"
    rec.mkdir()
    (rec / "k_force_traffic.txt").write_text(
        f"source_sha256_16={bench.force_source_hash()}\n"
        "bytes_per_launch=1000\nlist_entries=100\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "force_source_hash", lambda: "0123456789abcdef")
    assert bench.force_traffic_record(150) is None          # another source
    (rec / "k_force_traffic.txt").write_text(
        "source_sha256_16=0123456789abcdef\nbytes_per_launch=1000\nlist_entries=100\n")
    assert bench.force_traffic_record(150) == 1500.0
    assert bench.force_traffic_record() == 1000.0


def test_l2_note_follows_the_input_size():
    w = dict(theta=0.6, eps=5e-4, n_crit=256, dt=1 / 1024)
    assert bench.workload_config("a", 2_870_000, w, 1)["l2"].startswith("inputs larger")
    assert bench.workload_config("b", 500_000, w, 1)["l2"].startswith("interaction lists")
