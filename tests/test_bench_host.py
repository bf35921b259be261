"""Host arithmetic of bench.py (no GPU): the launch count it reports per step, the
whole-job throughput over ranks, the roofline denominator."""
import json
import os
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _tree(grid_level, levelmax, n_ghost=0, n_inst=0):
    return SimpleNamespace(t=SimpleNamespace(grid_level=grid_level, n_ghost=n_ghost, n_inst=n_inst),
                           levelmax=levelmax)


def test_launches_on_the_uniform_benchmark_box():
    # the z-column kernel and two restriction launches (levels 6-4 and 3-1)
    assert bench.launches_per_step(_tree(8, 8)) == 3


def test_launches_on_the_plummer_mesh():
    # column kernel, ghost pass, tile kernel, reflux of levels 11..7, restriction of 6..1
    assert bench.launches_per_step(_tree(8, 12, n_ghost=770758)) == 1 + 2 + 5 + 2


def test_launches_of_a_box_batch_and_a_coarse_tree():
    assert bench.launches_per_step(_tree(0, 0, n_inst=48)) == 1
    # complete to level 2 only: no column kernel; tiles (no ghosts); reflux of levels 3..1
    assert bench.launches_per_step(_tree(2, 4)) == 1 + 3


def test_job_value_counts_every_rank_over_the_slowest_time():
    assert bench.job_value(1000, 1, 2.0) == 1000 / 2e-3
    assert bench.job_value(1000, 4, 2.0) == 4 * 1000 / 2e-3
    assert bench.job_ms(1.5, 1, "cpu") == 1.5


def test_peak_is_the_measured_hbm_rate_when_recorded():
    hbm, kind = bench.peaks()
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        assert kind == "measured" and hbm == float(json.load(open(p))["hbm_gbs"])
    else:
        assert (hbm, kind) == (6800.0, "fallback")
