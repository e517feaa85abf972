"""bench.py's measurement helpers on CPU: the paired learned-vs-plain
statistics use only the problems both arms solved (an arm's extra solves
change its solved count, never the common-set percentiles), the clock
sampler's parser (median SM clock, maximum, throttle reasons seen active),
the derived FP32 peak and the algorithmic per-point and per-node counts that
the roofline figures divide by."""
import dataclasses
import os

import numpy as np
import pytest

import bench


@dataclasses.dataclass
class Arm:
    solved: np.ndarray
    first_ms: np.ndarray
    first_iter: np.ndarray
    U: np.ndarray


def test_paired_statistics_use_the_common_set_only():
    a = Arm(np.array([1, 1, 1, 0, 0], bool), np.array([10.0, 20.0, 30.0, 0, 0]),
            np.array([2, 4, 6, 0, 0]), np.array([5.0, 6.0, 7.0, 0, 0]))
    # The learned arm solves two more problems, very fast: they must not enter
    # the common-set statistics.
    b = Arm(np.array([1, 0, 1, 1, 1], bool), np.array([12.0, 0, 28.0, 0.1, 0.1]),
            np.array([3, 0, 5, 1, 1]), np.array([4.0, 0, 6.5, 1.0, 1.0]))
    p = bench._paired(a, b)
    assert (p["plain_solved"], p["learned_solved"], p["common_solved"]) == (3, 4, 2)
    assert p["plain_first_ms_p50"] == pytest.approx(20.0) and p["learned_first_ms_p50"] == pytest.approx(20.0)
    assert p["plain_first_iter_p50"] == pytest.approx(4.0) and p["learned_first_iter_p50"] == pytest.approx(4.0)
    assert p["plain_mean_arrival"] == pytest.approx(6.0) and p["learned_mean_arrival"] == pytest.approx(5.25)
    assert p["plain_first_ms_p99"] == pytest.approx(np.percentile([10.0, 30.0], 99))


def test_paired_statistics_without_common_solves():
    a = Arm(np.array([1, 0], bool), np.zeros(2), np.zeros(2), np.zeros(2))
    b = Arm(np.array([0, 1], bool), np.zeros(2), np.zeros(2), np.zeros(2))
    p = bench._paired(a, b)
    assert p["common_solved"] == 0 and p["plain_first_ms_p50"] is None and p["learned_mean_arrival"] is None


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = os.path.join(tmp_path, "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.f = open(os.path.join(tmp_path, "unused.txt"), "w")
    s.proc = _Proc()
    return s


def test_clock_parser_median_max_and_reasons(tmp_path):
    row = "0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {cap}"
    lines = [row.format(sm=2070, hw="Not Active", cap="Not Active"),
             row.format(sm=2055, hw="Not Active", cap="Active"),
             row.format(sm=2070, hw="Not Active", cap="Not Active"),
             "garbage line", "0, [N/A], 2070, 1, 0, x, x, x, x"]
    r = _sampler(tmp_path, lines).stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    lines = [row.format(sm=1500, hw="Active", cap="Not Active")]
    r = _sampler(tmp_path, lines).stop()
    assert r["reasons"] == ["hw_slowdown"] and r["sm_mhz"] == 1500.0


def test_clock_parser_without_samples(tmp_path):
    assert _sampler(tmp_path, ["header only"]).stop() is None
    s = bench.ClockSampler(0)
    assert s.stop() is None                      # never started


def test_derived_peak_and_algorithmic_counts():
    assert bench.fp32_peak_tflops(152, 2070) == pytest.approx(80.54784)

    class P:
        spheres = np.zeros((32, 5))
        obs_r = np.zeros(16)
        dof = 6
    # 18 per sphere + 60 per joint + 9 per obstacle; with 32 x 16 pair tests of 8
    # flops each a UR5e check point is 5,176 flops.
    assert bench.point_flops(P) == 1080 and bench.point_flops(P) + 32 * 16 * 8 == 5176
    assert [bench.scan_bytes_per_node(d) for d in (2, 3, 6, 7)] == [20, 20, 36, 36]
