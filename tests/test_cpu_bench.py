"""Host logic of bench.py: the clock record that decides whether a timed run
counts (throttle reasons, median SM clock), and the workload generators of
the batched and served configurations, checked against their stated
readings (batched sizes T = round(2^(12 + 6u)), domain the next power of
two; served classes of floor((N - 3) / 486) transactions).  No GPU."""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2603_10242_gb300 import inputs  # noqa: E402

HEADER_FREE = [  # index, sm, max sm, power, active mask, hw, hw_thermal, sw_thermal, sw_power
    "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "1, 1200, 2070, 400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
    "0, 2055, 2070, 1000.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
    "0, 1980, 2070, 1398.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
]


def _write(tmp_path, lines):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(lines) + "\n")
    return str(p)


def test_clock_summary_filters_device_and_collects_reasons(tmp_path):
    s = bench._clock_summary(_write(tmp_path, HEADER_FREE), 0)
    assert s["samples"] == 3 and s["sm_max_mhz"] == 2070.0
    assert s["sm_mhz"] == 2055.0  # median of 2070, 2055, 1980
    assert s["reasons"] == ["sw_power_cap"]  # device 1's samples are not ours
    s1 = bench._clock_summary(_write(tmp_path, HEADER_FREE), 1)
    assert s1["samples"] == 1 and s1["sm_mhz"] == 1200.0 and s1["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_thermal_and_unsampled(tmp_path):
    lines = ["0, 1500, 2070, 1400.0, 0x48, Active, Active, Not Active, Not Active",
             "0, garbage, 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = bench._clock_summary(_write(tmp_path, lines), 0)
    assert s["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"] and s["samples"] == 1
    empty = bench._clock_summary(str(tmp_path / "missing.csv"), 0)
    assert empty["sm_mhz"] is None and empty["reasons"] == ["unsampled"]


def test_batch_sizes_follow_the_log_uniform_reading():
    k = 64
    sizes = bench.batch_sizes(4000, k)
    words = inputs.splitmix64(4000, inputs.PURPOSE["sizes"], k)
    assert len(sizes) == k
    for (log_n, t, n_perm, n_pack, bits), w in zip(sizes, words):
        u = (int(w) >> 11) / float(1 << 53)
        assert 0.0 <= u < 1.0
        assert abs(t - 2.0 ** (12 + 6 * u)) <= 0.5
        assert 4096 <= t <= 1 << 18
        assert (1 << (log_n - 1)) < t <= (1 << log_n)  # next power of two
        assert n_perm == (t - 3) // 243 and n_pack == 0 and bits == 0
        assert 243 * n_perm + 3 <= t  # permutations, 2 input rows and >= 1 chain row fit
    # log-uniform: about a sixth of the sizes per octave of the 2^12..2^18 range
    octaves = [min(5, int(math.log2(t) - 12)) for _, t, *_ in sizes]
    assert all(octaves.count(o) >= 3 for o in range(6))


@pytest.mark.parametrize("log_n,cap", [(19, 1078), (20, 2157), (21, 4315), (22, 8630), (23, 17260)])
def test_serve_class_capacities(log_n, cap):
    params, c = bench.serve_class_params(log_n)
    assert c == cap
    ln, rows, n_perm, n_pack, bits = params
    assert ln == log_n and rows == 1 << log_n and n_perm == 2 * cap and n_pack == 0 and bits == 0
    # 2 permutations of 243 rows per transaction, 2 input rows, and at least one chain row
    assert 486 * cap + 3 <= rows < 486 * (cap + 1) + 3


def test_sm_max_clock_source(tmp_path):
    """The roofline's clock: the sampled maximum when there is one, else the
    driver's measured-peaks record or the GB300 default."""
    assert bench._sm_max_mhz({"sm_max_mhz": 1965.0}) == 1965.0
    v = bench._sm_max_mhz({"sm_max_mhz": None})
    assert v > 1000.0


def test_traffic_belongs_to_the_current_kernel():
    """The recorded DRAM traffic names the kernel version its capture was
    taken on; the bench reports it only for that version."""
    t = bench.G1_BUCKET_TRAFFIC
    assert t["bytes_per_unit"] > 0 and "ncu" in t["source"]
    assert isinstance(bench.G1_BUCKET_KERNEL_VERSION, str)
