"""Host logic of bench.py that decides whether a measurement stands: the
summary of the clock samples taken during the timed region, and the flop
count of the HQRRP line.  No GPU needed."""
import pytest

import bench

FIELDS = "idx,sm,smmax,power,active,hw_slow,hw_thermal,sw_thermal,sw_power"


def _row(sm, smax, hw="Not Active", hwt="Not Active", swt="Not Active", swp="Not Active"):
    return f"0, {sm}, {smax}, 900.0, 0x0, {hw}, {hwt}, {swt}, {swp}\n"


def test_clock_summary_clean_run():
    rows = [_row(2070, 2070)] * 5 + [_row(2055, 2070)]
    out = bench.parse_clock_samples(rows)
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == [] and out["samples"] == 6


def test_clock_summary_collects_every_reason_seen():
    rows = [_row(2070, 2070), _row(1800, 2070, hwt="Active"), _row(1900, 2070, swp="Active"),
            _row(2000, 2070, hw="Active", swt="Active")]
    out = bench.parse_clock_samples(rows)
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap",
                              "sw_thermal_slowdown"]
    assert out["sm_mhz"] == pytest.approx(1950.0)  # median of 2070, 1800, 1900, 2000


def test_clock_summary_skips_malformed_lines_and_reports_unsampled():
    assert bench.parse_clock_samples([])["reasons"] == ["unsampled"]
    out = bench.parse_clock_samples(["garbage\n", "0, [N/A], 2070, 1, 0, a, b, c, d\n",
                                     _row(2070, 2070)])
    assert out["samples"] == 1


def test_hqrrp_flops_leading_terms():
    # square, b dividing n: the per-step terms summed by a direct loop
    n, b = 1024, 128
    direct = 0.0
    for k in range(0, n, b):
        rm = rn = n - k
        direct += 2 * b * rm * rn + 2 * b * b * (rm - b / 3) + rm * b * b \
            + 4 * rm * (rn - b) * b + 4 * n * rm * b
    assert bench.hqrrp_flops(n, n, b) == pytest.approx(direct)
    # leading order 4 n^3 for m = n: sketch 2/3, left update 4/3, Q 2 (in units of n^3)
    big = 8192
    assert bench.hqrrp_flops(big, big, 64) / big ** 3 == pytest.approx(4.0, rel=0.03)
