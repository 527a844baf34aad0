"""bench.py's host-side bookkeeping, without a GPU: the roofline object of the bench line
and the move counts it is built on."""
import types

import pytest

import bench


def test_move_counts_of_the_configured_instances():
    # M(M+V-2) relocations and M(M-1)/2 swaps: 155, 16,750 and 259,000 moves per iteration
    # for the tiny, paper-shaped and large instances
    for (M, V), total in (((10, 3), 155), ((100, 20), 16_750), ((400, 50), 259_000)):
        R, S = bench.moves_split(M, V)
        assert R == M * (M + V - 2) and S == M * (M - 1) // 2 and R + S == total


def test_roofline_of_a_known_launch():
    """Achieved = algorithmic int32 operations per launch over the mean launch time; peak =
    the larger of the issue bound (128 lanes per clock per SM) and the best measured mix,
    times the SMs and the clock; the gather fractions against both shared-memory rates."""
    r = {"step_ms": [10.0, 30.0], "p": types.SimpleNamespace(iterations=100), "R": 1000, "S": 500,
         "plan": types.SimpleNamespace(cluster_size=4, grid_clusters=2)}
    peaks = {"int32_ops_per_clk_sm": 96.0, "int32_add_xor_ops_per_clk_sm": 127.0,
             "lds_gather_words_per_clk_sm": 12.0, "lds_words_per_clk_sm": 32.0}
    out = bench.roofline(r, peaks, sms=10, sm_max_mhz=2000.0, traffic=1234)
    launch_s = 0.020  # the mean of 10 and 30 ms
    ops = (1000 * 20 + 500 * 30) * 100
    peak = 128 * 10 * 2.0e9 / 1e12  # the issue bound is above both measured rates
    assert out["bound"] == "alu" and out["unit"] == "Tops/s" and out["traffic"] == 1234
    assert out["achieved"] == pytest.approx(ops / launch_s / 1e12)
    assert out["peak"] == pytest.approx(peak)
    assert out["frac"] == pytest.approx(ops / launch_s / 1e12 / peak)
    assert out["sms_used"] == 8
    assert out["frac_of_sms_used"] == pytest.approx(out["frac"] * 10 / 8)
    gathers_s = (1000 * 3 + 500 * 6) * 100 / launch_s
    assert out["smem"]["gathers_per_s"] == pytest.approx(gathers_s)
    assert out["smem"]["frac_of_gather_peak"] == pytest.approx(gathers_s / (12.0 * 10 * 2.0e9))
    assert out["smem"]["frac_of_conflict_free_peak"] == pytest.approx(gathers_s / (32.0 * 10 * 2.0e9))


def test_roofline_peak_follows_a_measured_rate_above_the_issue_bound():
    r = {"step_ms": [5.0], "p": types.SimpleNamespace(iterations=1), "R": 1, "S": 0,
         "plan": types.SimpleNamespace(cluster_size=1, grid_clusters=1)}
    peaks = {"int32_ops_per_clk_sm": 140.0, "lds_gather_words_per_clk_sm": 1.0, "lds_words_per_clk_sm": 1.0}
    out = bench.roofline(r, peaks, sms=2, sm_max_mhz=1000.0, traffic=None)
    assert out["peak"] == pytest.approx(140.0 * 2 * 1.0e9 / 1e12)
    assert out["traffic"] is None
