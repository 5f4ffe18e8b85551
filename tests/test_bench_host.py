"""Host-side arithmetic of bench.py's roofline object (no GPU): the
block-product figures follow the algorithmic-bytes model of the
per-frequency products (Eq. (blockDiagonal): one B x B spectrum block and the
input and output vectors per frequency and right-hand side)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def test_measured_traffic_per_frequency_is_the_algorithmic_stream(bench):
    # the ncu-measured DRAM bytes per frequency of the B = 1200, one
    # right-hand-side product: the float-float block (B^2 x 16 bytes) plus the
    # two vectors (2 x B x 16 bytes), within 1 % (no re-reads)
    B, R = bench.BP_TRAFFIC_SHAPE
    algorithmic = B * B * 16 + 2 * R * B * 16
    assert algorithmic <= bench.BP_TRAFFIC_PER_FREQUENCY <= 1.01 * algorithmic


def test_block_product_roofline_scales_traffic_by_frequencies(bench):
    w = bench.WORKLOADS[bench.WORKLOAD]
    B, F = 1200, 200
    assert len(w.directions) == bench.BP_TRAFFIC_SHAPE[1]
    prof = {"block_product": (10, 7.5), "build_blocks": (1, 3.0)}
    bp_bytes = F * B * B * 16 + 2 * F * B * 16
    bp_ms = 0.68
    bp_gbs = bp_bytes / (bp_ms / 1e3) / 1e9
    roof = bench.dominant_roofline(("block_product", prof["block_product"]), prof, w, None, None, 2, 6748.0, {},
                                   bp_gbs, bp_ms, B, F)
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["frac"] == pytest.approx(bp_gbs / 6748.0)
    assert roof["traffic"] == pytest.approx(bench.BP_TRAFFIC_PER_FREQUENCY * F)
    assert 1.0 <= roof["traffic"] / bp_bytes < 1.01
    assert roof["ms_per_launch_in_timed_steps"] == pytest.approx(0.75)
    # no measured counters for another block size: traffic is null
    other = bench.dominant_roofline(("block_product", prof["block_product"]), prof, w, None, None, 2, 6748.0, {},
                                    bp_gbs, bp_ms, 1000, F)
    assert other["traffic"] is None


def test_unmodelled_kernel_reports_no_fraction(bench):
    w = bench.WORKLOADS[bench.WORKLOAD]
    roof = bench.dominant_roofline(("givens", (5, 1.0)), {}, w, None, None, 2, 6748.0, {}, 0.0, 0.0)
    assert roof["bound"] == "unmodelled" and roof["frac"] is None and roof["traffic"] is None
