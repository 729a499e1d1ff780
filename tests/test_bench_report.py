"""Report fields of bench.py that are computed on the host: the class-4 HBM
roofline from the floor of its algorithmic bytes (the Hlc block written once)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_class4_roofline_floor_bytes():
    bench = _bench()
    # the precision workload's class-4 block: 30000 L2 functions x 20000 contracted rows
    r = bench.class4_roofline(30000, 20000, 12.5, {"hbm_gbs": 6800.0})
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["bytes_per_launch"] == 8.0 * 30000 * 20000
    assert r["achieved"] == pytest.approx(4.8e9 / 12.5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0)
    assert 0.0 < r["frac"] < 1.0


def test_class4_roofline_degenerate():
    bench = _bench()
    assert bench.class4_roofline(0, 20000, 1.0, {"hbm_gbs": 1.0}) is None      # no L2 functions
    assert bench.class4_roofline(100, 0, 1.0, {"hbm_gbs": 1.0}) is None        # no contracted rows
    assert bench.class4_roofline(100, 100, 0.0, {"hbm_gbs": 1.0}) is None      # not timed
    r = bench.class4_roofline(100, 100, 1.0, {})                                # no measured peak
    assert r["peak"] is None and r["frac"] is None and r["achieved"] > 0
