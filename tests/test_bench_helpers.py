"""bench.py's roofline numerator and JSON helpers on the CPU: the algorithmic
bytes per launch stated in the design (deposit 12 B per 2D FP32 particle,
push 36 B per particle plus the combined field once)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_algorithmic_bytes_2d_landau():
    import bench
    np_, n, d = 4194304, 10, 2
    a = bench.algorithmic_bytes(np_, n, d)
    assert a["deposit"] == np_ * 12                       # u (2 floats) + w
    assert a["push"] == np_ * 36 + 2 * (1 << 20) * 4      # read u, v, w; write u, v; field once
    assert abs(a["push"] / 1e6 - 159.4) < 0.1 and abs(a["deposit"] / 1e6 - 50.3) < 0.1


def test_algorithmic_bytes_3d():
    import bench
    a = bench.algorithmic_bytes(16777216, 7, 3)
    assert a["deposit"] == 16777216 * 16
    assert a["push"] == 16777216 * 52 + 3 * (1 << 21) * 4


def test_measured_peak_is_read():
    import bench
    peak, kind = bench.measured_peaks()
    assert peak > 1000 and kind in ("measured", "fallback")
