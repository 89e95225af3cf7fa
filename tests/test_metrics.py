"""The reporting arithmetic reproduces the numbers the paper prints for its
cost model (Eq. 1, Eq. 2 and the Sec. VI.B rooflines)."""
import os

from paper_2005_13425_gb300 import metrics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eq2_roofline.txt")


def test_eq1_eq2_closed_forms():
    assert metrics.cg_flops_per_point(10) == 154
    assert metrics.cg_bytes_per_point() == 240
    assert abs(metrics.intensity(10) - 154 / 240) < 1e-15
    assert metrics.ax_flops_per_point(10) == 135
    assert metrics.ax_bytes_per_point() == 64 and metrics.ax_bytes_per_point(4) == 32
    assert abs(metrics.dssum_bytes_per_point(10) - 2 * 8 * (1 - 0.8 ** 3)) < 1e-12


def test_paper_printed_rooflines():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 2
    for n, bw, printed in rows:
        got = metrics.roofline_gflops(float(bw), int(n))
        # the paper prints whole GFlop/s, truncated (900 x 154/240 = 577.5 -> 577)
        assert int(got) == int(printed), (got, printed)
