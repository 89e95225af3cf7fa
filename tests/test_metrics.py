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


def _count_line_eo(n):
    """Count the FP32 instructions of an even-odd line product by walking
    its steps (pair sums/differences, Dot2 chains, output pair additions)."""
    first, dot2, norm, add, add_raw = 4, 12, 3, 11, 8
    h = n // 2
    ops = 0
    for _ in range(h):
        ops += 2 * add                       # x_l + x_{n-1-l}, x_l - x_{n-1-l}
    for _ in range(h):
        for chain_len in (h, h + (n % 2)):   # P over differences, Q over sums (+ middle)
            ops += first + dot2 * (chain_len - 1)
        ops += 2 * add_raw                   # y_m = P + Q, y_{n-1-m} = P - Q (unnormalised)
    if n % 2:
        ops += first + dot2 * h + norm       # middle output
    return ops


def test_double_float_op_counts():
    for n in range(2, 17):
        assert metrics.df_line_ops(n) == _count_line_eo(n)
    # n = 10: 71 per point per line product, 6 line products, 84 for the
    # contraction (three 3-term Dot2 sums), 22 for the partial sums, 2 for
    # the split
    assert metrics.df_fp32_ops_per_point(10) == 6 * 71 + 84 + 22 + 2
    assert abs(metrics.FP32_PEAK_TOPS - 152 * 128 * 2.07e9 / 1e12) < 1e-9
    assert metrics.cg_head_bytes_per_point() == 96


def test_recorded_traffic_needs_matching_digest(tmp_path):
    import json
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps({"kernels": {"head": {"source_digest": "abcdef0123456789",
                                                  "dram_bytes_per_launch": 393216000}}}))
    assert metrics.recorded_traffic(str(p), "head", "abcdef0123456789") == 393216000
    assert metrics.recorded_traffic(str(p), "head", "0000000000000000") is None
    assert metrics.recorded_traffic(str(p), "other", "abcdef0123456789") is None
    assert metrics.recorded_traffic(str(tmp_path / "missing.json"), "head", "abcdef0123456789") is None


def test_committed_traffic_file_is_well_formed():
    import json
    path = os.path.join(os.path.dirname(os.path.dirname(__file__)), "profiles", "traffic.json")
    rec = json.load(open(path))["kernels"]
    assert rec
    for k, v in rec.items():
        assert len(v["source_digest"]) == 16 and int(v["dram_bytes_per_launch"]) > 0, k
        assert os.path.exists(os.path.join(os.path.dirname(path), v["profile"])), k


def test_source_digest_ignores_comments_only(tmp_path):
    code = "int f(int a) {\n    return a + 1;  // one more\n}\n/* block\n comment */\n"
    (tmp_path / "k.cu").write_text(code)
    d0 = metrics.source_digest(str(tmp_path), ("k.cu",))
    (tmp_path / "k.cu").write_text(code.replace("one more", "the successor").replace("block", "other"))
    assert metrics.source_digest(str(tmp_path), ("k.cu",)) == d0
    (tmp_path / "k.cu").write_text(code.replace("a + 1", "a + 2"))
    assert metrics.source_digest(str(tmp_path), ("k.cu",)) != d0
