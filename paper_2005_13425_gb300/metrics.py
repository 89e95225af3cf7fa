"""Cost model and roofline arithmetic used for reporting.

arXiv 2005.13425 Sec. III.A: a CG iteration costs C(D, n) = D (12n + 34)
flops (Eq. 1) and moves 24D reads + 6D writes of 8-byte words, so its
intensity is I(n) = (12n + 34) / 240 flop/B (Eq. 2).  Listing 1's ax_e alone
is (12n + 15) flops per point (6n + 6n for the forward and transposed
derivatives, 15 for the geometric contraction) and streams u plus six gxyz
words in and w out: 64 B per point in FP64, 32 B in FP32.
"""
from __future__ import annotations

import hashlib
import json
import os
import re

FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
# FP64 ALU ceiling: the nominal GB300 FP64 rate (TFLOP/s).
NOMINAL_FP64_TFLOPS = 1.25
# Nominal FP32-pipe ceiling of GB300: 152 SMs x 128 FP32 lanes x 2070 MHz
# maximum SM clock, one FADD, FMUL or FFMA per lane per clock (10^12
# instr/s).  The ALU roofline uses the rate measured on the device
# (nb_fp32_rate); this is the context figure.
GB300_SMS = 152
FP32_LANES_PER_SM = 128
MAX_SM_MHZ = 2070.0
FP32_PEAK_TOPS = GB300_SMS * FP32_LANES_PER_SM * MAX_SM_MHZ * 1e6 / 1e12

# FP32-pipe instructions of the double-float building blocks (df.cuh):
# TwoSum 6; first product (TwoProd + cross terms) 4; Dot2 step 12;
# normalisation 3; pair addition 11; the unnormalised pair addition of the
# line outputs (add_acc_raw) 8.
_TWO_SUM, _FIRST, _DOT2, _NORM, _ADD, _ADD_RAW = 6, 4, 12, 3, 11, 8


def df_line_ops(n: int) -> int:
    """FP32 instructions of one even-odd line product of n points: n/2 pair
    sums and differences, then per output pair two Dot2 sums of n/2 terms
    and two unnormalised pair additions; odd n adds the middle term and the
    (normalised) middle output."""
    h = n // 2
    ops = 2 * h * _ADD
    if n % 2 == 0:
        ops += h * (2 * (_FIRST + _DOT2 * (h - 1)) + 2 * _ADD_RAW)
    else:
        ops += h * (2 * (_FIRST + _DOT2 * (h - 1)) + _DOT2 + 2 * _ADD_RAW)
        ops += _FIRST + _DOT2 * h + _NORM
    return ops


def df_fp32_ops_per_point(n: int) -> float:
    """FP32 instructions per point of the double-float ax_e (algorithmic:
    the operation counts of the arithmetic as written, no overheads):
    3 forward and 3 backward line products per point, the geometric
    contraction (3 Dot2 sums of 3 terms, kept unnormalised), the sum of the
    three partials (2 pair additions) and the 2 FP32 operations of the input
    split."""
    lines = 6 * df_line_ops(n) / n
    contraction = 3 * (_FIRST + 2 * _DOT2)
    return lines + contraction + 2 * _ADD + 2


def cg_flops_per_point(n: int) -> int:
    """Eq. 1: flops per degree of freedom per CG iteration."""
    return 12 * n + 34


def cg_bytes_per_point() -> int:
    """Eq. 2: 24 reads + 6 writes of 8 bytes per degree of freedom."""
    return 8 * 30


def intensity(n: int) -> float:
    """Eq. 2: I(n) = (12n + 34) / 240 flop/B."""
    return cg_flops_per_point(n) / cg_bytes_per_point()


def roofline_gflops(bw_gbs: float, n: int) -> float:
    """Bandwidth-bound performance BW x I(n) (Sec. VI.B)."""
    return bw_gbs * intensity(n)


def ax_flops_per_point(n: int) -> int:
    return 12 * n + 15


def ax_bytes_per_point(word: int = 8) -> int:
    """u + 6 gxyz read, w written."""
    return 8 * word


def cg_head_bytes_per_point(word: int = 8) -> int:
    """The fused CG head (x += alpha p, p = r + beta p, w = ax_e(p)): gxyz
    (6 words), r, p and x read, p, x and w written: 12 words per point."""
    return 12 * word


def dssum_bytes_per_point(n: int, word: int = 8) -> float:
    """Read + write of the element-boundary fraction 1 - ((n-2)/n)^3."""
    frac = 1.0 - ((n - 2) / n) ** 3
    return 2.0 * frac * word


def measured_peaks(root: str):
    """(hbm_gbs, bf16_tflops, source) from MEASURED_PEAKS.json or fallback."""
    path = os.path.join(root, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS, "fallback"


# Sources of the double-float CG head kernel; a recorded DRAM traffic figure
# is valid only for the sources it was measured on.
CG_HEAD_SOURCES = ("ax_df.cu", "ax_df_core.cuh", "df.cuh", "reduce.cuh")


_C_COMMENT = re.compile(r"//[^\n]*|/\*.*?\*/", re.S)


def code_tokens(text: str) -> str:
    """C/C++ source with comments removed and whitespace collapsed: what
    the compiler sees, so that editing a comment keeps a digest valid.
    (String literals holding comment markers do not occur in these files.)"""
    return " ".join(_C_COMMENT.sub(" ", text).split())


def source_digest(csrc_dir: str, names=CG_HEAD_SOURCES) -> str:
    h = hashlib.sha256()
    for nm in names:
        with open(os.path.join(csrc_dir, nm), encoding="utf-8") as fh:
            h.update(nm.encode() + b"\0" + code_tokens(fh.read()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(data_path: str, kernel: str, digest: str):
    """DRAM bytes per launch of `kernel` recorded in the profiles' data file
    (JSON: {"kernels": {kernel: {"source_digest": hex,
    "dram_bytes_per_launch": int, ...}}}), or None when the file or the
    entry is missing or was measured on other sources."""
    try:
        with open(data_path) as fh:
            rec = json.load(fh)["kernels"][kernel]
        if rec["source_digest"] != digest:
            return None
        return int(rec["dram_bytes_per_launch"])
    except (OSError, KeyError, TypeError, ValueError):
        return None
