"""Cost model and roofline arithmetic used for reporting.

arXiv 2005.13425 Sec. III.A: a CG iteration costs C(D, n) = D (12n + 34)
flops (Eq. 1) and moves 24D reads + 6D writes of 8-byte words, so its
intensity is I(n) = (12n + 34) / 240 flop/B (Eq. 2).  Listing 1's ax_e alone
is (12n + 15) flops per point (6n + 6n for the forward and transposed
derivatives, 15 for the geometric contraction) and streams u plus six gxyz
words in and w out: 64 B per point in FP64, 32 B in FP32.
"""
from __future__ import annotations

import json
import os

FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
# FP64 ALU ceiling: the recipe's nominal GB300 FP64 rate (TFLOP/s).
NOMINAL_FP64_TFLOPS = 1.25


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
