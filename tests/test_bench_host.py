"""Host-side pieces of bench.py that need no GPU: the GEMM phase times behind the rooflines and the
description of the q x q cores the timed solves used."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_w_time_from_its_side_stream_mark():
    # W = G^T L on the side stream beside the FP64 C core: the main-stream phase ends with the core
    # (0.3136 ms); W's own time is its side mark minus the main phases before it
    ph = {"G=AS | D core": 0.2256, "S^T G": 0.0221, "W=G^TL | C core": 0.3136, "V, S^": 0.0161,
          "update L + next S": 0.4117, "@C core done": 0.5406, "@W done": 0.4720, "@next D core done": 0.9912}
    assert abs(bench.gemm_ms(ph, "W=G^TL | C core") - (0.4720 - 0.2256 - 0.0221)) < 1e-12
    assert bench.gemm_ms(ph, "G=AS | D core") == 0.2256
    assert bench.gemm_ms(ph, "update L + next S") == 0.4117
    assert bench.gemm_ms(ph, "S=LS~") is None


def test_w_time_without_side_mark_is_the_phase():
    ph = {"sketch": 0.01, "S=LS~": 0.2, "G=AS | D core": 0.2254, "S^T G": 0.0221, "W=G^TL | C core": 0.2236}
    assert bench.gemm_ms(ph, "W=G^TL | C core") == 0.2236
    # a mark that precedes the phase start (clock skew) falls back to the phase length
    ph["@W done"] = 0.1
    assert bench.gemm_ms(ph, "W=G^TL | C core") == 0.2236


class _Args:
    def __init__(self, core):
        self.core = core


class _B:
    RB_FP64, RB_FP32, RB_BF16X3 = 0, 1, 6


def test_core_description_follows_the_options():
    assert bench.core_desc(_Args("default"), _B.RB_BF16X3, _B)["C (S^T A S)"].startswith("fp64")
    assert bench.core_desc(_Args("default"), _B.RB_BF16X3, _B)["D (S~^T S~)"] == "fp32"
    assert bench.core_desc(_Args("fp32"), _B.RB_BF16X3, _B) == {"C (S^T A S)": "fp32", "D (S~^T S~)": "fp32"}
    assert bench.core_desc(_Args("fp64"), _B.RB_BF16X3, _B) == {"C (S^T A S)": "fp64", "D (S~^T S~)": "fp64"}
    assert bench.core_desc(_Args("default"), _B.RB_FP32, _B)["C (S^T A S)"] == "fp32"
