"""The byte and flop model behind the benchmark's roofline (CPU): the per-site figures the
documentation derives by hand, one launch of the 64^3 x 16 bundle solve, and the benchmark's
record of the reliable-update thresholds against the library's source."""
import os
import re

import pytest

from paper_1409_1510_gb300 import accounting as acc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_per_site_flops():
    # 16 complex 3x3 matrix-vector products (66 flop) and 15 colour-vector additions (6 flop)
    assert acc.DSLASH_FLOPS_PER_SITE == 16 * 66 + 15 * 6 == 1146
    assert acc.CG_FLOPS_PER_SITE == 2 * 1146 + 72


def test_compulsory_bytes_of_the_fp16_dslash():
    """FP16 storage: 16 links of 18 halves per output site (576 B) plus one float scale per field
    (8 B), and per right-hand side one 16-byte record in and one out."""
    for n in (1, 4, 16):
        got = acc.compulsory_bytes(n, 2, 2, 18, 8.0, 4.0)
        assert got == 584 + 32 * n, (n, got)


def test_bundle_solve_bytes_of_one_benchmark_launch():
    """64^3 x 16 (V/2 = 2,097,152), 16 right-hand sides, FP16: 172 bundle iterations, 2740
    right-hand-side iterations, 14 recomputation passes, 112 recomputations -> per even site
    172 x 1168 + 2740 x 264 + 14 x 4608 + 112 x 408 + 16 x 160 bytes."""
    vh = 64 * 64 * 64 * 16 // 2
    per_site = 172 * 1168 + 2740 * 264 + 14 * 4608 + 112 * 408 + 16 * 160
    got = acc.bundle_solve_bytes(2, vh, 2740, 172, 112, 14, 16)
    assert got == per_site * vh == 2174796955648


def test_recompute_flops():
    vh = 131072
    assert acc.recompute_flops(vh, 7) == 2 * 1146 * vh * 7


def test_benchmark_thresholds_match_the_library():
    """bench.py names the reliable-update threshold of each storage precision in its workload
    string; the values must be the ones the library's default_delta returns."""
    import bench
    src = open(os.path.join(ROOT, "paper_1409_1510_gb300", "csrc", "solver.cu")).read()
    body = src[src.index("static double default_delta(int prec)"):]
    body = body[:body.index("}\n")]
    cases = dict(re.findall(r"case HISQ_(FP32|FP16): return ([0-9.]+);", body))
    default = float(re.search(r"default: return ([0-9.]+);", body).group(1))
    assert bench.DEFAULT_DELTA["fp32"] == pytest.approx(float(cases["FP32"]))
    assert bench.DEFAULT_DELTA["fp16"] == pytest.approx(float(cases["FP16"]))
    assert bench.DEFAULT_DELTA["bf16"] == pytest.approx(default)
