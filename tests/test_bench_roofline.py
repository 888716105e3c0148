"""The bench's roofline arithmetic on hand-worked numbers (CPU): the level
kernels' L2 accesses per sample, and the fractions of the mixed-probe,
separate-kind and HBM ceilings that a run's time gives."""
import math
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_accesses_per_sample():
    # level 0, M = 5: 2 + 5 position gathers and 5 node records (8-byte loads),
    # 7 atomic adds, one edge record from HBM; L2 bytes 7*8 + 5*8 + 7*8
    assert bench.sample_accesses("k_hogwild", 5, 0, False) == (12, 0, 7, 1, 152)
    # coarse levels: the level node records are 16 bytes, plus the two
    # endpoints' ancestors; 7*8 + 5*16 + 2*4 + 7*8
    assert bench.sample_accesses("k_hogwild", 5, 0, True) == (9, 5, 7, 1, 200)
    # half-precision negatives: 4-byte gathers (one request each) and the
    # epoch's copy rewrite, 12 bytes per node = per sample
    l8, l16, r8, h, b = bench.sample_accesses("k_hogwild", 5, 1, False)
    assert (l16, r8, h) == (0, 7, 1) and math.isclose(l8, 12 + 12 / 32) and b == 2 * 8 + 5 * 4 + 5 * 8 + 7 * 8 + 12


def test_fractions_of_the_ceilings():
    probes = {"l2_load8": 3e11, "l2_load16": 3e11, "l2_red8": 2e11, "l2_mix": 2.2e11, "hbm_load16": 4e10}
    l2, hbm = bench.roofline_l2_hbm("k_hogwild", 5, 0, [(1e9, False)], 100.0, probes, 6700.0)
    # 1e9 samples of 19 L2 accesses in 0.1 s: the mixed probe would take
    # 19e9 / 2.2e11 s, the separate kinds 12e9 / 3e11 + 7e9 / 2e11 s
    assert l2["frac"] == pytest.approx(19e9 / 2.2e11 / 0.1)
    assert l2["separate"]["frac"] == pytest.approx((12e9 / 3e11 + 7e9 / 2e11) / 0.1)
    assert l2["achieved"] == pytest.approx(152e9 / 0.1 / 1e9)
    assert l2["peak"] == pytest.approx(152e9 / (19e9 / 2.2e11) / 1e9)
    assert l2["algorithmic_bytes_per_sample"] == pytest.approx(152)
    # HBM: one random 16-byte record per sample
    assert hbm["frac_random16"] == pytest.approx(1e9 / 4e10 / 0.1)
    assert hbm["frac_copy"] == pytest.approx(1e9 * 16 / 0.1 / 1e9 / 6700.0)
    # a mixed run weights each level's samples by its own accesses
    l2m, _ = bench.roofline_l2_hbm("k_hogwild", 5, 0, [(1e9, False), (2e9, True)], 100.0, probes, 6700.0)
    assert l2m["frac"] == pytest.approx((1e9 * 19 + 2e9 * 21) / 2.2e11 / 0.1)
    assert l2m["algorithmic_bytes_per_sample"] == pytest.approx((152 + 2 * 200) / 3)


def test_whole_job_rate():
    assert bench.whole_job_rate(1e9, 4, 2.0) == pytest.approx(2e9)
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
