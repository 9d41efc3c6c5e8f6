"""Host-side helpers of bench.py (CPU only): the host description, the oracle
sample on spawned processes, the served-code grid and the capacities that set
its rates."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1204_5882_gb300 import synth as S  # noqa: E402


def test_cpu_model_names_the_cores():
    s = bench.cpu_model()
    assert s.endswith(f"{os.cpu_count()} cores") and len(s) > len(" cores") + 2


def test_oracle_sample_times_both_modes():
    r = bench.oracle_sample(S.WORKLOADS["bsc_p02_n16"], 2)
    assert r["kind"] == "oracle" and r["cores"] == min(os.cpu_count(), 100)
    assert r["minsum_fp32"]["value"] > 0 and r["exact_fp64"]["value"] > 0
    # float64 exact f (two log1p / expm1 per update) is slower than float32 min-sum
    assert r["exact_fp64"]["single_core"] < r["minsum_fp32"]["single_core"]


def test_capacities():
    # BSC: 1 - h2(p); h2(0.11) = 0.4999 (the rate-1/2 threshold)
    assert bench.capacity_of("bsc", 0.11) == pytest.approx(0.5, abs=5e-4)
    assert bench.capacity_of("bsc", 0.5) == pytest.approx(0.0, abs=1e-12)
    # BI-AWGN with +-1 inputs: 0.4859 bit at sigma^2 = 1 (SNR 0 dB), monotone in SNR
    assert bench.capacity_of("biawgn", 1.0) == pytest.approx(0.4859, abs=2e-4)
    caps = [bench.capacity_of("biawgn", s2) for s2 in (0.25, 0.5, 1.0, 2.0, 4.0)]
    assert all(a > b for a, b in zip(caps, caps[1:]))


def test_served_code_grid():
    rng = np.random.default_rng(7)
    seen = set()
    for _ in range(400):
        log2n, ch, par = bench.served_code_grid(rng)
        assert log2n in (16, 18, 20, 22)
        if ch == "bsc":
            assert 0.01 <= par <= 0.05 and round(par, 3) == par
        else:
            sigma = math.sqrt(par)
            assert 0.8 - 1e-9 <= sigma <= 1.4 + 1e-9
            assert abs(round(sigma, 2) - sigma) < 1e-9
        seen.add((log2n, ch))
    assert len(seen) == 8


def test_rooflines_and_captured_traffic():
    """The sequential decoder's roofline (f / g evaluations per launch over
    the event time, against the FP32-lane peak; ns per leaf per frame), the
    streamed stages' algorithmic bytes over their event time against the HBM
    peak, and the DRAM bytes of an ncu capture attached only to the schedule
    it was taken on."""
    F, t, s = 64, 14, 15
    prof = {"subtree": (0.0, 0, 0.0), "node": (8.0, 32, 0.0), "chain": (0.0, 0, 0.0),
            "stream_f": (0.40, 31, 31 * 50e6), "stream_g": (0.45, 31, 31 * 55e6)}
    sub, st = bench.leg_rooflines(prof, F, t, "events", 152, 2.07, s)
    ops = 32 * F * s * 2 ** s
    assert sub["kernel"] == "node" and sub["launches"] == 32
    assert sub["achieved"] == pytest.approx(ops / 8.0e-3 / 1e12)
    assert sub["peak"] == pytest.approx(152 * 128 * 2.07 / 1e3)
    assert sub["frac"] == pytest.approx(sub["achieved"] / sub["peak"])
    assert sub["ns_per_leaf_per_frame"] == pytest.approx(8.0e6 / (32 * 2 ** s))
    hbm = (bench.measured_peaks() or {}).get("hbm_gbs", 6800.0)
    assert st["achieved"] == pytest.approx(31 * (50e6 + 55e6) / 0.85e-3 / 1e9)
    assert st["frac"] == pytest.approx(st["achieved"] / hbm)
    assert st["launches"] == 62 and sub["traffic"] is None
    bench.attach_traffic(sub, "bsc_p03_n20", F, t, s, "minsum", "fp32")
    assert sub["traffic"] == bench.NCU_TRAFFIC[("bsc_p03_n20", F, t, s, "minsum", "fp32", "node")]
    for key in (("bsc_p03_n20", F, 13, s), ("bsc_p03_n20", F, t, 16), ("biawgn_s1_n24", 16, t, s)):
        other, _ = bench.leg_rooflines(prof, F, t, "events", 152, 2.07, s)
        bench.attach_traffic(other, *key, "minsum", "fp32")
        assert other["traffic"] is None, key
