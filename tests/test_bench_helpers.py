"""Host-side helpers of bench.py: the confidence interval of the median, per-step
samples, the clock record, the traffic record and the peak file."""
import json
import math
import random

import bench


def test_median_ci95_uses_binomial_order_statistics():
    xs = list(range(1, 21))  # n = 20: P(Bin(20, 1/2) <= 5) = 0.0207 -> order statistics 6 and 15
    med, lo, hi = bench.median_ci95(list(reversed(xs)))
    assert (med, lo, hi) == (10.5, 6, 15)
    cover = 1 - 2 * sum(math.comb(20, k) for k in range(6)) / 2 ** 20
    assert 0.95 <= cover < 0.97


def test_median_ci95_small_samples_span_the_range():
    assert bench.median_ci95([3.0, 1.0, 2.0]) == (2.0, 1.0, 3.0)


def test_median_ci95_covers_the_median_about_95_percent():
    rng = random.Random(5)
    hits = 0
    for _ in range(2000):
        xs = [rng.expovariate(1.0) for _ in range(20)]
        _, lo, hi = bench.median_ci95(xs)
        hits += lo <= math.log(2) <= hi  # the exponential law's median
    assert 0.94 <= hits / 2000 <= 0.98


def test_step_samples_rates_follow_the_times():
    s = bench.step_samples([50.0] * 10 + [40.0, 60.0] * 5, 1e9)
    assert s["n"] == 20 and s["median_ms"] == 50.0
    assert s["median_gbs"] == 20.0
    lo_gbs, hi_gbs = s["ci95_gbs"]
    assert lo_gbs <= s["median_gbs"] <= hi_gbs  # slower step -> lower rate first


def test_clock_summary_reads_reasons_and_skips_bad_lines():
    ok = "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    cap = "0, 2040, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1900, 2070, 1400.0, 0x8, Active, Not Active, Not Active, Not Active"
    r = bench.ClockSampler.summarise([ok, ok, cap, "garbage", "0, [N/A], 2070"])
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.ClockSampler.summarise([ok, hot])["reasons"] == ["hw_slowdown"]
    assert bench.ClockSampler.summarise(["garbage"]) is None


def test_traffic_record_matches_only_its_sources_digest():
    kernel = "k_zmarch<F64_SCALED4>"
    recs = [ln.split() for ln in open(bench.os.path.join(bench.ROOT, "profiles", "traffic.txt"))
            if ln.startswith("TRAFFIC " + kernel + " ")]
    assert len(recs) == 1
    n_cap, digest = int(recs[0][2]), recs[0][4]
    at_cap = bench.profiled_traffic(kernel, digest, n_cap)
    algo = 3 * n_cap ** 3 * 8
    assert at_cap is not None and algo <= at_cap < 1.05 * algo  # measured: no re-reads beyond halos
    assert bench.profiled_traffic(kernel, digest, n_cap // 2) == at_cap / 8  # scaled by the node count
    assert bench.profiled_traffic(kernel, "0" * 16, n_cap) is None
    assert bench.profiled_traffic("k_unknown", digest, n_cap) is None


def test_measured_peaks_falls_back_without_the_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6767.4}))
    assert bench.measured_peaks() == (6767.4, "measured")
