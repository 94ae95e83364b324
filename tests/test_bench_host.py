"""Host-side arithmetic of the benchmark line (no GPU): the roofline fields
and the parsing of the clock samples taken during the timed region."""
import pytest

import bench


def test_smem_bytes_per_attempt_by_layout():
    d = 2 * 41459 / 7000   # mean degree of the G63-shaped graph
    # multi-spin coded: the measurement plan's (8 + 6 d) / 32 -- own word read
    # and written, a 4-byte neighbour word and its 2-byte index per bond
    assert bench.smem_bytes_per_attempt(("k_sweep_msc+pair", 256), d, 0.06) == pytest.approx((8 + 6 * d) / 32)
    assert bench.smem_bytes_per_attempt(("k_sweep_msc_pair", 256), 4.0, 0.5) == pytest.approx(1.0)
    # 4-replica layouts: byte read + written, threshold word, and neighbour
    # field bytes read + written on an accepted flip
    assert bench.smem_bytes_per_attempt(("k_sweep_packed", 128), 10.0, 0.1) == pytest.approx(6 + 2.0)


def test_msc_ops_per_attempt_counts_each_part():
    # per 32-replica item: 48 for the count bytes, 80 for two Philox calls, 12
    # per 4-replica group for the decision (two pair-table lookups), 4 for
    # energies; bonds: 11 ops per 4 bonds and 5 to decode with 5 planes
    assert bench.msc_ops_per_attempt(0.0) == pytest.approx((5 + 48 + 80 + 96 + 32) / 32)
    assert bench.msc_ops_per_attempt(12.0) - bench.msc_ops_per_attempt(4.0) == pytest.approx(11 / 4 * 8 / 32)
    # 3 planes (degree <= 7): 13 ops per 4 bonds, nothing to decode
    assert bench.msc_ops_per_attempt(4.0, 4) == pytest.approx((13 + 48 + 80 + 96 + 32) / 32)
    # 7 planes: 15 ops per 4 bonds, single-entry decisions (16 per group)
    assert bench.msc_ops_per_attempt(0.0, 100) == pytest.approx((7 + 48 + 80 + 128 + 32) / 32)
    assert [bench.msc_planes(d) for d in (4, 7, 8, 15, 16, 31, 32, 63, 64, 127)] == [3, 3, 4, 4, 5, 5, 6, 6, 7, 7]


def test_sweep_roofline_fractions():
    stats = {"sweep_ms": 1500.0, "sweep_launches": 1000}
    attempts = 7000 * 16384 * 10
    probe = {"int_ops_per_s": 30e12, "philox_words_per_s": 1.6e12, "smem_bytes_per_s": 38e12, "sms": 152}
    r = bench.sweep_roofline(stats, attempts, probe, 2000.0, ("k_sweep_msc+pair", 256), 12.0, 0.06)
    t = 1.5e-3
    aps = attempts / t
    assert r["bound"] == "alu" and r["unit"] == "Tops/s"
    assert r["avg_launch_ms"] == pytest.approx(1.5)
    assert r["attempts_per_s_in_kernel"] == pytest.approx(aps)
    assert r["achieved"] == pytest.approx(aps * bench.msc_ops_per_attempt(12.0) / 1e12)
    assert r["frac_first_formulation"] == pytest.approx(aps * (4.5 * 12.0 + 288) / 32 / 1e12 / 30.0)
    assert r["peak"] == pytest.approx(30.0) and r["frac"] == pytest.approx(r["achieved"] / 30.0)
    assert r["peak_derived"] == pytest.approx(152 * 128 * 2000e6 / 1e12)
    assert r["smem_frac"] == pytest.approx(aps * (8 + 6 * 12.0) / 32 / 38e12)
    assert r["smem_frac_vs_derived"] == pytest.approx(aps * (8 + 6 * 12.0) / 32 / (152 * 128 * 2000e6))
    assert r["smem_target_met"] is False
    assert r["philox_frac"] == pytest.approx(aps * 0.25 / 1.6e12)
    # without a probe the unit-count peak is used
    r2 = bench.sweep_roofline(stats, attempts, None, 2000.0, ("k_sweep_msc+pair", 256), 12.0, 0.06)
    assert r2["peak"] == pytest.approx(r2["peak_derived"]) and r2["philox_frac"] is None
    # traffic only while the captured source is the one that runs
    saved = dict(bench.SWEEP_TRAFFIC)
    try:
        bench.SWEEP_TRAFFIC["k_sweep_msc+pair"] = (123.0e6, bench.sweep_source_sha())
        r3 = bench.sweep_roofline(stats, attempts, probe, 2000.0, ("k_sweep_msc+pair", 256), 12.0, 0.06)
        assert r3["traffic"] == 123.0e6
        bench.SWEEP_TRAFFIC["k_sweep_msc+pair"] = (123.0e6, "0000000000000000")
        r4 = bench.sweep_roofline(stats, attempts, probe, 2000.0, ("k_sweep_msc+pair", 256), 12.0, 0.06)
        assert r4["traffic"] is None
    finally:
        bench.SWEEP_TRAFFIC.clear()
        bench.SWEEP_TRAFFIC.update(saved)
    assert bench.sweep_roofline({"sweep_ms": 0.0, "sweep_launches": 0}, attempts, probe, 2000.0, ("k_sweep", 512),
                                12.0, 0.06) is None


def test_recorded_traffic_belongs_to_the_current_sweep_source():
    """The DRAM traffic the bench line reports was captured on the sweep source
    that is checked in (else it reports none)."""
    entry = bench.SWEEP_TRAFFIC.get("k_sweep_msc+pair")
    assert entry is None or entry[1] == bench.sweep_source_sha()


def test_clock_summary_reads_samples_and_reasons(tmp_path):
    p = tmp_path / "clocks.csv"
    p.write_text("0, 2070, 2070, 450.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 1980, 2070, 610.5, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, 2070, 2070, 455.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "garbage line\n")
    s = bench.ClockSampler(0)
    s.path = str(p)
    out = s.summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["power_w_max"] == pytest.approx(610.5)


def test_clock_summary_without_samples(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "missing.csv")
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
