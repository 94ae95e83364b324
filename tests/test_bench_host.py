"""Host-side arithmetic of the benchmark line (no GPU): the roofline fields
and the parsing of the clock samples taken during the timed region."""
import pytest

import bench


def test_smem_bytes_per_attempt_by_layout():
    d = 2 * 41459 / 7000   # mean degree of the G63-shaped graph
    # multi-spin coded: neighbour words + own word read and written per
    # 32-replica item, plus two 4-byte table halves per attempt
    assert bench.smem_bytes_per_attempt(("k_sweep_msc+pair", 256), d, 0.06) == pytest.approx((4 * d + 8) / 32 + 8)
    assert bench.smem_bytes_per_attempt(("k_sweep_msc_pair", 256), 4.0, 0.5) == pytest.approx(0.75 + 8)
    # 4-replica layouts: byte read + written, threshold word, and neighbour
    # field bytes read + written on an accepted flip
    assert bench.smem_bytes_per_attempt(("k_sweep_packed", 128), 10.0, 0.1) == pytest.approx(6 + 2.0)


def test_sweep_roofline_fractions():
    stats = {"sweep_ms": 1500.0, "sweep_launches": 1000}
    attempts = 7000 * 16384 * 10
    r = bench.sweep_roofline(stats, attempts, {"sm_max_mhz": 2000.0}, ("k_sweep_msc+pair", 256), 12.0, 0.06)
    t = 1.5e-3
    assert r["bound"] == "alu" and r["unit"] == "Tops/s"
    assert r["avg_launch_ms"] == pytest.approx(1.5)
    assert r["achieved"] == pytest.approx(attempts * bench.OPS_PER_ATTEMPT / t / 1e12)
    assert r["peak"] == pytest.approx(bench.SMS * 128 * 2000e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["attempts_per_s_in_kernel"] == pytest.approx(attempts / t)
    smem = attempts * r["smem_bytes_per_attempt"] / t
    assert r["smem_frac"] == pytest.approx(smem / (bench.SMS * 128 * 2000e6))
    assert r["traffic"] == bench.SWEEP_TRAFFIC.get(("k_sweep_msc+pair", 256))
    packed = bench.sweep_roofline(stats, attempts, {}, ("k_sweep_packed", 128), 12.0, 0.06)
    assert packed["traffic"] == bench.SWEEP_TRAFFIC[("k_sweep_packed", 128)]
    # a kernel with no ncu capture reports no traffic; no launches, no line
    assert bench.sweep_roofline(stats, attempts, {}, ("k_sweep", 512), 12.0, 0.06)["traffic"] is None
    assert bench.sweep_roofline({"sweep_ms": 0.0, "sweep_launches": 0}, attempts, {}, ("k_sweep", 512), 12.0, 0.06) is None


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
