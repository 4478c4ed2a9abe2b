"""Host-side arithmetic of bench.py (CPU only): the ray-sample counts the
throughput is quoted in, the roofline report built from per-(kernel, level)
event times, and the gate that keeps DRAM counters of an older kernel source
out of the report."""
import json
import math

import numpy as np
import pytest

import bench
from paper_2412_10249_gb300 import inputs


def test_samples_per_iteration_is_two_m_n_ell():
    # one forward and one back-projection of the drawn level, each m rays x
    # N_ell lines (the per-level cost linear in the grid side, Sec. 4.1)
    p = inputs.fan512_problem()
    got = bench.samples_per_iteration(p, [0, 1, 2, 3, 0])
    want = [2 * 720 * 768 * (512 >> l) for l in (0, 1, 2, 3, 0)]
    np.testing.assert_array_equal(got, want)


def test_expected_samples_per_solve_uniform_levels():
    p = inputs.fan512_problem()
    # uniform p over r = 4 levels: 2 m N (1 + 1/2 + 1/4 + 1/8) / 4 per iteration
    want = 500 * 2 * 720 * 768 * 512 * (1 + 0.5 + 0.25 + 0.125) / 4
    assert bench.expected_samples_per_solve(p, 500) == pytest.approx(want, rel=1e-15)
    # and it is the mean of the exact per-iteration counts over a long stream
    lv = np.random.default_rng(0).integers(0, 4, 400000)
    mean = bench.samples_per_iteration(p, lv).mean() * 500
    assert mean == pytest.approx(want, rel=5e-3)


def _prof(kind_level_ms_cnt):
    ms = [0.0] * 24
    cnt = [0] * 24
    for (kind, lvl), (t, c) in kind_level_ms_cnt.items():
        ms[kind * 8 + lvl] = t
        cnt[kind * 8 + lvl] = c
    return ms, cnt


def test_roofline_report_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "_dram_traffic", lambda kname, level: 1234)
    p = inputs.fan512_problem()
    # back-projector level 0 dominates: 10 launches of 0.25 ms
    ms, cnt = _prof({(1, 0): (2.5, 10), (0, 0): (1.3, 10), (2, 1): (0.2, 12)})
    rep = bench.roofline_report(p, ms, cnt, 80.0, period=32, smem_probe=(39000.0, 39500.0))
    avg_s = 0.25e-3
    samples = 720 * 768 * 512
    assert rep["bound"] == "alu" and rep["unit"] == "TFLOP/s"
    assert rep["avg_launch_us"] == pytest.approx(250.0)
    assert rep["achieved"] == pytest.approx(samples * 7.0 / avg_s / 1e12)
    assert rep["frac"] == pytest.approx(rep["achieved"] / 80.0)
    assert rep["traffic"] == 1234
    assert rep["gsamples_per_s"] == pytest.approx(samples / avg_s / 1e9)
    sm = rep["smem"]
    assert sm["achieved_gbs"] == pytest.approx(samples * 17.0 / avg_s / 1e9)
    assert sm["measured_peak_gbs"] == 39500.0     # read-modify-write ceiling for k_bp
    assert sm["measured_frac"] == pytest.approx(sm["achieved_gbs"] / 39500.0)
    # shares add up to one; per-level averages are time / count
    assert sum(rep["time_share"].values()) == pytest.approx(1.0, abs=1e-3)
    av = rep["avg_launch_us_by_level"]
    assert av["back-projector l0"] == pytest.approx(250.0)
    assert av["forward projector l0"] == pytest.approx(130.0)
    assert av["primal update l1"] == pytest.approx(0.2 / 12 * 1e3, abs=0.05)
    assert "forward projector l1" not in av


def test_roofline_report_projector_uses_the_load_ceiling(monkeypatch):
    monkeypatch.setattr(bench, "_dram_traffic", lambda kname, level: None)
    p = inputs.fan512_problem()
    ms, cnt = _prof({(0, 2): (5.0, 100), (1, 0): (1.0, 4)})
    rep = bench.roofline_report(p, ms, cnt, 80.0, smem_probe=(39000.0, 39500.0))
    assert rep["kernel"].startswith("forward projector (k_fp) at level 2 (128x128 grid)")
    samples = 720 * 768 * 128
    assert rep["achieved"] == pytest.approx(samples * 6.0 / 50e-6 / 1e12)
    assert rep["smem"]["measured_peak_gbs"] == 39000.0
    assert rep["traffic"] is None


def test_dram_counters_are_gated_by_the_kernel_source(monkeypatch, tmp_path):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "roofline_counters.json").write_text(json.dumps(
        {"kernels_cu_sha256_prefix": "abc", "k_bp": {"0": {"dram_bytes_per_launch": 77}}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernels_sha", lambda: "abc")
    assert bench._dram_traffic("k_bp", 0) == 77
    assert bench._dram_traffic("k_bp", 1) is None
    monkeypatch.setattr(bench, "_kernels_sha", lambda: "def")
    assert bench._dram_traffic("k_bp", 0) is None


def test_committed_counters_name_a_kernel_source():
    with open(f"{bench.ROOT}/profiles/roofline_counters.json") as f:
        c = json.load(f)
    assert len(c["kernels_cu_sha256_prefix"]) == 16
    for k in ("k_bp", "k_fp"):
        b = c[k]["0"]["dram_bytes_per_launch"]
        # a level-0 launch reads the ray list and the sinogram once: tens of MB
        assert 1e6 < b < 1e8 and math.isfinite(b)


def test_smem_peak_is_the_unit_count_times_clock():
    assert bench.SMEM_PEAK_GBS == pytest.approx(152 * 128 * 2.07e9 / 1e9)
