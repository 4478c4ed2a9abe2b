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


DEV = {"n_sm": 152, "max_mhz": 2070.0}


def test_roofline_report_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "_dram_traffic",
                        lambda kname, level, field="dram_bytes_per_launch":
                        1234 if field == "dram_bytes_per_launch" else 99)
    p = inputs.fan512_problem()
    # back-projector level 0 dominates: 10 launches of 0.25 ms
    ms, cnt = _prof({(1, 0): (2.5, 10), (0, 0): (1.3, 10), (2, 1): (0.2, 12)})
    rep = bench.roofline_report(p, ms, cnt, DEV, period=32, smem_probe=(39000.0, 39500.0),
                                l2_gbs=7900.0, hbm_gbs=6677.0)
    avg_s = 0.25e-3
    samples = 720 * 768 * 512
    # the shared-memory measure: 8 bytes (two 4-byte accesses) per sample
    # against the measured load ceiling
    assert rep["bound"] == "smem" and rep["unit"] == "GB/s"
    assert rep["avg_launch_us"] == pytest.approx(250.0)
    assert rep["achieved"] == pytest.approx(samples * 8.0 / avg_s / 1e9)
    assert rep["peak"] == 39000.0
    assert rep["frac"] == pytest.approx(rep["achieved"] / 39000.0)
    assert rep["traffic"] == 1234
    alg = 4.0 * (720 * 768 + 512 * 512)          # y in, image out
    assert rep["algorithmic_dram_bytes"] == pytest.approx(alg)
    assert rep["traffic_over_algorithmic"] == pytest.approx(1234 / alg)
    assert rep["traffic_in_solve"] == 99
    assert rep["gsamples_per_s"] == pytest.approx(samples / avg_s / 1e9)
    alu = rep["alu_view"]
    assert alu["achieved_tflops"] == pytest.approx(samples * 7.0 / avg_s / 1e12)
    assert alu["peak_tflops"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert rep["smem_derived_peak_gbs"] == pytest.approx(152 * 128 * 2.07e9 / 1e9)
    # the memory view lists every timed (kernel, level) on its algorithmic bytes
    mv = {(v["kernel"], v["level"]): v for v in rep["memory_view"]["launches"]}
    fp0 = mv[("k_fp", 0)]
    assert fp0["algorithmic_bytes"] == pytest.approx(4.0 * (512 * 512 + 7 * 720 * 768))
    assert fp0["achieved_gbs"] == pytest.approx(fp0["algorithmic_bytes"] / 0.13e-3 / 1e9)
    assert fp0["frac_of_l2_copy"] == pytest.approx(fp0["achieved_gbs"] / 7900.0)
    assert fp0["frac_of_hbm"] == pytest.approx(fp0["achieved_gbs"] / 6677.0)
    # shares add up to one; per-level averages are time / count
    assert sum(rep["time_share"].values()) == pytest.approx(1.0, abs=1e-3)
    av = rep["avg_launch_us_by_level"]
    assert av["back-projector l0"] == pytest.approx(250.0)
    assert av["forward projector l0"] == pytest.approx(130.0)
    assert av["primal update l1"] == pytest.approx(0.2 / 12 * 1e3, abs=0.05)
    assert "forward projector l1" not in av


def test_roofline_report_projector_at_a_coarse_level(monkeypatch):
    monkeypatch.setattr(bench, "_dram_traffic", lambda kname, level, field=None: None)
    p = inputs.fan512_problem()
    ms, cnt = _prof({(0, 2): (5.0, 100), (1, 0): (1.0, 4)})
    dev = {"n_sm": 148, "max_mhz": 1965.0}
    rep = bench.roofline_report(p, ms, cnt, dev)
    assert rep["kernel"].startswith("forward projector (k_fp) at level 2 (128x128 grid)")
    samples = 720 * 768 * 128
    # no probe: the derived ceiling from the device's own unit count and clock
    assert rep["peak"] == pytest.approx(148 * 128 * 1965e6 / 1e9)
    assert rep["achieved"] == pytest.approx(samples * 8.0 / 50e-6 / 1e9)
    assert rep["alu_view"]["achieved_tflops"] == pytest.approx(samples * 6.0 / 50e-6 / 1e12)
    assert rep["traffic"] is None and rep["traffic_over_algorithmic"] is None
    assert rep["memory_view"]["l2_copy_gbs"] is None


def test_update_algorithmic_bytes():
    p = inputs.fan512_problem()
    d = 512 * 512
    nxt = 2 * sum((512 >> l) ** 2 for l in range(4)) / 4
    assert bench.algorithmic_dram_bytes(p, 2, 0) == pytest.approx(4 * (d + 4 * d + 2 * d + nxt))
    assert bench.algorithmic_dram_bytes(p, 2, 2) == pytest.approx(
        4 * (128 * 128 + 4 * d + 2 * 128 * 128 + nxt))


def test_device_units_fall_back_to_the_clock_record():
    assert bench.device_units(None, {"sm_max_mhz": 1900.0}) == {"n_sm": 152, "max_mhz": 1900.0}


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


def test_cpu_description_names_the_host():
    h = bench.cpu_description()
    assert h["nproc"] >= 1 and isinstance(h["cpu_model"], str) and h["cpu_model"]


def test_oracle_pool_runs_independent_processes(oracle_lib):
    # two spawned oracle processes, one iteration each on a small fan problem:
    # the wall time covers both and the samples are the sum of both streams
    p = inputs.Problem(n=16, n_angles=12, n_det=24, geometry=1, angle_span=2 * math.pi,
                       levels=2)
    _, b, _ = inputs.measurements(p, seed=0, noise="none")
    params = dict(p.params(), mu=0.5, sigma=0.05)
    pool = bench.OraclePool(2)
    try:
        wall, samples = pool.run(p, params, b.ravel(), 0, 3)
    finally:
        pool.close()
    per_run = [bench.samples_per_iteration(p, oracle_lib.Oracle(**params).run(b.ravel(), s, 3)[1])
               .sum() for s in (0, 1)]
    assert samples == pytest.approx(sum(per_run))
    assert wall > 0


def test_both_arms_name_the_same_workload_config():
    # the GPU arm and the reference arm print one `config` object built from
    # the arguments alone (device-chosen values go to the GPU line's `plan`)
    args = bench.parse_args([])
    p = inputs.fan512_problem()
    a, b = bench.workload_config(p, args, 1), bench.workload_config(p, args, 1)
    assert a == b and a["workload"] == bench.WORKLOAD
    assert not {"mu", "sigma", "theta", "bp_view_groups", "fp_strip_lines"} & set(a)
    json.dumps(a)
