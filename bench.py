"""Throughput benchmark of the ImaSk hot path on the 512x512 fan-beam workload.

Workload (one "step" = one whole ImaSk solve): 512x512 random-ellipse phantom,
fan beam with 720 views over 2 pi and 768 bins, source 2W and detector 1W from
the centre, Poisson counts with I0 = 1e4 then log-transformed, four levels
(512/256/128/64) drawn uniformly, quadratic regulariser with mu and sigma
chosen by the plan (power method + Thm. 3), 500 iterations of Alg. 1.

Our arm: each step solves from b resident in HBM (seed = step index) through
the C ABI (imask_solve).  Per-step device time comes from CUDA events on the
solve's stream; L2 is flushed (a 512 MB write) between steps, outside the
events.  ``e2e`` repeats the steps with the measurement vector in pinned host
memory: H2D copy of b, the solve, D2H copy of x, all inside the timed region.

Reference arm (--impl reference): the FP64 CPU oracle, as it stands, on a
bounded sample of the same workload (a few Alg. 1 iterations per step),
converted to solves/s through the ray-samples it processed.

Under torchrun (N > 1) every rank runs its own replica of the workload (no
collective on the data path; "scaling": "weak"); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2412_10249_gb300 import inputs  # noqa: E402

METRIC = "ImaSk solves/sec & Gray-samples/s at rel.err≤1e-3 vs plain FP32 form; p99 ms"
WORKLOAD = "fan512: 512x512 fan beam 720x768, r=4 uniform, K=500, quadratic R"
ITERS = 500


def samples_per_iteration(p: inputs.Problem, levels) -> np.ndarray:
    """Joseph samples (forward + back) of each iteration: 2 m N_ell."""
    lv = np.asarray(levels)
    return 2.0 * p.m * (p.n >> lv)


def expected_samples_per_solve(p: inputs.Problem, iters: int = ITERS) -> float:
    pr = np.full(p.levels, 1.0 / p.levels) if p.probs is None else np.asarray(p.probs)
    return iters * 2.0 * p.m * sum(pr[l] * (p.n >> l) for l in range(p.levels))


# ---------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [s.strip() for s in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return float("nan")

        sm = np.array([num(r[1]) for r in rows])
        mx = np.array([num(r[2]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": float(np.nanmedian(sm)), "sm_max_mhz": float(np.nanmax(mx)),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------
# distributed plumbing (replicas)
# ---------------------------------------------------------------------------------
def dist_setup(use_cuda: bool):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if use_cuda else "gloo")
    return world, rank, local


def dist_max(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_sum(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def dist_barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------------
# reference arm: the FP64 oracle on host cores
# ---------------------------------------------------------------------------------
def oracle_sample(p: inputs.Problem, params: dict, b: np.ndarray, seed: int, iters: int,
                  want_x: bool = False):
    """Runs `iters` oracle iterations of the workload; returns (seconds,
    samples) and, with want_x, the oracle's iterate."""
    from oracle import Oracle
    o = Oracle(**params)
    t0 = time.perf_counter()
    st, lv = o.run(b, seed, iters)
    dt = time.perf_counter() - t0
    if want_x:
        return dt, float(samples_per_iteration(p, lv).sum()), st["x"]
    return dt, float(samples_per_iteration(p, lv).sum())


def cpu_description() -> dict:
    """Host core count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    import platform
    return {"nproc": os.cpu_count() or 1, "cpu_model": model or platform.machine()}


def _oracle_worker(job):
    """One oracle process's share: `iters` iterations from seed `seed`;
    returns (seconds, level stream)."""
    params, b, seed, iters = job
    from oracle import Oracle
    o = Oracle(**params)
    t0 = time.perf_counter()
    _, lv = o.run(b, seed, iters)
    return time.perf_counter() - t0, np.asarray(lv)


class OraclePool:
    """Independent, unmodified oracle processes, one per host core (spawned,
    so that no CUDA state is inherited), each running its own seed: the
    oracle on all host cores without changing it."""

    def __init__(self, cores: int):
        import multiprocessing as mp
        self.cores = max(1, int(cores))
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
        os.environ["OMP_NUM_THREADS"] = "1"
        os.environ["OPENBLAS_NUM_THREADS"] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.cores)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run(self, p: inputs.Problem, params: dict, b: np.ndarray, seed0: int, iters: int):
        """All cores at once, `iters` iterations each; returns (wall seconds,
        total ray-samples)."""
        jobs = [(params, b, seed0 + k, iters) for k in range(self.cores)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, jobs, chunksize=1)
        wall = time.perf_counter() - t0
        return wall, float(sum(samples_per_iteration(p, lv).sum() for _, lv in res))

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    world, rank, _ = dist_setup(False)
    if rank != 0:
        return 0
    p = inputs.fan512_problem()
    _, b, _ = inputs.measurements(p, seed=0)
    # the oracle needs mu and sigma: fixed values close to those the GPU plan
    # derives for this workload (its cost per iteration does not depend on them)
    params = dict(p.params(), mu=args.mu, sigma=args.sigma)
    per_solve = expected_samples_per_solve(p)
    host = cpu_description()
    pool = OraclePool(host["nproc"])
    try:
        for w in range(args.warmup):
            pool.run(p, params, b.ravel(), 1000 + 100 * w, args.ref_iters)
        times, samples = [], []
        for k in range(args.steps):
            dt, sm = pool.run(p, params, b.ravel(), 100 * k, args.ref_iters)
            times.append(dt)
            samples.append(sm)
    finally:
        pool.close()
    T, S = sum(times), sum(samples)
    gs = S / T / 1e9
    solves = S / per_solve / T
    line = {
        "impl": "reference", "metric": METRIC, "value": solves, "unit": "solves/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(p, args, world),
        "gsamples_per_s": gs,
        "cpu_baseline": {"value": solves, "unit": "solves/s", "cores": pool.cores,
                         "kind": "oracle", "cpu_model": host["cpu_model"],
                         "nproc": host["nproc"],
                         "sample": f"per step, {pool.cores} independent oracle processes (one "
                                   f"per host core, seeds differ), {args.ref_iters} iterations "
                                   f"of the fan512 solve each, wall time of the step; "
                                   f"extrapolated by ray-samples to {ITERS}-iteration solves"},
        "e2e": {"value": solves, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------
# roofline
# ---------------------------------------------------------------------------------
KINDS = ["forward projector (k_fp)", "back-projector (k_bp)", "primal update (k_update)"]
KNAMES = ["k_fp", "k_bp", "k_update"]
# algorithmic work per (ray, line) sample: FP32 flops, and the shared-memory
# bytes of the method (two 4-byte pixel accesses: the projector's two loads,
# the back-projector's two accumulations)
FLOPS_PER_SAMPLE = {0: 6.0, 1: 7.0}          # q FMA 2, f 1, lerp 3 | q 2, f 1, weights 2, adds 2
SMEM_BYTES_PER_SAMPLE = 8.0


def device_units(torch=None, clocks=None) -> dict:
    """SM count of the current device and its maximum SM clock (from the clock
    record of the run, else the driver's measurement file, else 2070 MHz)."""
    n_sm = None
    if torch is not None:
        try:
            n_sm = int(torch.cuda.get_device_properties(torch.cuda.current_device())
                       .multi_processor_count)
        except Exception:
            n_sm = None
    mhz = (clocks or {}).get("sm_max_mhz") or measured_peaks().get("sm_max_mhz") or 2070.0
    return {"n_sm": n_sm or 152, "max_mhz": float(mhz)}


def algorithmic_dram_bytes(p: inputs.Problem, kind: int, lvl: int) -> float:
    """Bytes a launch must move at least (each input read once, each output
    written once), fp32: projector with its dual epilogue: the sketch image and
    y in, b, psi_l in / out, psi_mean in / out, y out (7 m); back-projector: y
    in, the level image out; update: the back-projector's image, x, phi_mean
    and the level's table in / out, and the next level's sketch in its two
    layouts (expected over the level draw)."""
    nl = p.n >> lvl
    d, m = p.n * p.n, p.m
    pr = np.full(p.levels, 1.0 / p.levels) if p.probs is None else np.asarray(p.probs)
    if kind == 0:
        return 4.0 * (nl * nl + 7 * m)
    if kind == 1:
        return 4.0 * (m + nl * nl)
    nxt = 2.0 * sum(pr[l] * (p.n >> l) ** 2 for l in range(p.levels))
    table = 2.0 * d if lvl == 0 else 2.0 * nl * nl
    return 4.0 * (nl * nl + 4 * d + table + nxt)


def roofline_report(p, prof_ms, prof_cnt, dev, period=1, smem_probe=None, l2_gbs=None,
                    hbm_gbs=None):
    """Dominant (kernel, level) by total event time.  The projectors bind on
    the on-chip shared-memory pipe (Sec. 4.1 workload: hundreds of millions of
    samples against tens of MB of state): achieved = samples x 8 B per launch
    / average launch time against the measured shared-memory load ceiling.
    The FP32-ALU view is kept beside it, and every (kernel, level) is also
    put against the measured L2 copy and HBM bandwidth on its algorithmic
    DRAM bytes (the memory view, the measure for the fused epilogues and the
    coarse levels)."""
    best = int(np.argmax(prof_ms))
    kind, lvl = best // 8, best % 8
    cnt = max(1, prof_cnt[best])
    avg_s = prof_ms[best] / cnt / 1e3
    nl = p.n >> lvl
    samples_launch = p.m * nl
    n_sm, clk = dev["n_sm"], dev["max_mhz"] * 1e6
    smem_derived = n_sm * 128 * clk / 1e9
    alu_peak = n_sm * 128 * 2 * clk / 1e12
    alg_dram = algorithmic_dram_bytes(p, kind, lvl)
    traffic = _dram_traffic(KNAMES[kind], lvl)
    rep = {"kernel": f"{KINDS[kind]} at level {lvl} ({nl}x{nl} grid)",
           "avg_launch_us": avg_s * 1e6, "launches": int(prof_cnt[best]),
           "timed_launches": f"CUDA events around the launches of every {period}-th iteration "
                             f"inside the timed region",
           "gsamples_per_s": samples_launch / avg_s / 1e9,
           "traffic": traffic, "algorithmic_dram_bytes": alg_dram,
           "traffic_over_algorithmic": (traffic / alg_dram) if traffic else None,
           "traffic_in_solve": _dram_traffic(KNAMES[kind], lvl, "dram_bytes_per_launch_in_solve"),
           "device": {"n_sm": n_sm, "max_sm_mhz": dev["max_mhz"]}}
    if kind in FLOPS_PER_SAMPLE:
        ach = samples_launch * SMEM_BYTES_PER_SAMPLE / avg_s / 1e9
        if smem_probe is not None:
            peak, src = float(smem_probe[0]), ("measured here: conflict-free 32-bit shared-memory "
                                                "loads on every SM (imask_probe_smem)")
        else:
            peak, src = smem_derived, f"derived: {n_sm} SMs x 128 B x {dev['max_mhz']:.0f} MHz"
        flops = samples_launch * FLOPS_PER_SAMPLE[kind] / avg_s / 1e12
        rep.update(bound="smem", unit="GB/s", achieved=ach, peak=peak, peak_source=src,
                   frac=ach / peak,
                   algorithmic={"samples_per_launch": samples_launch,
                                "smem_bytes_per_sample": SMEM_BYTES_PER_SAMPLE,
                                "flops_per_sample": FLOPS_PER_SAMPLE[kind]},
                   smem_derived_peak_gbs=smem_derived,
                   alu_view={"achieved_tflops": flops, "peak_tflops": alu_peak,
                             "peak_source": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 flop x "
                                            f"{dev['max_mhz']:.0f} MHz",
                             "frac": flops / alu_peak})
    else:
        ach = alg_dram / avg_s / 1e9
        peak = l2_gbs or hbm_gbs
        rep.update(bound="hbm", unit="GB/s", achieved=ach, peak=peak,
                   peak_source="measured L2 copy" if l2_gbs else "measured HBM copy",
                   frac=(ach / peak) if peak else None)
    views = []
    for k in range(24):
        if prof_cnt[k] <= 0:
            continue
        kd, lv = k // 8, k % 8
        a_s = prof_ms[k] / prof_cnt[k] / 1e3
        by = algorithmic_dram_bytes(p, kd, lv)
        gbs = by / a_s / 1e9
        views.append({"kernel": KNAMES[kd], "level": lv, "avg_us": round(a_s * 1e6, 2),
                      "algorithmic_bytes": by, "achieved_gbs": gbs,
                      "frac_of_l2_copy": (gbs / l2_gbs) if l2_gbs else None,
                      "frac_of_hbm": (gbs / hbm_gbs) if hbm_gbs else None})
    rep["memory_view"] = {"l2_copy_gbs": l2_gbs, "hbm_gbs": hbm_gbs, "launches": views}
    total = max(1e-12, float(sum(prof_ms)))
    rep["time_share"] = {f"{KINDS[k // 8].split(' (')[0]} l{k % 8}": round(prof_ms[k] / total, 4)
                         for k in range(24) if prof_cnt[k] > 0}
    rep["avg_launch_us_by_level"] = {
        f"{KINDS[k // 8].split(' (')[0]} l{k % 8}": round(prof_ms[k] / prof_cnt[k] * 1e3, 1)
        for k in range(24) if prof_cnt[k] > 0}
    return rep


def _kernels_sha() -> str:
    import hashlib
    path = os.path.join(ROOT, "paper_2412_10249_gb300", "csrc", "kernels.cu")
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _dram_traffic(kname: str, level: int, field: str = "dram_bytes_per_launch"):
    """DRAM bytes per launch from the committed ncu summary (cold caches, or
    with field "dram_bytes_per_launch_in_solve" the same launch in a solve with
    the caches as the solve left them), if it still describes the current
    kernel source (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "roofline_counters.json")) as f:
            c = json.load(f)
        if c.get("kernels_cu_sha256_prefix") != _kernels_sha():
            return None
        return c[kname][str(level)][field]
    except (OSError, KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def l2_copy_gbs(torch, stream, mib: int = 32, reps: int = 20) -> float:
    """Read + write bandwidth of a device-to-device copy of a buffer that fits
    in L2 (the ceiling for the solve state, which stays L2-resident)."""
    a = torch.ones(mib * 1024 * 1024 // 4, device="cuda")
    b = torch.empty_like(a)
    best = 0.0
    with torch.cuda.stream(stream):
        for _ in range(3):
            b.copy_(a)
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                b.copy_(a)
            e1.record(stream)
            e1.synchronize()
            best = max(best, 2.0 * a.numel() * 4 * reps / (e0.elapsed_time(e1) / 1e3) / 1e9)
    return best


# ---------------------------------------------------------------------------------
# iteration variants (Alg. 7, snapshot tables, independent draws)
# ---------------------------------------------------------------------------------
def variant_params(variant: str, dual_tables: int, draws: int) -> dict:
    return {"variant": 1 if variant == "seq" else 0, "theta": 1.0,
            "dual_tables": int(dual_tables), "draws": int(draws)}


L2_NOTE = ("GPU arm: L2 flushed between steps (512 MB write outside the step events); "
           "CPU reference arm: no flush (FP64 oracle processes)")


def workload_config(p, args, world: int) -> dict:
    """The `config` object of the JSON line: what the workload is, the same for
    the GPU arm and the reference arm (what a plan chooses on the device, its
    step sizes and tuned splits, goes to the line's `plan` object)."""
    return {"workload": WORKLOAD, "n": p.n, "views": p.n_angles, "bins": p.n_det,
            "levels": p.levels, "iters_per_solve": args.iters,
            "iteration": dict(variant_params(args.variant, args.dual_tables, args.draws),
                              autotune=args.autotune),
            "l2": L2_NOTE, "parallelism": f"replicas x{world}"}


VARIANT_SET = {
    "alg7_seq": ("seq", 0, 0, {}),
    "snapshot_tables": ("alg1", 1, 0, {}),
    "independent_draws": ("alg1", 0, 1, {}),
    "alg7_seq_snapshot_tables": ("seq", 1, 0, {}),
    # TV with nonnegativity (Sec. 4.5), prox by 20 dual-FISTA steps
    "tv_nonneg": ("alg1", 0, 0, {"reg": 2, "tv_inner": 20}),
    # back-projector split measured at plan time instead of the occupancy rule
    "autotuned_plan": ("alg1", 0, 0, {"autotune": 1}),
}


def parallel512_problem():
    """The paper's own geometry at the headline size: 512 x 512, parallel beam,
    720 views over 180 degrees, ceil(sqrt(2) 512) = 725 bins at the pixel
    pitch, r = 4 uniform levels."""
    return inputs.Problem(n=512, n_angles=720, n_det=725, geometry=0, angle_span=math.pi,
                          levels=4, reg=0, mu=1.0)


def time_parallel_backprojectors(imask, iters, stream, flush, steps=3, period=16):
    """Parallel-beam solves with the owner-computes and the pixel-driven
    back-projector (bp_gather), and with the form the plan picks by timing
    both (bp_gather = -1): solves/s, the back-projector's average launch per
    level (CUDA events on every `period`-th iteration) and the distance
    between the two forms' results after `iters` iterations."""
    import torch
    p = parallel512_problem()
    _, b, _ = inputs.measurements(p, seed=0)
    bt = torch.as_tensor(b.ravel().astype(np.float32), device="cuda")
    out, xs, mu, sigma = {}, {}, 0.0, 0.0
    for name, gather in (("owner_scatter", 0), ("pixel_gather", 1), ("chosen_at_plan_time", -1)):
        plan = imask.Plan(dict(p.params(), mu=mu, sigma=sigma, autotune=1, bp_gather=gather))
        mu, sigma = plan.info["mu"], plan.info["sigma"]
        x = torch.empty(p.d, device="cuda", dtype=torch.float32)
        with torch.cuda.stream(stream):
            plan.solve(bt, 777, iters, out=x, stream=stream)
        stream.synchronize()
        imask.imask_profile_read(reset=True)
        imask.imask_profile_enable(period)
        ms = []
        for k in range(steps):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                a.record(stream)
                plan.solve(bt, 5000 + k, iters, out=x, stream=stream)
                e.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(e))
        imask.imask_profile_enable(False)
        pms, pcnt = imask.imask_profile_read(reset=True)
        plan.check()
        bp_us = {f"l{l}": round(1e3 * pms[8 + l] / pcnt[8 + l], 1)
                 for l in range(p.levels) if pcnt[8 + l] > 0}
        out[name] = {"solves_per_s": 1e3 * steps / float(sum(ms)),
                     "back_projector_us_by_level": bp_us,
                     "bp_view_groups": list(plan.info["bp_view_groups"][:p.levels]),
                     "form": "pixel_gather" if plan.info["bp_gather"] else "owner_scatter"}
        xs[name] = x.double().cpu().numpy()
        plan.close()
    out["rel_diff_x"] = float(np.linalg.norm(xs["pixel_gather"] - xs["owner_scatter"]) /
                              np.linalg.norm(xs["owner_scatter"]))
    out["speedup"] = out["pixel_gather"]["solves_per_s"] / out["owner_scatter"]["solves_per_s"]
    out["config"] = {"workload": "par512: 512x512 parallel beam 720 views over 180 deg x 725 "
                                 "bins, r=4 uniform, K=%d, quadratic R, autotuned" % iters}
    return out


def time_variants(imask, p, bt, info, iters, stream, flush, x, steps=3):
    """solves/s of each variant over `steps` solves (after one warm-up solve),
    same workload, mu and (Alg. 1) sigma; Alg. 7 takes sigma = 0.05; then the
    per-iteration time of PDHG on the same sketched problem."""
    import torch
    out = {}
    for name, (v, dt, dr, extra) in VARIANT_SET.items():
        sigma = 0.05 if v == "seq" else info["sigma"]
        if extra.get("reg") == 2:
            extra = dict(extra, tv_lambda=0.02 * info["mu"])
        plan = imask.Plan(dict(p.params(), mu=info["mu"], sigma=sigma,
                               **variant_params(v, dt, dr), **extra))
        with torch.cuda.stream(stream):
            plan.solve(bt, 777, iters, out=x, stream=stream)
        ms = []
        for k in range(steps):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
                a.record(stream)
                plan.solve(bt, 5000 + k, iters, out=x, stream=stream)
                e.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(e))
        plan.check()
        out[name] = {"solves_per_s": 1e3 * steps / float(sum(ms)), "sigma": sigma,
                     "ms_per_solve": float(np.mean(ms))}
        plan.close()
    # PDHG (every level's K and K^T per iteration), printed parameters
    plan = imask.Plan(dict(p.params(), mu=info["mu"], sigma=info["sigma"]))
    s_, t_, th_ = imask.imask_pdhg_params(info["L"] * math.sqrt(info["mu"]), info["mu"], 0.99)
    n_it = 20
    with torch.cuda.stream(stream):
        plan.pdhg(bt, 2, s_, t_, th_, out=x, stream=stream)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.pdhg(bt, n_it, s_, t_, th_, out=x, stream=stream)
        e.record(stream)
    torch.cuda.synchronize()
    out["pdhg"] = {"ms_per_iteration": a.elapsed_time(e) / n_it, "s": s_, "t": t_,
                   "theta": th_, "note": "includes the per-call work-buffer allocation"}
    plan.close()
    # the 64x64 parallel-beam workload with quadratic + smoothed TV (two levels,
    # 50 iterations; the parity case run against the oracle by the tests)
    sp = inputs.small_problem()
    _, sb, _ = inputs.measurements(sp, seed=0)
    sbt = torch.as_tensor(sb.ravel().astype(np.float32), device="cuda")
    splan = imask.Plan(dict(sp.params(), mu=0.0, sigma=0.0))
    sinfo = splan.info
    splan.close()
    splan = imask.Plan(dict(sp.params(), mu=sinfo["mu"], sigma=sinfo["sigma"],
                            tv_lambda=0.1 * sinfo["mu"]))
    xs = torch.empty(sp.n * sp.n, device="cuda")
    with torch.cuda.stream(stream):
        splan.solve(sbt, 1, 50, out=xs, stream=stream)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for k in range(20):
            splan.solve(sbt, 2 + k, 50, out=xs, stream=stream)
        e.record(stream)
    torch.cuda.synchronize()
    out["small_tv64"] = {"solves_per_s": 20e3 / a.elapsed_time(e),
                         "ms_per_solve": a.elapsed_time(e) / 20,
                         "workload": "64x64 parallel 60x92, r=2, quadratic + smoothed TV, 50 its"}
    splan.close()
    return out


def cg_fixed_point(plan, p, b, mu, iters=150):
    """x_nat = argmin 1/2|Kbar x - b|^2 + mu/2|x|^2 (eq. min_obj_new), Kbar =
    sum_l p_l K_l, by conjugate gradients on the normal equations; operator
    applications through the library (FP32), vectors in FP64."""
    import torch
    pr = np.asarray(p.probs if p.probs is not None else [1.0 / p.levels] * p.levels)

    def apply_K(v):
        v32 = v.float()
        acc = torch.zeros(p.m, dtype=torch.float64, device=v.device)
        for ell in range(p.levels):
            acc += pr[ell] * plan.project(ell, v32).double()
        return acc

    def apply_KT(w):
        w32 = w.float()
        acc = torch.zeros(p.d, dtype=torch.float64, device=w.device)
        for ell in range(p.levels):
            acc += pr[ell] * plan.backproject(ell, w32).double()
        return acc

    def normal(v):
        return apply_KT(apply_K(v)) + mu * v

    bb = b.double()
    rhs = apply_KT(bb)
    xk = torch.zeros_like(rhs)
    r = rhs.clone()
    d = r.clone()
    rr = float(r @ r)
    r0 = math.sqrt(rr)
    for _ in range(iters):
        q = normal(d)
        a = rr / float(d @ q)
        xk += a * d
        r -= a * q
        rn = float(r @ r)
        if math.sqrt(rn) < 1e-9 * r0:
            break
        d = r + (rn / rr) * d
        rr = rn
    return xk.float(), math.sqrt(rr) / r0


def run_ablation(args):
    """Step-size ablation (sigma*/2, sigma*, sigma_B of Sec. 3.6) and Alg. 7 on
    the fan512 workload: squared relative distance |x^k - x_nat|^2 / |x_nat|^2
    to the fixed point after K iterations (the paper's convergence measure),
    mean over seeds."""
    import torch
    from paper_2412_10249_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2412_10249_gb300 import imask
    p = inputs.fan512_problem()
    _, b, _ = inputs.measurements(p, seed=0)
    bt = torch.as_tensor(b.ravel().astype(np.float32), device="cuda")
    base = imask.Plan(dict(p.params(), mu=0.0, sigma=0.0))
    info = base.info
    mu = info["mu"]
    xnat, cg_res = cg_fixed_point(base, p, bt, mu)
    sig_star = info["sigma"]
    sig_b = 1.0 / (info["L"] ** 2 + 3.0 * info["Lbar"] ** 2)
    runs = {"alg1_sigma_star_half": dict(sigma=0.5 * sig_star),
            "alg1_sigma_star": dict(sigma=sig_star),
            "alg1_sigma_B": dict(sigma=sig_b),
            "alg7_seq_sigma_0.05_theta_1": dict(sigma=0.05, variant=1, theta=1.0)}
    marks = [50, 100, 200, 500, 1000, 2000]
    res = {}
    for name, extra in runs.items():
        plan = imask.Plan(dict(p.params(), mu=mu, **extra))
        dist = np.zeros(len(marks))
        for seed in range(args.ablation_seeds):
            s = plan.state(bt, seed)
            done = 0
            for i, k in enumerate(marks):
                s.step(k - done)
                done = k
                dist[i] += imask.imask_rel_distance(s.get(s.X), xnat)   # squared
            s.close()
        plan.close()
        res[name] = {"sigma": extra["sigma"],
                     "rel_dist_sq": {str(k): float(v / args.ablation_seeds)
                                  for k, v in zip(marks, dist)}}
    line = {"ablation": "step size and variant, fan512", "mu": mu, "sigma_star": sig_star,
            "theta_star": info["theta"], "sigma_B": sig_b, "L": info["L"], "Lbar": info["Lbar"],
            "Lbar_p": info["Lbar_p"], "cg_rel_residual": cg_res, "seeds": args.ablation_seeds,
            "runs": res}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------
# batched solves (mixed slice sizes) through captured CUDA graphs
# ---------------------------------------------------------------------------------
def _sinogram_job(args):
    p, seed = args
    return inputs.sinogram(p, seed).ravel().astype(np.float32)


def batch_sigma():
    """Thm. 3 step for the normalised constants every slice shares (mu chosen so
    that L = 2.46; uniform 4 levels give Lbar = L/2, Lbar_p = L)."""
    from paper_2412_10249_gb300 import imask
    return imask.imask_optimal_step(2.46, 1.23, 2.46, 0.25)[0]


def run_batch(args):
    """Mixed-size slices (side 256..1024, 180..1440 views, 1.5x side bins, fan
    beam, 4 levels, 500 iterations, quadratic R): every slice solved one after
    the other with plain launches, then all slices at once as one batch
    (graph-captured pairs of iterations, one branch per slice)."""
    import multiprocessing as mp
    probs = inputs.slice_mix(args.batch_slices, seed=0)
    # host-side inputs first, in a spawn pool (no CUDA context in the workers)
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        sinos = pool.map(_sinogram_job, [(p, 1000 + i) for i, p in enumerate(probs)])
    import torch
    from paper_2412_10249_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2412_10249_gb300 import imask
    sigma = batch_sigma()
    plans = {}
    t0 = time.perf_counter()
    for p in probs:
        key = (p.n, p.n_angles)
        if key not in plans:
            plans[key] = imask.Plan(dict(p.params(), mu=0.0, sigma=sigma))
    t_plans = time.perf_counter() - t0
    bs = [torch.as_tensor(b, device="cuda") for b in sinos]
    xs_plain = [torch.empty(p.d, device="cuda") for p in probs]
    samples = 0.0
    for i, p in enumerate(probs):
        lv = plans[(p.n, p.n_angles)].levels(i, 0, args.iters).cpu().numpy()
        samples += float(samples_per_iteration(p, lv).sum())
    stream = torch.cuda.Stream()
    # warm-up: one short solve per plan
    with torch.cuda.stream(stream):
        for key, pl in plans.items():
            b = bs[[k for k, p in enumerate(probs) if (p.n, p.n_angles) == key][0]]
            pl.solve(b, 0, 4, stream=stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with torch.cuda.stream(stream):
        e[0].record(stream)
        for i, p in enumerate(probs):
            plans[(p.n, p.n_angles)].solve(bs[i], i, args.iters, out=xs_plain[i], stream=stream)
        e[1].record(stream)
    torch.cuda.synchronize()
    forms = {}
    for name, fused in (("batched", False), ("fused", True)):
        states = [plans[(p.n, p.n_angles)].state(bs[i], i, stream=stream)
                  for i, p in enumerate(probs)]
        batch = imask.Batch(states, fused=fused)
        torch.cuda.synchronize()
        launches0 = imask.imask_launch_count()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            batch.step(args.iters, stream=stream)
            z.record(stream)
        torch.cuda.synchronize()
        launches = imask.imask_launch_count() - launches0
        t = a.elapsed_time(z) / 1e3
        worst, identical = 0.0, True
        for i, s in enumerate(states):
            xi = s.get(s.X)
            torch.cuda.synchronize()
            worst = max(worst, imask.imask_rel_distance(xi, xs_plain[i]))
            identical = identical and bool(torch.equal(xi, xs_plain[i]))
        batch.close()
        for s in states:
            s.close()
        forms[name] = {"value": len(probs) / t, "seconds": t,
                       "gsamples_per_s": samples / t / 1e9,
                       "includes": "graph capture and instantiation in the first call",
                       "gpu_launches": int(launches),
                       "max_rel_dist_sq_vs_plain": worst,
                       "bit_identical_to_plain": identical}
    clk = clocks.stop()
    t_plain = e[0].elapsed_time(e[1]) / 1e3
    oracle_err = batch_oracle_check(imask, plans, probs, sinos, args.cpu_iters)
    n = len(probs)
    line = {"metric": "batched ImaSk solves/s (mixed slice sizes)", "unit": "solves/s",
            "slices": n, "iters_per_solve": args.iters, "sigma": sigma,
            "plain": {"value": n / t_plain, "seconds": t_plain,
                      "gsamples_per_s": samples / t_plain / 1e9},
            "batched": forms["batched"], "fused": forms["fused"],
            "speedup": t_plain / forms["batched"]["seconds"],
            "speedup_fused": t_plain / forms["fused"]["seconds"],
            "rel_err_vs_fp64_oracle": oracle_err,
            "plan_setup_s": t_plans, "distinct_plans": len(plans),
            "clocks": clk,
            "config": {"workload": "mixed slices: side {256,384,512,768,1024}, views "
                                   "{180,360,720,1080,1440}, bins 1.5 x side, fan beam, r=4, "
                                   "K=500, quadratic R, mu = |K|^2/2.46^2 per plan"}}
    print(json.dumps(line))
    return 0


def batch_oracle_check(imask, plans, probs, sinos, iters, n_check=3):
    """The smallest n_check slices of a batch, advanced `iters` iterations as
    one fused batch from their timed seeds, each against the FP64 oracle on
    the same seed and iterations (relative L2 of x)."""
    import torch
    from oracle import Oracle
    idx = sorted(range(len(probs)), key=lambda i: (probs[i].n, probs[i].n_angles))[:n_check]
    states = [plans[(probs[i].n, probs[i].n_angles)].state(
        torch.as_tensor(sinos[i], device="cuda"), i) for i in idx]
    batch = imask.Batch(states, fused=True)
    batch.step(iters)
    torch.cuda.synchronize()
    out = []
    for i, s in zip(idx, states):
        p = probs[i]
        info = plans[(p.n, p.n_angles)].info
        st, _ = Oracle(**dict(p.params(), mu=info["mu"], sigma=info["sigma"])).run(
            np.asarray(sinos[i], dtype=np.float64), i, iters)
        x = s.get(s.X).double().cpu().numpy()
        out.append({"slice": i, "n": p.n, "views": p.n_angles, "iters": iters,
                    "rel_l2": float(np.linalg.norm(x - st["x"]) / np.linalg.norm(st["x"]))})
    batch.close()
    for s in states:
        s.close()
    return out


def time_mixed_precision_fan512(imask, p, bt, info, iters, stream, x_plain, n_states=8,
                                cpu_iters=8, with_oracle=True):
    """The batched 16-bit form of the headline solve: n_states states whose
    measurement-side tables are stored in binary16 / bfloat16 (fp32
    arithmetic), advanced as one graph-captured batch, with the SM clocks of
    the timed region; the first state's iterate after `iters` iterations
    against the plain fp32 form (same seed), and, after cpu_iters
    iterations, against the FP64 oracle with the same rounding and against
    the oracle's exact (fp32-table-free) iteration."""
    import torch
    out = {}
    exact = None
    if with_oracle:
        from oracle import Oracle
        _, b, _ = inputs.measurements(p, seed=0)
        o = Oracle(**dict(p.params(), mu=info["mu"], sigma=info["sigma"]))
        exact, _ = o.run(b.ravel(), 0, cpu_iters)
    for name, fmt in (("fp16_tables", 2), ("bf16_tables", 1)):
        plan = imask.Plan(dict(p.params(), mu=info["mu"], sigma=info["sigma"], storage=fmt))
        warm = [plan.state(bt, 900 + i, stream=stream) for i in range(n_states)]
        wb = imask.Batch(warm)
        wb.step(4, stream=stream)
        torch.cuda.synchronize()
        wb.close()
        for w in warm:
            w.close()
        states = [plan.state(bt, 950 + i, stream=stream) for i in range(n_states)]
        batch = imask.Batch(states)
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            batch.step(iters, stream=stream)
            e.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        t = a.elapsed_time(e) / 1e3
        x0 = states[0].get(states[0].X, stream=stream)
        torch.cuda.synchronize()
        rel_plain = math.sqrt(imask.imask_rel_distance(x0, x_plain))
        batch.close()
        for s in states:
            s.close()
        rec = {"states": n_states, "storage": fmt, "solves_per_s": n_states / t, "seconds": t,
               "rel_err_vs_plain_fp32": rel_plain, "clocks": clk,
               "state_bytes": plan.info["state_bytes"],
               "includes": "graph capture and instantiation"}
        if with_oracle:
            st_r, _, _ = o.run_variant(b.ravel(), 0, cpu_iters, storage=fmt)
            st_e = exact
            xg = plan.solve(bt, 0, cpu_iters, stream=stream)
            torch.cuda.synchronize()
            xg = xg.double().cpu().numpy()
            rec["rel_err_vs_fp64_oracle"] = {
                "iters": cpu_iters, "seed": 0,
                "same_rounding": float(np.linalg.norm(xg - st_r["x"]) / np.linalg.norm(st_r["x"])),
                "exact_iteration": float(np.linalg.norm(xg - st_e["x"]) / np.linalg.norm(st_e["x"]))}
        plan.close()
        out[name] = rec
    return out


def time_batch_fan512(imask, p, bt, info, iters, stream, n_states=8):
    """n_states copies of the headline solve advanced as one batch, with one
    graph branch per state and fused (one launch of each kernel per iteration
    for all states); the first batched state's iterate is compared bit for bit
    with a plain solve of the same seed."""
    import torch
    plan = imask.Plan(dict(p.params(), mu=info["mu"], sigma=info["sigma"]))
    out = {"states": n_states, "includes": "graph capture and instantiation"}
    x_plain = plan.solve(bt, 950, iters, stream=stream)
    for name, fused in (("branches", False), ("fused", True)):
        warm = [plan.state(bt, 900 + i, stream=stream) for i in range(n_states)]
        wb = imask.Batch(warm, fused=fused)
        wb.step(4, stream=stream)
        torch.cuda.synchronize()
        wb.close()
        for w in warm:
            w.close()
        states = [plan.state(bt, 950 + i, stream=stream) for i in range(n_states)]
        batch = imask.Batch(states, fused=fused)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            batch.step(iters, stream=stream)
            e.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(e) / 1e3
        x0 = states[0].get(states[0].X, stream=stream)
        torch.cuda.synchronize()
        same = bool(torch.equal(x0, x_plain))
        batch.close()
        for s in states:
            s.close()
        out[name] = {"solves_per_s": n_states / t, "seconds": t,
                     "bit_identical_to_plain_solve": same}
    plan.close()
    return out


# ---------------------------------------------------------------------------------
# 16-bit table storage with an fp32 refinement sweep (1024x1024 fan workload)
# ---------------------------------------------------------------------------------
def run_precision(args):
    """1024x1024 fan beam, 1440 views x 1024 bins (bin pitch 1.5 W / 1024 so the
    magnified field of view stays covered), 5 levels, 500 iterations: the plain
    fp32 form (one solve at a time) against bf16 / fp16 measurement-side tables,
    alone and as a graph-captured batch, each followed by an fp32 refinement
    sweep in steps of 10 iterations while its error against the plain fp32
    result exceeds 1e-3 (at most 100 iterations).  Errors are also given
    against the fixed point of eq. min_obj_new (CG)."""
    import torch
    from paper_2412_10249_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2412_10249_gb300 import imask
    p = inputs.Problem(n=1024, n_angles=1440, n_det=1024, geometry=1, angle_span=2 * math.pi,
                       src_dist=2.0, det_dist=1.0, det_spacing=1.5 / 1024, levels=5)
    b = inputs.sinogram(p, 0)
    bt = torch.as_tensor(b.ravel().astype(np.float32), device="cuda")
    base = imask.Plan(dict(p.params(), mu=0.0, sigma=0.0, autotune=1))
    info = base.info
    xnat, cg_res = cg_fixed_point(base, p, bt, info["mu"])
    flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)
    stream = torch.cuda.Stream()
    K = args.iters
    B = args.precision_batch

    def timed(fn):
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            fn()
            e.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(e) / 1e3

    def refine(states, x_ref):
        """fp32 sweep until every state is within 1e-3 of x_ref; device seconds."""
        t, its = 0.0, 0
        errs = [math.sqrt(imask.imask_rel_distance(s.get(s.X), x_ref)) for s in states]
        first = list(errs)
        while max(errs) > 1e-3 and its < 100:
            if its == 0:
                for s in states:
                    s.set_storage(0, stream=stream)
            t += timed(lambda: [s.step(10, stream=stream) for s in states])
            its += 10
            errs = [math.sqrt(imask.imask_rel_distance(s.get(s.X), x_ref)) for s in states]
        return t, its, first, errs

    plans = {fmt: imask.Plan(dict(p.params(), mu=info["mu"], sigma=info["sigma"], storage=fmt,
                                  autotune=1)) for fmt in (0, 1, 2)}
    # warm-up
    for fmt, plan in plans.items():
        w = plan.state(bt, 99, stream=stream)
        timed(lambda: w.step(10, stream=stream))
        w.close()
    out = {}
    # plain fp32, one solve at a time
    s = plans[0].state(bt, 0, stream=stream)
    flush.fill_(1.0)
    t = timed(lambda: s.step(K, stream=stream))
    x_plain = s.get(s.X)
    out["fp32_plain"] = {"solves_per_s": 1.0 / t, "ms_per_solve": 1e3 * t,
                         "rel_err_vs_fixed_point": math.sqrt(imask.imask_rel_distance(x_plain, xnat)),
                         "state_mb": plans[0].info["state_bytes"] / 2 ** 20}
    for name, fmt in (("bf16", 1), ("fp16", 2)):
        s = plans[fmt].state(bt, 0, stream=stream)
        flush.fill_(1.0)
        t = timed(lambda: s.step(K, stream=stream))
        tr, its, e0, e1 = refine([s], x_plain)
        x = s.get(s.X)
        out[name] = {"solves_per_s": 1.0 / (t + tr), "ms_per_solve": 1e3 * (t + tr),
                     "rel_err_vs_plain_fp32_before_refinement": e0[0],
                     "refine_iters": its, "rel_err_vs_plain_fp32": e1[0],
                     "rel_err_vs_fixed_point": math.sqrt(imask.imask_rel_distance(x, xnat)),
                     "state_mb": plans[fmt].info["state_bytes"] / 2 ** 20}
        s.close()
    # batched bf16: B solves (seeds 0..B-1; seed 0 is compared with the plain result)
    states = [plans[1].state(bt, i, stream=stream) for i in range(B)]
    batch = imask.Batch(states)
    flush.fill_(1.0)
    t = timed(lambda: batch.step(K, stream=stream))
    batch.close()
    tr, its, e0, e1 = refine(states[:1], x_plain)
    if its:
        tr = timed(lambda: [st.step(its, stream=stream) for st in states[1:]]) + tr
    out[f"bf16_batch{B}"] = {"solves_per_s": B / (t + tr), "ms_per_solve": 1e3 * (t + tr) / B,
                             "rel_err_vs_plain_fp32_before_refinement": e0[0],
                             "refine_iters": its, "rel_err_vs_plain_fp32": e1[0],
                             "includes": "graph capture and instantiation"}
    for st in states:
        st.close()
    line = {"metric": "ImaSk solves/s at rel.err<=1e-3 vs plain FP32: 16-bit tables, batched",
            "unit": "solves/s", "iters": K,
            "config": {"workload": "1024x1024 fan 1440x1024 (pitch 1.5W/1024), r=5, K=500, "
                                   "quadratic R", "batch": B},
            "mu": info["mu"], "sigma": info["sigma"], "cg_rel_residual": cg_res,
            "forms": out}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------
# serving: Poisson arrivals, continuous batching under a device-memory budget
# ---------------------------------------------------------------------------------
def serving_mean_samples(n_draws: int = 20000, n_geometries: int = 0) -> float:
    """Mean ray-samples per request of the serving mix (Monte Carlo over the
    request generator; with a geometry fleet, over the fleet the timed run
    draws)."""
    if n_geometries > 0:
        draws = inputs.serving_requests(n_draws / 10.0, 10.0, seed=0,
                                        n_geometries=n_geometries)
    else:
        draws = inputs.serving_requests(n_draws / 10.0, 10.0, seed=12345)
    return float(np.mean([expected_samples_per_solve(p, it) for _, p, it, _ in draws]))


def run_serve(args):
    from paper_2412_10249_gb300 import build as pkg_build
    pkg_build.build()
    print(json.dumps(serving_line(args)))
    return 0


def serving_line(args) -> dict:
    """One serving run (Poisson arrivals over args.serve_seconds, continuous
    batching through serve.Server); returns the report."""
    from paper_2412_10249_gb300 import serve
    rate = args.serve_rate
    mean_samples = serving_mean_samples(n_geometries=args.serve_geometries)
    if args.serve_load > 0:
        # arrivals at a fraction of one GPU's capacity: the request mix's mean
        # ray-samples per solve against the measured solve rate of the GPU
        # (G ray-samples/s of the 512x512 fan workload)
        rate = args.serve_load * args.serve_capacity_gsps * 1e9 / mean_samples
    reqs = []
    problems = {}
    offered = 0.0
    for i, (t, p, iters, seed) in enumerate(inputs.serving_requests(
            args.serve_seconds, rate, seed=0, n_geometries=args.serve_geometries)):
        problems[i] = p
        def make_b(p=p, seed=seed):
            return inputs.poisson_log(inputs.disk_sinogram(p), 1e4, seed)
        reqs.append(serve.Request(rid=i, params=p.params(), b=make_b, iters=iters,
                                  seed=seed, arrival=t))
        offered += expected_samples_per_solve(p, iters)
    srv = serve.Server(budget_bytes=int(args.serve_budget_gb * (1 << 30)),
                       max_active=args.serve_slots, max_queue=args.serve_queue,
                       quantum=10, power_iters=20)
    clocks = ClockSampler(0)
    clocks.start()
    # at a load below capacity every admitted request is served to the end
    # (latencies of all of them); at the overloaded rate the window closes
    drain = args.serve_load > 0
    t0 = time.perf_counter()
    st = srv.run(reqs, duration=args.serve_seconds, drain=drain)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    done = [r for r in reqs if r.status == "done"]
    achieved = sum(expected_samples_per_solve(problems[r.rid], r.iters) for r in done)
    # work launched in the window, unfinished solves included (iterations
    # launched; an upper bound on the iterations executed)
    launched = achieved + sum(expected_samples_per_solve(problems[a.req.rid],
                                                         a.req.iters - a.remaining)
                              for a in srv.active)
    lat = np.array(st.latencies) * 1e3
    wait = np.array(st.waits) * 1e3
    T = wall if drain else args.serve_seconds
    line = {"metric": "served ImaSk solves/s (Poisson arrivals, continuous batching)",
            "unit": "solves/s", "value": len(done) / T, "seconds": T,
            "arrival_window_s": args.serve_seconds, "drained": drain,
            "offered": {"requests": len(reqs), "rate_per_s": rate,
                        "gsamples_per_s": offered / T / 1e9,
                        "load": (rate * mean_samples / (args.serve_capacity_gsps * 1e9)),
                        "mix_mean_gsamples_per_request": mean_samples / 1e9,
                        "capacity_gsamples_per_s": args.serve_capacity_gsps},
            "achieved_gsamples_per_s": achieved / T / 1e9,
            "launched_gsamples_per_s": launched / T / 1e9,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "queue_wait_p50_ms": float(np.percentile(wait, 50)) if wait.size else None,
            "completed": st.completed, "admitted": st.admitted,
            "rejected_queue_full": st.rejected_queue_full,
            "rejected_too_large": st.rejected_too_large,
            "unfinished_at_end": len(srv.active) + len(srv.queue),
            "failed": st.failed, "failed_plans": [[list(k), e] for k, e in st.failed_plans[:5]],
            "max_active": st.max_active, "peak_gb": st.peak_bytes / (1 << 30),
            "plans_built": st.plans_built, "plan_seconds": st.plan_seconds,
            "clocks": clk,
            "config": {"workload": "serving: Poisson arrivals, r in {2..6}, side log-uniform "
                                   "[128, 2048], views [180, 2048], bins 1.5 x side, fan beam, "
                                   "K in [100, 1000]; centred-disk sinograms with Poisson "
                                   "noise", "budget_gb": args.serve_budget_gb,
                       "slots": args.serve_slots, "queue": args.serve_queue, "quantum": 10,
                       "geometries": args.serve_geometries or "one per request"}}
    srv.close()
    return line


# ---------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------# ---------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------
def run_ours(args):
    import torch

    world, rank, local = dist_setup(True)
    torch.cuda.set_device(local)
    from paper_2412_10249_gb300 import build as pkg_build
    if rank == 0 or world == 1:
        pkg_build.build()
    dist_barrier(world)
    from paper_2412_10249_gb300 import imask

    p = inputs.fan512_problem()
    _, b, _ = inputs.measurements(p, seed=rank)
    bt = torch.as_tensor(b.ravel().astype(np.float32), device="cuda")
    # mu and sigma: derived by the plan (power method + Thm. 3) unless given
    n_launch_start = imask.imask_launch_count()
    vopts = dict(variant_params(args.variant, args.dual_tables, args.draws),
                 autotune=args.autotune)
    plan = imask.Plan(dict(p.params(), mu=max(args.mu, 0.0), sigma=max(args.sigma, 0.0),
                           **vopts))
    info = plan.info
    n_launch_plan = imask.imask_launch_count() - n_launch_start
    stream = torch.cuda.Stream()
    x = torch.empty(p.d, device="cuda", dtype=torch.float32)
    flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)

    # level streams (our device draw) to count the ray-samples of every step
    seeds = [rank * 100003 + k for k in range(args.steps)]
    samples = []
    for sd in seeds:
        lv = plan.levels(sd, 0, args.iters).cpu().numpy()
        samples.append(float(samples_per_iteration(p, lv).sum()))

    with torch.cuda.stream(stream):
        for w in range(args.warmup):
            plan.solve(bt, 10**6 + w, args.iters, out=x, stream=stream)
    stream.synchronize()

    clocks = ClockSampler(local)
    starts = [torch.cuda.Event(enable_timing=True) for _ in seeds]
    ends = [torch.cuda.Event(enable_timing=True) for _ in seeds]
    imask.imask_profile_read(reset=True)
    imask.imask_profile_enable(args.profile_period)
    launches0 = imask.imask_launch_count()
    dist_barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k, sd in enumerate(seeds):
            flush.fill_(float(k))   # evict the previous solve's state from L2
            starts[k].record(stream)
            plan.solve(bt, sd, args.iters, out=x, stream=stream)
            ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    dist_barrier(world)
    clk = clocks.stop()
    launches = imask.imask_launch_count() - launches0
    imask.imask_profile_enable(False)
    prof_ms, prof_cnt = imask.imask_profile_read(reset=True)
    plan.check()

    step_ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    T = float(step_ms.sum()) / 1e3
    T_max = dist_max(T, world)
    total_solves = args.steps * world
    value = total_solves / T_max
    gs = dist_sum(sum(samples), world) / T_max / 1e9

    # ---- error of the timed form against the plain FP32 form (no autotuned
    # split, Alg. 1 tables), same seed: relative L2 of the final iterate ----
    plain = imask.Plan(dict(p.params(), mu=info["mu"], sigma=info["sigma"]))
    with torch.cuda.stream(stream):
        x_plain = plain.solve(bt, seeds[0], args.iters, stream=stream)
        x_form = plan.solve(bt, seeds[0], args.iters, stream=stream)
    torch.cuda.synchronize()
    rel_err_plain = math.sqrt(imask.imask_rel_distance(x_form, x_plain))
    plain.close()

    # ---- end to end through the C ABI with host buffers ----
    b_host = torch.empty(p.m, dtype=torch.float32, pin_memory=True)
    b_host.copy_(torch.as_tensor(b.ravel().astype(np.float32)))
    x_host = torch.empty(p.d, dtype=torch.float32, pin_memory=True)
    bdev = torch.empty(p.m, device="cuda", dtype=torch.float32)
    e2e_s = torch.cuda.Event(enable_timing=True)
    e2e_e = torch.cuda.Event(enable_timing=True)
    dist_barrier(world)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e2e_s.record(stream)
        for k, sd in enumerate(seeds):
            bdev.copy_(b_host, non_blocking=True)
            plan.solve(bdev, sd, args.iters, out=x, stream=stream)
            x_host.copy_(x, non_blocking=True)
        e2e_e.record(stream)
    torch.cuda.synchronize()
    T_e2e = dist_max(e2e_s.elapsed_time(e2e_e) / 1e3, world)
    e2e_value = total_solves / T_e2e

    # ---- roofline of the dominant kernel (kind, level) ----
    smem_probe = imask.imask_probe_smem()
    hbm = measured_peaks().get("hbm_gbs")
    l2 = l2_copy_gbs(torch, stream)
    dev = device_units(torch, clk)
    roofline = roofline_report(p, prof_ms, prof_cnt, dev, args.profile_period, smem_probe,
                               l2_gbs=l2, hbm_gbs=hbm)
    # the fused epilogues' algorithmic traffic (7 m + 5 d floats per
    # iteration: y in/out, b, psi_l in/out, psi_mean in/out; x, phi_0 in/out,
    # phi_mean in/out) against the measured HBM copy bandwidth
    bytes_it = 4.0 * (7 * p.m + 5 * p.d)
    mem_gbs = bytes_it * args.iters * args.steps / T_max / 1e9
    memory = {"algorithmic_bytes_per_iteration": bytes_it, "achieved_gbs": mem_gbs,
              "hbm_peak_gbs": hbm, "frac_of_hbm": (mem_gbs / hbm) if hbm else None,
              "l2_copy_gbs": l2, "frac_of_l2_copy": mem_gbs / l2,
              "l2_copy_source": "measured here: device-to-device copy of a 32 MiB buffer "
                                "(L2-resident), read + write bytes, best of 5 x 20 copies",
              "note": "the solve state (about 22 MB) stays in L2; memory is not the bound",
              "smem_probe_gbs": {"load": smem_probe[0], "read_modify_write": smem_probe[1]}}

    # ---- the other iteration variants on the same workload (short runs) ----
    variants = None
    if not args.no_variants:
        plain_ref = imask.Plan(dict(p.params(), mu=info["mu"], sigma=info["sigma"]))
        variants = time_variants(imask, p, bt, info, args.iters, stream, flush, x)
        variants["parallel512_backprojectors"] = time_parallel_backprojectors(
            imask, args.iters, stream, flush)
        variants["batch_fan512"] = time_batch_fan512(imask, p, bt, info, args.iters, stream)
        # the mixed-precision comparison: the batched 16-bit form against the
        # plain fp32 form (the headline value) at the same seed
        with torch.cuda.stream(stream):
            x_ref = plain_ref.solve(bt, 950, args.iters, stream=stream)
        torch.cuda.synchronize()
        mp = time_mixed_precision_fan512(imask, p, bt, info, args.iters, stream, x_ref,
                                         with_oracle=rank == 0 and not args.no_cpu_baseline,
                                         cpu_iters=args.cpu_iters)
        mp["plain_fp32_solves_per_s"] = value
        variants["mixed_precision_fan512"] = mp
        # serving: Poisson arrivals at 0.7 of this GPU's measured capacity, the
        # requests sharing a fleet of four geometries, drained
        sargs = argparse.Namespace(**vars(args))
        sargs.serve_seconds, sargs.serve_load, sargs.serve_geometries = 15.0, 0.7, 4
        sargs.serve_capacity_gsps = gs
        variants["serving"] = serving_line(sargs)

    # ---- CPU baseline: the oracle on a bounded sample ----
    cpu = None
    oracle_err = None
    if rank == 0 and not args.no_cpu_baseline:
        params = dict(p.params(), mu=info["mu"], sigma=info["sigma"])
        dt, sm, x_orc = oracle_sample(p, params, b.ravel(), 0, args.cpu_iters, want_x=True)
        # the timed form against the FP64 oracle on the same seed and iterations
        with torch.cuda.stream(stream):
            x_gpu = plan.solve(bt, 0, args.cpu_iters, stream=stream)
        torch.cuda.synchronize()
        xg = x_gpu.double().cpu().numpy()
        oracle_err = {"iters": args.cpu_iters, "seed": 0,
                      "rel_l2": float(np.linalg.norm(xg - x_orc) / np.linalg.norm(x_orc))}
        per_solve = expected_samples_per_solve(p)
        single = {"value": sm / per_solve / dt, "unit": "solves/s", "cores": 1,
                  "gsamples_per_s": sm / dt / 1e9,
                  "sample": f"{args.cpu_iters} FP64 oracle iterations of the fan512 solve "
                            f"({sm / 1e9:.2f} G ray-samples in {dt:.1f} s)"}
        # all host cores: one unmodified oracle process per core, own seeds
        host = cpu_description()
        pool = OraclePool(host["nproc"])
        try:
            pool.run(p, params, b.ravel(), 500, 1)          # process start-up and imports
            wall, sm_all = pool.run(p, params, b.ravel(), 600, args.cpu_iters)
        finally:
            pool.close()
        cpu = {"value": sm_all / per_solve / wall, "unit": "solves/s", "cores": pool.cores,
               "kind": "oracle", "nproc": host["nproc"], "cpu_model": host["cpu_model"],
               "sample": f"{pool.cores} independent FP64 oracle processes (one per host core, "
                         f"seeds differ), {args.cpu_iters} iterations of the fan512 solve each "
                         f"({sm_all / 1e9:.2f} G ray-samples in {wall:.1f} s of wall time), "
                         f"extrapolated by ray-samples to {ITERS}-iteration solves",
               "gsamples_per_s": sm_all / wall / 1e9,
               "single_thread": single}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded random-ellipse phantom, exact fan-beam line integrals, "
                    "Poisson I0=1e4)",
            "config": workload_config(p, args, world),
            "plan": {"mu": info["mu"], "sigma": info["sigma"], "theta": info["theta"],
                     "bp_view_groups": list(info["bp_view_groups"][:p.levels]),
                     "fp_strip_lines": list(info["fp_strip_lines"][:p.levels])},
            "gsamples_per_s": gs,
            "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
            "rel_err_vs_plain_fp32": rel_err_plain,
            "rel_err_vs_fp64_oracle": oracle_err,
            "wall_s": wall,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 4 * p.m,
                    "d2h_bytes_per_step": 4 * p.d},
            "gpu_launches": int(launches),
            "launches_before_timed": int(launches0),
            "launches_plan": int(n_launch_plan),
            "clocks": clk,
            "roofline": roofline,
            "memory": memory,
            "cpu_baseline": cpu,
            "variants": variants,
        }
        print(json.dumps(line))
    return 0


def build_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters", type=int, default=ITERS)
    ap.add_argument("--ref-iters", type=int, default=3)
    ap.add_argument("--cpu-iters", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--probe", action="store_true",
                    help="time the bare projector / back-projector per level and exit")
    ap.add_argument("--variant", default="alg1", choices=["alg1", "seq"],
                    help="iteration timed on the headline line: Alg. 1 or Alg. 7")
    ap.add_argument("--dual-tables", type=int, default=0, choices=[0, 1])
    ap.add_argument("--draws", type=int, default=0, choices=[0, 1])
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="time the back-projector split per level at plan time")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--ablation", action="store_true",
                    help="distance to the fixed point for the step sizes of Sec. 3.6 and Alg. 7")
    ap.add_argument("--ablation-seeds", type=int, default=3)
    ap.add_argument("--batch", action="store_true",
                    help="mixed-size slices: one after the other vs one graph-captured batch")
    ap.add_argument("--batch-slices", type=int, default=64)
    ap.add_argument("--precision", action="store_true",
                    help="1024x1024: bf16/fp16 tables with an fp32 refinement sweep vs fp32")
    ap.add_argument("--precision-batch", type=int, default=4)
    ap.add_argument("--serve", action="store_true",
                    help="Poisson-arrival serving run with continuous batching")
    ap.add_argument("--serve-seconds", type=float, default=20.0)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-queue", type=int, default=64)
    ap.add_argument("--serve-load", type=float, default=0.0,
                    help="arrival rate as this fraction of one GPU's capacity (else --serve-rate)")
    ap.add_argument("--serve-geometries", type=int, default=0,
                    help="requests share this many geometries (0: every request its own)")
    ap.add_argument("--serve-capacity-gsps", type=float, default=1500.0,
                    help="G ray-samples/s one GPU sustains (the headline workload's rate)")
    ap.add_argument("--profile-period", type=int, default=32,
                    help="time the kernels of every N-th iteration with CUDA events")
    ap.add_argument("--mu", type=float, default=0.0)
    ap.add_argument("--sigma", type=float, default=0.0)
    ap.add_argument("--parallel", action="store_true",
                    help="only the parallel-beam line: owner-computes against pixel-driven "
                         "back-projector")
    return ap


def parse_args(argv=None):
    return build_parser().parse_args(argv)


def main():
    ap = build_parser()
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        # The oracle's cost per iteration does not depend on mu and sigma, and
        # deriving them with the FP64 oracle (power method on 552960 x 262144
        # operators) would take hours; fixed positive values keep the arithmetic.
        if args.mu <= 0 or args.sigma <= 0:
            args.mu, args.sigma = 0.229, 0.0314
        return run_reference(args)
    if args.probe:
        return run_probe(args)
    if args.parallel:
        import torch
        from paper_2412_10249_gb300 import build as pkg_build
        pkg_build.build()
        from paper_2412_10249_gb300 import imask
        stream = torch.cuda.Stream()
        flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)
        line = time_parallel_backprojectors(imask, args.iters, stream, flush)
        print(json.dumps(line))
        return 0
    if args.ablation:
        return run_ablation(args)
    if args.batch:
        return run_batch(args)
    if args.serve:
        return run_serve(args)
    if args.precision:
        return run_precision(args)
    return run_ours(args)


def run_probe(args):
    """Bare K_ell / K_ell^T launches on the fan512 geometry (with --parallel:
    the 512 x 512 parallel-beam geometry and its pixel-driven back-projector),
    a small, fixed workload for profilers: three of each per level, timed with
    CUDA events; then four iterations of one solve."""
    import torch
    from paper_2412_10249_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2412_10249_gb300 import imask
    p = parallel512_problem() if args.parallel else inputs.fan512_problem()
    extra = dict(bp_gather=1) if args.parallel else {}
    plan = imask.Plan(dict(p.params(), mu=0.25, sigma=0.03, **extra))
    _, img = inputs.phantom(0, p.n)
    x = torch.as_tensor(img.ravel().astype(np.float32), device="cuda")
    y = torch.rand(p.m, device="cuda")
    sino = torch.empty(p.m, device="cuda")
    out = torch.empty(p.d, device="cuda")
    res = {}
    for ell in range(p.levels):
        for name, fn in (("K", lambda: plan.project(ell, x, out=sino)),
                         ("KT", lambda: plan.backproject(ell, y, out=out))):
            ts = []
            for _ in range(3):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            res[f"{name}_l{ell}_ms"] = min(ts)
            res[f"{name}_l{ell}_gsamples_per_s"] = p.m * (p.n >> ell) / (min(ts) / 1e3) / 1e9
    # four iterations of a solve from the fan512 sinogram (seed 0): the
    # projector with its fused dual update and the back-projector as the timed
    # solves launch them, inside the library's "imask_step" NVTX range
    _, b, _ = inputs.measurements(p, seed=0)
    bt = torch.as_tensor(b.ravel().astype(np.float32), device="cuda")
    st = plan.state(bt, 0)
    st.step(4)
    torch.cuda.synchronize()
    res["solve_levels"] = [int(v) for v in plan.levels(0, 0, 4).cpu()]
    st.close()
    plan.check()
    print(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
