"""Batched stepping through captured CUDA graphs: identical to plain stepping,
state by state, for mixed plans, variants, odd counts and interleaved calls."""
import math

import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2412_10249_gb300 import build as pkg_build
from paper_2412_10249_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def imask():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pkg_build.build()
    from paper_2412_10249_gb300 import imask as m
    m.lib()
    return m


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32).ravel(), device="cuda")


FAN64 = inputs.Problem(n=64, n_angles=90, n_det=96, geometry=1, angle_span=2 * math.pi,
                       levels=4)
PAR40 = inputs.Problem(n=40, n_angles=36, n_det=61, geometry=0, angle_span=math.pi, levels=3)
TV64 = inputs.small_problem()


def _setups(imask):
    """(plan, b) pairs covering Alg. 1, Alg. 7, snapshot tables, independent
    draws and a TV prox (extra launches inside the iteration)."""
    out = []
    for prob, extra in ((FAN64, {}), (PAR40, dict(variant=1, theta=1.0, dual_tables=1)),
                        (FAN64, dict(draws=1, dual_tables=1)),
                        (TV64, dict(reg=1, tv_lambda=0.02, variant=1, theta=0.7))):
        plan = imask.Plan(dict(prob.params(), mu=0.1, sigma=0.04, **extra))
        _, b, _ = inputs.measurements(prob, seed=len(out), noise="none")
        out.append((plan, cuda(b)))
    return out


def test_batch_equals_plain_steps(imask):
    setups = _setups(imask)
    ref = []
    for i, (plan, b) in enumerate(setups):
        s = plan.state(b, 100 + i)
        s.step(20)
        ref.append(s.get(s.X))
    states = [plan.state(b, 100 + i) for i, (plan, b) in enumerate(setups)]
    batch = imask.Batch(states)
    batch.step(20)
    torch.cuda.synchronize()
    for s, r in zip(states, ref):
        assert s.k == 20
        assert torch.equal(s.get(s.X), r)
    batch.close()


def test_batch_mixed_with_plain_and_odd_counts(imask):
    setups = _setups(imask)[:3]
    ref = []
    for i, (plan, b) in enumerate(setups):
        s = plan.state(b, 7 + i)
        s.step(31)
        ref.append((s.get(s.X), s.get(s.Y)))
    states = [plan.state(b, 7 + i) for i, (plan, b) in enumerate(setups)]
    states[0].step(3)          # parities differ across the batch
    batch = imask.Batch(states)
    batch.step(9)              # 4 replays + one plain iteration each
    for s in states[1:]:
        s.step(3)
    batch.step(16)
    states[0].step(3)
    for s in states[1:]:
        s.step(3)
    torch.cuda.synchronize()
    for s, (rx, ry) in zip(states, ref):
        assert s.k == 31
        assert torch.equal(s.get(s.X), rx)
        assert torch.equal(s.get(s.Y), ry)
    batch.close()


def test_batch_matches_oracle(imask):
    prob = FAN64
    params = dict(prob.params(), mu=0.1, sigma=0.04, variant=1, theta=1.0)
    _, b, _ = inputs.measurements(prob, seed=3, noise="none")
    o = Oracle(**dict(prob.params(), mu=0.1, sigma=0.04))
    st, _, _ = o.run_variant(b.ravel(), 5, 24, sequential=True)
    plan = imask.Plan(params)
    s = plan.state(cuda(b), 5)
    batch = imask.Batch([s])
    batch.step(24)
    x = s.get(s.X).double().cpu().numpy()
    assert np.linalg.norm(x - st["x"]) / np.linalg.norm(st["x"]) <= 1e-4
    batch.close()


def test_batch_counts_replayed_launches(imask):
    plan = imask.Plan(dict(FAN64.params(), mu=0.1, sigma=0.04))
    _, b, _ = inputs.measurements(FAN64, seed=1, noise="none")
    states = [plan.state(cuda(b), i) for i in range(3)]
    batch = imask.Batch(states)
    batch.step(2)     # capture
    torch.cuda.synchronize()
    c0 = imask.imask_launch_count()
    batch.step(10)
    torch.cuda.synchronize()
    # every replayed or plain iteration launches its three kernels; each graph
    # replay adds one counter kernel and a batch step at most one counter reset
    # per state
    extra = imask.imask_launch_count() - c0 - 3 * 10 * 3
    assert 0 <= extra <= 3 * (10 // 2 + 1)
    batch.close()


def test_graphs_follow_storage_changes(imask):
    # a state's own graph and a batch's graph are captured again after its
    # tables moved (16-bit -> fp32); plain single-iteration steps are the reference
    plan = imask.Plan(dict(FAN64.params(), mu=0.1, sigma=0.04, storage=2))
    _, b, _ = inputs.measurements(FAN64, seed=4, noise="none")
    bt = cuda(b)
    ref = plan.state(bt, 3)
    for _ in range(12):
        ref.step(1)
    ref.set_storage(0)
    for _ in range(12):
        ref.step(1)
    own = plan.state(bt, 3)
    own.step(12)              # its own graph
    own.set_storage(0)
    own.step(12)
    a, c = plan.state(bt, 3), plan.state(bt, 5)
    batch = imask.Batch([a, c])
    batch.step(12)
    a.set_storage(0)
    batch.step(12)
    torch.cuda.synchronize()
    assert torch.equal(own.get(own.X), ref.get(ref.X))
    assert torch.equal(a.get(a.X), ref.get(ref.X))
    batch.close()


def test_profiled_steps_equal_graph_steps(imask):
    # with profiling at period 8 the profiled iterations run kernel by kernel
    # and the pairs between them replay the graph; the iterates are the same
    plan = imask.Plan(dict(FAN64.params(), mu=0.1, sigma=0.04))
    _, b, _ = inputs.measurements(FAN64, seed=6, noise="none")
    bt = cuda(b)
    x_graph = plan.solve(bt, 8, 37)
    imask.imask_profile_read(reset=True)
    imask.imask_profile_enable(8)
    try:
        x_prof = plan.solve(bt, 8, 37)
        torch.cuda.synchronize()
        ms, cnt = imask.imask_profile_read(reset=True)
    finally:
        imask.imask_profile_enable(0)
    assert torch.equal(x_graph, x_prof)
    # iterations 0, 8, 16, 24, 32 were profiled: 5 of each kind
    assert sum(cnt[0:8]) == 5 and sum(cnt[8:16]) == 5 and sum(cnt[16:24]) == 5


@pytest.mark.parametrize("extra", [{}, dict(dual_tables=1, draws=1), dict(reg=1, tv_lambda=0.02)],
                         ids=["alg1", "alg1_snapshots_independent", "alg1_tv"])
def test_overlapped_streams_equal_serial_order(imask, extra):
    # profiling at period 1 runs every kernel in order on one stream; the
    # default path overlaps projector, back-projector and update on the
    # state's streams inside four-iteration graphs -- same iterates
    prob = TV64 if extra.get("reg") else FAN64
    plan = imask.Plan(dict(prob.params(), mu=0.1, sigma=0.04, **extra))
    _, b, _ = inputs.measurements(prob, seed=8, noise="none")
    bt = cuda(b)
    x_fast = plan.solve(bt, 12, 41)
    imask.imask_profile_enable(1)
    try:
        x_serial = plan.solve(bt, 12, 41)
        torch.cuda.synchronize()
    finally:
        imask.imask_profile_enable(0)
        imask.imask_profile_read(reset=True)
    assert torch.equal(x_fast, x_serial)


# ---- fused batches: one launch of each kernel per iteration for all states ----
def _mixed_setups(imask):
    """Quadratic solves of different sizes, geometries, level counts and
    iteration forms (the fused batch takes reg = 0 only)."""
    probs = (
        (FAN64, {}),
        (PAR40, dict(variant=1, theta=1.0, dual_tables=1)),
        (inputs.Problem(n=48, n_angles=37, n_det=75, geometry=1, angle_span=2 * math.pi,
                        angle_start=0.3, levels=4), dict(draws=1)),
        (inputs.Problem(n=96, n_angles=60, n_det=144, geometry=1, angle_span=2 * math.pi,
                        levels=2), dict(storage=1)),
        (FAN64, dict(dual_tables=1)),
    )
    out = []
    for prob, extra in probs:
        plan = imask.Plan(dict(prob.params(), mu=0.1, sigma=0.04, **extra))
        _, b, _ = inputs.measurements(prob, seed=len(out), noise="none")
        out.append((prob, extra, plan, cuda(b)))
    return out


def test_fused_batch_equals_plain_steps(imask):
    setups = _mixed_setups(imask)
    ref = []
    for i, (_, _, plan, b) in enumerate(setups):
        s = plan.state(b, 40 + i)
        s.step(23)
        ref.append((s.get(s.X), s.get(s.Y), s.get(s.PSI_MEAN)))
    states = [plan.state(b, 40 + i) for i, (_, _, plan, b) in enumerate(setups)]
    states[2].step(1)                 # one state starts at the other parity
    batch = imask.Batch(states, fused=True)
    batch.step(12)                    # three replays
    batch.step(10)                    # two replays and two plain iterations each
    states[0].step(1)
    states[1].step(1)
    for s in states[3:]:
        s.step(1)
    torch.cuda.synchronize()
    for s, (rx, ry, rp) in zip(states, ref):
        assert s.k == 23
        assert torch.equal(s.get(s.X), rx)
        assert torch.equal(s.get(s.Y), ry)
        assert torch.equal(s.get(s.PSI_MEAN), rp)
    batch.close()
    for (_, _, plan, _) in setups:
        plan.check()


def test_fused_batch_matches_oracle(imask):
    # three solves of different sizes and geometries in one fused batch, each
    # against the FP64 oracle on the same seed
    setups = _mixed_setups(imask)[:3]
    states = [plan.state(b, 9 + i) for i, (_, _, plan, b) in enumerate(setups)]
    batch = imask.Batch(states, fused=True)
    batch.step(24)
    torch.cuda.synchronize()
    for i, ((prob, extra, _, _), s) in enumerate(zip(setups, states)):
        _, b, _ = inputs.measurements(prob, seed=i, noise="none")
        o = Oracle(**dict(prob.params(), mu=0.1, sigma=0.04))
        if extra.get("variant") == 1 or extra.get("dual_tables") or extra.get("draws"):
            st, _, _ = o.run_variant(b.ravel(), 9 + i, 24,
                                     sequential=extra.get("variant") == 1,
                                     snapshots=bool(extra.get("dual_tables")),
                                     independent=bool(extra.get("draws")))
        else:
            st, _ = o.run(b.ravel(), 9 + i, 24)
        x = s.get(s.X).double().cpu().numpy()
        err = np.linalg.norm(x - st["x"]) / np.linalg.norm(st["x"])
        assert err <= 1e-4, (i, err)
    batch.close()


def test_fused_batch_launches_three_kernels_per_iteration(imask):
    setups = _mixed_setups(imask)
    states = [plan.state(b, i) for i, (_, _, plan, b) in enumerate(setups)]
    batch = imask.Batch(states, fused=True)
    batch.step(4)     # capture
    torch.cuda.synchronize()
    c0 = imask.imask_launch_count()
    batch.step(8)
    torch.cuda.synchronize()
    # per iteration: projector, planner + back-projector, update; per replay
    # one counter kernel
    assert imask.imask_launch_count() - c0 == 2 * (4 * 4 + 1)
    batch.close()


def test_fused_batch_refuses_a_tv_state(imask):
    plan = imask.Plan(dict(TV64.params(), mu=0.1, sigma=0.04, reg=1, tv_lambda=0.02))
    _, b, _ = inputs.measurements(TV64, seed=0, noise="none")
    s = plan.state(cuda(b), 1)
    with pytest.raises(imask.ImaskError):
        imask.Batch([s], fused=True)
    s.close()
