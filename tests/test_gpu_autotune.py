"""Plan-time autotuning of the back-projector split and the projector's strip
height: the tuned plan keeps parity with the oracle (the split only changes
the order of the partial-image sum, the strip height only how the image
streams through shared memory) and reports what it chose."""
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


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prob", [
    inputs.Problem(n=64, n_angles=90, n_det=96, geometry=1, angle_span=2 * math.pi, levels=4),
    inputs.Problem(n=48, n_angles=37, n_det=75, geometry=1, angle_span=2 * math.pi,
                   angle_start=0.3, levels=4, probs=[0.3, 0.3, 0.2, 0.2]),
    inputs.Problem(n=80, n_angles=45, n_det=117, geometry=0, angle_span=math.pi, levels=3),
], ids=["fan64_r4", "fan48_p3322", "par80_r3"])
def test_autotuned_plan_keeps_parity(imask, prob):
    params = dict(prob.params(), mu=0.1, sigma=0.04)
    plan = imask.Plan(dict(params, autotune=1))
    info = plan.info
    assert info["autotuned"] == 1
    assert all(v >= 1 for v in info["bp_view_groups"][:prob.levels])
    assert all(t >= 4 and t % 4 == 0 for t in info["fp_strip_lines"][:prob.levels])
    o = Oracle(**params)
    rng = np.random.default_rng(0)
    y = rng.standard_normal(o.m)
    yt = torch.as_tensor(y.astype(np.float32), device="cuda")
    x = rng.standard_normal(prob.n * prob.n)
    xt = torch.as_tensor(x.astype(np.float32), device="cuda")
    for ell in range(prob.levels):
        got = plan.backproject(ell, yt).double().cpu().numpy()
        assert rel(got, o.KT(ell, y)) <= 1e-5, ell
        got = plan.project(ell, xt).double().cpu().numpy()
        assert rel(got, o.K(ell, x)) <= 1e-5, ell
    _, b, _ = inputs.measurements(prob, seed=1, noise="none")
    st, _ = o.run(b.ravel(), 3, 30)
    s = plan.state(torch.as_tensor(b.ravel().astype(np.float32), device="cuda"), 3)
    s.step(30)
    assert rel(s.get(s.X).double().cpu().numpy(), st["x"]) <= 1e-4


def test_shared_memory_probe(imask):
    # ceilings of the roofline report: positive, below the unit-count bound
    # (SMs x 128 B per clock at the maximum clock) with some slack
    load, rmw = imask.imask_probe_smem()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    bound = n_sm * 128 * 2.2e9 / 1e9
    assert 0.2 * bound < load < 1.1 * bound
    assert 0.1 * bound < rmw < 1.1 * bound


def test_strip_loop_variants_keep_parity(imask):
    # The projector's strip loop is compiled separately for strip heights of
    # 16, 20 and 32 lines and once for any other height.  Plans whose default
    # heights hit every one of them (n = 80: 20 at level 0; n = 64: 32, 32,
    # 16 and 8; n = 48: 24, 24, 12 and 8) project within the operator
    # tolerance of the oracle at every level.
    seen = set()
    for n, lv in ((80, 3), (64, 4), (48, 4)):
        prob = inputs.Problem(n=n, n_angles=30, n_det=int(1.5 * n) + 1, geometry=1,
                              angle_span=2 * math.pi, levels=lv)
        params = dict(prob.params(), mu=0.1, sigma=0.04)
        plan = imask.Plan(params)
        heights = plan.info["fp_strip_lines"][:lv]
        seen.update(heights)
        o = Oracle(**params)
        x = np.random.default_rng(n).standard_normal(n * n)
        xt = torch.as_tensor(x.astype(np.float32), device="cuda")
        for ell in range(lv):
            got = plan.project(ell, xt).double().cpu().numpy()
            assert rel(got, o.K(ell, x)) <= 1e-5, (n, ell, heights[ell])
    assert {16, 20, 32} <= seen and seen - {16, 20, 32}, seen
