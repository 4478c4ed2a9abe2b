"""The pixel-driven back-projector of parallel-beam plans (bp_gather = 1, or
-1 when the plan picks the faster form) against the FP64 oracle and against
the owner-computes back-projector: every
pixel adds Joseph's weight Lambda(q - i) g y over the bins of each view whose
ray passes within one pixel of it.

Tolerances as in the parity tests: relative L2 1e-5 for the operator, 1e-4 for
iterates, 1e-6 for the dot test between the projector and this
back-projector (their weights agree up to the fp32 rounding of the pixel's
local offsets)."""
import math

import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2412_10249_gb300 import build as pkg_build
from paper_2412_10249_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_OP = 1e-5
TOL_ITER = 1e-4


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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32).ravel(), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


CASES = {
    "par64_r4": inputs.Problem(n=64, n_angles=90, n_det=91, geometry=0, angle_span=math.pi,
                               levels=4).params(),
    # views across 45 degrees (the major axis changes between views), a ragged
    # size and non-uniform probabilities
    "par40_r3": inputs.Problem(n=40, n_angles=37, n_det=61, geometry=0, angle_span=math.pi,
                               angle_start=0.2, levels=3, probs=[0.5, 0.3, 0.2]).params(),
    # detector pitch below the pixel width: three or more bins per pixel at level 0
    "par48_fine": inputs.Problem(n=48, n_angles=30, n_det=150, geometry=0, angle_span=math.pi,
                                 det_spacing=0.45 / 48, levels=2).params(),
    "tiny8_r4": inputs.Problem(n=8, n_angles=3, n_det=5, geometry=0, levels=4).params(),
    "par128_r8": inputs.Problem(n=128, n_angles=24, n_det=190, geometry=0, levels=8).params(),
}


def _plans(imask, name):
    params = dict(CASES[name], mu=1.0, sigma=0.1)
    return params, imask.Plan(dict(params, bp_gather=1)), imask.Plan(params)


@pytest.mark.parametrize("name", sorted(CASES))
def test_gather_matches_oracle_and_scatter(imask, name):
    params, gather, scatter = _plans(imask, name)
    o = Oracle(**params)
    yv = np.random.default_rng(1).standard_normal(o.m)
    y = cuda(yv)
    for ell in range(-1, params["levels"]):
        got = host(gather.backproject(ell, y))
        assert rel(got, o.KT(ell, yv).ravel()) <= TOL_OP, (name, ell)
        assert rel(got, host(scatter.backproject(ell, y))) <= TOL_OP, (name, ell)
        # every pixel is written by one thread: two calls agree bit for bit
        assert np.array_equal(got, host(gather.backproject(ell, y)))


@pytest.mark.parametrize("name", sorted(CASES))
def test_gather_dot_test(imask, name):
    # <K_l x, y> = <x, K_l^T y> between the projector and this back-projector
    params, gather, _ = _plans(imask, name)
    n, m = params["n"], params["n_angles"] * params["n_det"]
    rng = np.random.default_rng(3)
    x, y = cuda(rng.random(n * n) + 0.1), cuda(rng.random(m))
    for ell in range(-1, params["levels"]):
        lhs = float(torch.dot(gather.project(ell, x).double(), y.double()))
        rhs = float(torch.dot(x.double(), gather.backproject(ell, y).double()))
        assert abs(lhs - rhs) <= 1e-6 * (abs(lhs) + abs(rhs)), (name, ell, lhs, rhs)


@pytest.mark.parametrize("autotune", [0, 1])
def test_gather_iterates(imask, autotune):
    # Alg. 1 with the pixel-driven back-projector: 12 iterations (three graph
    # replays of four) against the oracle
    prob = inputs.Problem(n=64, n_angles=90, n_det=91, geometry=0, angle_span=math.pi,
                          levels=4)
    _, b, _ = inputs.measurements(prob, seed=2, noise="none")
    params = dict(prob.params(), mu=0.5, sigma=0.05)
    plan = imask.Plan(dict(params, bp_gather=1, autotune=autotune))
    st, _ = Oracle(**params).run(b.ravel(), 7, 12)
    s = plan.state(cuda(b), 7)
    s.step(12)
    assert rel(host(s.get(s.X)), st["x"]) <= TOL_ITER
    assert rel(host(s.get(s.Y)), st["y"]) <= TOL_ITER


def test_gather_is_for_parallel_beam(imask):
    fan = inputs.Problem(n=32, n_angles=20, n_det=48, geometry=1, angle_span=2 * math.pi,
                         levels=2).params()
    with pytest.raises(RuntimeError, match="parallel"):
        imask.Plan(dict(fan, mu=1.0, sigma=0.1, bp_gather=1))


def test_fused_batches_refuse_gather_plans(imask):
    prob = inputs.Problem(n=32, n_angles=20, n_det=46, geometry=0, angle_span=math.pi, levels=2)
    _, b, _ = inputs.measurements(prob, seed=0, noise="none")
    plan = imask.Plan(dict(prob.params(), mu=1.0, sigma=0.1, bp_gather=1))
    s = plan.state(cuda(b), 0)
    with pytest.raises(RuntimeError, match="bp_gather"):
        imask.Batch([s], fused=True)
    batch = imask.Batch([s])   # graph branches run any back-projector
    batch.close()


def test_form_chosen_at_plan_time(imask):
    # bp_gather = -1: for parallel beam the faster form (timed when autotune
    # = 1, else the pixel-driven one), for fan beam the owners; either way the
    # plan reports the form and keeps parity
    name = "par64_r4"
    params = dict(CASES[name], mu=1.0, sigma=0.1)
    o = Oracle(**params)
    yv = np.random.default_rng(5).standard_normal(o.m)
    for autotune in (0, 1):
        plan = imask.Plan(dict(params, bp_gather=-1, autotune=autotune))
        form = plan.info["bp_gather"]
        assert form in (0, 1) and (autotune == 1 or form == 1)
        for ell in range(params["levels"]):
            assert rel(host(plan.backproject(ell, cuda(yv))), o.KT(ell, yv).ravel()) <= TOL_OP
    fan = inputs.Problem(n=32, n_angles=20, n_det=48, geometry=1, angle_span=2 * math.pi,
                         levels=2).params()
    plan = imask.Plan(dict(fan, mu=1.0, sigma=0.1, bp_gather=-1, autotune=1))
    assert plan.info["bp_gather"] == 0
