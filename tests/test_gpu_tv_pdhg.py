"""GPU parity of the TV-with-nonnegativity regulariser (Sec. 4.5) and of PDHG
(Sec. 5 comparison method) against the FP64 oracle; relative L2 1e-4 on
iterates after K iterations."""
import math

import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2412_10249_gb300 import build as pkg_build
from paper_2412_10249_gb300 import inputs

pytestmark = pytest.mark.gpu

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


FAN48 = inputs.Problem(n=48, n_angles=37, n_det=75, geometry=1, angle_span=2 * math.pi,
                       angle_start=0.3, levels=4, probs=[0.3, 0.3, 0.2, 0.2])
PAR64 = inputs.small_problem(reg=0)


def _mu(prob):
    o = Oracle(**dict(prob.params(), mu=1.0))
    nk = o.norm_K(100)
    return nk, nk ** 2 / 2.46 ** 2


def _tv_params(prob, mu, inner=20):
    return dict(prob.params(), mu=mu, sigma=0.05, reg=2, tv_lambda=0.05 * mu, tv_inner=inner)


@pytest.mark.parametrize("prob", [FAN48, PAR64], ids=["fan48_p3322", "par64_r2"])
@pytest.mark.parametrize("seq", [False, True])
def test_tv_nonneg_iterates_match_oracle(imask, prob, seq):
    _, mu = _mu(prob)
    params = _tv_params(prob, mu)
    _, b, _ = inputs.measurements(prob, seed=1)
    o = Oracle(**params)
    st, _, _ = o.run_variant(b.ravel(), 3, 25, sequential=seq)
    plan = imask.Plan(dict(params, variant=int(seq), theta=1.0))
    s = plan.state(cuda(b), 3)
    s.step(25)
    x = host(s.get(s.X))
    assert x.min() >= 0.0
    ex, ey = rel(x, st["x"]), rel(host(s.get(s.Y)), st["y"])
    assert ex <= TOL_ITER and ey <= TOL_ITER, (ex, ey)


def test_tv_nonneg_objective(imask):
    prob = FAN48
    _, mu = _mu(prob)
    params = _tv_params(prob, mu)
    plan = imask.Plan(params)
    o = Oracle(**params)
    _, img = inputs.phantom(4, prob.n)
    bv = np.random.default_rng(5).standard_normal(o.m)
    got = plan.objective(cuda(img), cuda(bv))
    ref = o.objective(bv, img)
    assert abs(got - ref) <= 1e-5 * abs(ref)


@pytest.mark.parametrize("reg", [0, 2])
def test_pdhg_matches_oracle(imask, reg):
    prob = FAN48
    nk, mu = _mu(prob)
    params = dict(prob.params(), mu=mu, sigma=0.05)
    if reg == 2:
        params = _tv_params(prob, mu)
    s, t, th = Oracle.pdhg_params(nk, mu)
    _, b, _ = inputs.measurements(prob, seed=2)
    o = Oracle(**params)
    st = o.pdhg(b.ravel(), 20, s, t, th)
    plan = imask.Plan(params)
    x = host(plan.pdhg(cuda(b), 20, s, t, th))
    assert rel(x, st["x"]) <= TOL_ITER


def test_pdhg_reaches_the_fixed_point(imask):
    prob = PAR64
    nk, mu = _mu(prob)
    params = dict(prob.params(), mu=mu, sigma=0.05)
    o = Oracle(**params)
    _, b, _ = inputs.measurements(prob, seed=0)
    xn, _ = o.solve_quadratic(b.ravel())
    s, t, th = imask.imask_pdhg_params(nk, mu, 0.99)
    plan = imask.Plan(params)
    x = host(plan.pdhg(cuda(b), 300, s, t, th))
    assert rel(x, xn) <= 1e-5
