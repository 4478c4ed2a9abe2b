"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: relative L2 1e-5 for the FP32 projector and back-projector, 1e-4
for iterates after K iterations, bit-exact level streams.  The dot test bounds
the mismatch between the two GPU kernels (1e-6 relative).
"""
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
    "par64_r2": inputs.small_problem(reg=0).params(),
    "fan64_r4": inputs.Problem(n=64, n_angles=90, n_det=96, geometry=1, angle_span=2 * math.pi,
                               levels=4).params(),
    "fan48_ragged": inputs.Problem(n=48, n_angles=37, n_det=75, geometry=1,
                                   angle_span=2 * math.pi, angle_start=0.3, levels=4,
                                   probs=[0.4, 0.3, 0.2, 0.1]).params(),
    "par40_r3": inputs.Problem(n=40, n_angles=36, n_det=61, geometry=0, angle_span=math.pi,
                               levels=3).params(),
    "tiny8_r4": inputs.Problem(n=8, n_angles=3, n_det=5, geometry=0, levels=4).params(),
    "par128_r8": inputs.Problem(n=128, n_angles=24, n_det=190, geometry=0, levels=8).params(),
}


def _image(n, seed=0):
    _, img = inputs.phantom(seed, n)
    return img


@pytest.mark.parametrize("name", list(CASES))
def test_projector_parity_all_levels(imask, name):
    params = dict(CASES[name], mu=1.0, sigma=0.1)
    plan = imask.Plan(params)
    # the plan's major-axis tables are the host geometry's (and so the oracle's)
    assert plan.axis_split() == imask.imask_geometry_axis_split(params), name
    o = Oracle(**params)
    img = _image(params["n"], 1)
    x = cuda(img)
    for ell in range(-1, params["levels"]):
        got = host(plan.project(ell, x))
        ref = o.K(ell, img).ravel()
        assert rel(got, ref) <= TOL_OP, (name, ell, rel(got, ref))
    plan.check()


@pytest.mark.parametrize("name", list(CASES))
def test_backprojector_parity_all_levels(imask, name):
    params = dict(CASES[name], mu=1.0, sigma=0.1)
    plan = imask.Plan(params)
    o = Oracle(**params)
    rng = np.random.default_rng(2)
    yv = rng.standard_normal(o.m)
    y = cuda(yv)
    for ell in range(-1, params["levels"]):
        got = host(plan.backproject(ell, y))
        ref = o.KT(ell, yv).ravel()
        assert rel(got, ref) <= TOL_OP, (name, ell, rel(got, ref))


@pytest.mark.parametrize("name", ["fan64_r4", "fan48_ragged", "par40_r3", "par128_r8"])
def test_gpu_dot_test(imask, name):
    # <K_l x, y> = <x, K_l^T y> between the two GPU kernels
    params = dict(CASES[name], mu=1.0, sigma=0.1)
    plan = imask.Plan(params)
    n, m = params["n"], params["n_angles"] * params["n_det"]
    rng = np.random.default_rng(3)
    xv = _image(n, 4) + 0.1
    yv = rng.random(m)
    x, y = cuda(xv), cuda(yv)
    for ell in range(-1, params["levels"]):
        kx = plan.project(ell, x).double()
        kty = plan.backproject(ell, y).double()
        lhs = float(torch.dot(kx, y.double()))
        rhs = float(torch.dot(x.double(), kty))
        assert abs(lhs - rhs) <= 1e-6 * (abs(lhs) + abs(rhs)), (ell, lhs, rhs)


def test_level_stream_bit_exact(imask):
    for probs, r in ((None, 4), ([0.4, 0.3, 0.2, 0.1], 4), (None, 2), (None, 7)):
        params = inputs.Problem(n=64, n_angles=4, n_det=4, levels=r, probs=probs).params()
        plan = imask.Plan(dict(params, mu=1.0, sigma=0.1))
        o = Oracle(**params)
        for seed, k0 in ((0, 0), (12345, 10**9), (2**63 + 5, 77)):
            got = plan.levels(seed, k0, 1_000_000).cpu().numpy()
            ref = o.levels(seed, k0, 1_000_000)
            assert np.array_equal(got, ref), (probs, r, seed)


def _iterate_case(imask, params, b, seed, iters, reg_params=None):
    o = Oracle(**params)
    plan = imask.Plan(params)
    st, lv = o.run(b, seed, iters)
    bt = cuda(b)
    s = plan.state(bt, seed)
    s.step(iters)
    x = host(s.get(s.X))
    y = host(s.get(s.Y))
    plan.check()
    return rel(x, st["x"]), rel(y, st["y"]), lv


def _mu_sigma(params, iters=200):
    o = Oracle(**dict(params, mu=1.0))
    mu = o.norm_K(iters) ** 2 / 2.46 ** 2
    o.set(mu=mu)
    L, Lb, Lp = o.constants(iters)
    sigma, theta, _, _ = Oracle.optimal_step(L, Lb, Lp, o.probs().min())
    return mu, sigma


def test_iterates_small_tv_workload(imask):
    # 64x64 parallel beam, 60 views, 92 bins, 1% Gaussian noise, two levels,
    # quadratic + smoothed TV, 50 iterations
    p = inputs.small_problem()
    mu, sigma = _mu_sigma(dict(p.params(), reg=0), 100)
    params = dict(p.params(), mu=mu, sigma=sigma, tv_lambda=0.1 * mu)
    _, b, _ = inputs.measurements(p, seed=0)
    ex, ey, lv = _iterate_case(imask, params, b.ravel(), seed=0, iters=50)
    assert set(lv) == {0, 1}
    assert ex <= TOL_ITER and ey <= TOL_ITER, (ex, ey)


@pytest.mark.parametrize("name,iters", [("fan64_r4", 40), ("fan48_ragged", 30),
                                        ("par40_r3", 30), ("par128_r8", 12)])
def test_iterates_quadratic(imask, name, iters):
    base = CASES[name]
    mu, sigma = _mu_sigma(base, 60)
    params = dict(base, mu=mu, sigma=sigma)
    p = inputs.Problem(**{k: v for k, v in base.items()})
    _, b, _ = inputs.measurements(p, seed=3, noise="none")
    ex, ey, lv = _iterate_case(imask, params, b.ravel(), seed=11, iters=iters)
    assert ex <= TOL_ITER and ey <= TOL_ITER, (name, ex, ey)


def test_state_resume_and_solve_agree(imask):
    params = dict(CASES["fan64_r4"], mu=0.05, sigma=0.02)
    plan = imask.Plan(params)
    p = inputs.Problem(**CASES["fan64_r4"])
    _, b, _ = inputs.measurements(p, seed=5, noise="none")
    bt = cuda(b)
    x_solve = plan.solve(bt, 9, 20)
    s = plan.state(bt, 9)
    s.step(7)
    s.step(13)
    assert s.k == 20
    assert torch.equal(s.get(s.X), x_solve)
    # zero iterations returns the Alg. 1 default x0 = 0
    assert float(plan.solve(bt, 9, 0).abs().max()) == 0.0


def test_running_means_track_the_tables(imask):
    # psi_mean / phi_mean kept incrementally equal sum_l p_l K_l x_last(l) and
    # sum_l p_l K_l^T y_last(l) of the oracle run
    params = dict(CASES["fan48_ragged"], mu=0.05, sigma=0.02)
    o = Oracle(**params)
    plan = imask.Plan(params)
    p = inputs.Problem(**CASES["fan48_ragged"])
    _, b, _ = inputs.measurements(p, seed=6, noise="none")
    st, _ = o.run(b.ravel(), 4, 25)
    s = plan.state(cuda(b), 4)
    s.step(25)
    pr = o.probs()
    d, m, r = o.n * o.n, o.m, o.r
    psi_mean = sum(pr[l] * st["psi"][l * m:(l + 1) * m] for l in range(r))
    phi_mean = sum(pr[l] * st["phi"][l * d:(l + 1) * d] for l in range(r))
    assert rel(host(s.get(s.PSI_MEAN)), psi_mean) <= TOL_ITER
    assert rel(host(s.get(s.PHI_MEAN)), phi_mean) <= TOL_ITER


def test_plan_constants_match_oracle(imask):
    base = CASES["fan64_r4"]
    params = dict(base, mu=0.0, sigma=0.0)
    plan = imask.Plan(params)
    info = plan.info
    o = Oracle(**dict(base, mu=1.0))
    nk = o.norm_K(100)
    assert abs(info["norm_K"] - nk) <= 1e-4 * nk
    mu = nk ** 2 / 2.46 ** 2
    assert abs(info["mu"] - mu) <= 2e-4 * mu
    o.set(mu=info["mu"])
    L, Lb, Lp = o.constants(100)
    for got, ref in ((info["L"], L), (info["Lbar"], Lb), (info["Lbar_p"], Lp)):
        assert abs(got - ref) <= 1e-4 * ref, (got, ref)
    s_ref = Oracle.optimal_step(info["L"], info["Lbar"], info["Lbar_p"], 0.25)
    assert abs(info["sigma"] - s_ref[0]) <= 1e-12 * s_ref[0]
    assert 0 < info["theta"] < 1


def test_objective_matches_oracle(imask):
    for name, reg in (("par64_r2", 1), ("fan48_ragged", 0)):
        params = dict(CASES[name], mu=0.3, sigma=0.1, reg=reg, tv_lambda=0.05, tv_eps=0.01)
        plan = imask.Plan(params)
        o = Oracle(**params)
        n = params["n"]
        xv = _image(n, 7)
        bv = np.random.default_rng(8).standard_normal(o.m)
        got = plan.objective(cuda(xv), cuda(bv))
        ref = o.objective(bv, xv)
        assert abs(got - ref) <= 1e-5 * abs(ref), (name, got, ref)


def test_rel_distance(imask):
    a = torch.randn(10007, device="cuda")
    b = torch.randn(10007, device="cuda")
    got = imask.imask_rel_distance(a, b)
    ref = float(((a.double() - b.double()) ** 2).sum() / (b.double() ** 2).sum())
    assert abs(got - ref) <= 1e-12 * ref


def test_errors_are_reported(imask):
    plan = imask.Plan(dict(CASES["tiny8_r4"], mu=1.0, sigma=0.1))
    x = torch.zeros(64, device="cuda")
    with pytest.raises(imask.ImaskError):
        plan.project(4, x)
    with pytest.raises(ValueError):
        plan.project(0, torch.zeros(63, device="cuda"))
    with pytest.raises(TypeError):
        plan.project(0, torch.zeros(64, device="cuda", dtype=torch.float64))


# ---- the 512x512 fan-beam workload, in the launch configuration of the benchmark ----

@pytest.fixture(scope="module")
def fan512(imask):
    p = inputs.fan512_problem()
    mu, sigma = 0.25, 0.03
    params = dict(p.params(), mu=mu, sigma=sigma)
    _, b, _ = inputs.measurements(p, seed=0)
    return params, b.ravel(), imask.Plan(params), Oracle(**params)


def test_fan512_projector_and_backprojector(imask, fan512):
    params, b, plan, o = fan512
    img = _image(512, 0)
    x = cuda(img)
    yv = np.random.default_rng(1).standard_normal(o.m)
    y = cuda(yv)
    for ell in (0, 1, 2, 3):
        assert rel(host(plan.project(ell, x)), o.K(ell, img).ravel()) <= TOL_OP, ell
    for ell in (0, 3):
        assert rel(host(plan.backproject(ell, y)), o.KT(ell, yv).ravel()) <= TOL_OP, ell


def test_fan512_iterates(imask, fan512):
    params, b, plan, o = fan512
    seed = 21
    lv = o.levels(seed, 0, 6)
    assert len(set(lv.tolist())) >= 3
    st, _ = o.run(b, seed, 6)
    s = plan.state(cuda(b), seed)
    s.step(6)
    assert rel(host(s.get(s.X)), st["x"]) <= TOL_ITER
    assert rel(host(s.get(s.Y)), st["y"]) <= TOL_ITER


def test_fan512_autotuned_launch_configuration(imask, fan512):
    # the benchmark's plan: back-projector splits and projector strip heights
    # measured at plan time; 12 iterations in one call run as graph replays of
    # four iterations (the form the benchmark times), checked against the
    # oracle at full size
    params, b, _, o = fan512
    plan = imask.Plan(dict(params, autotune=1))
    assert plan.info["autotuned"] == 1
    yv = np.random.default_rng(2).standard_normal(o.m)
    y = cuda(yv)
    xv = np.random.default_rng(3).standard_normal(o.n * o.n)
    x = cuda(xv)
    for ell in (1, 2):
        assert rel(host(plan.backproject(ell, y)), o.KT(ell, yv).ravel()) <= TOL_OP, ell
        assert rel(host(plan.project(ell, x)), o.K(ell, xv).ravel()) <= TOL_OP, ell
    seed = 33
    st, _ = o.run(b, seed, 12)
    s = plan.state(cuda(b), seed)
    s.step(12)
    assert s.k == 12
    assert rel(host(s.get(s.X)), st["x"]) <= TOL_ITER
    assert rel(host(s.get(s.Y)), st["y"]) <= TOL_ITER
