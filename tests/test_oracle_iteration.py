"""Pins of the oracle's Alg. 1, its prox operators and its fixed point -- CPU only."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2412_10249_gb300 import inputs


def _tiny(levels=1, probs=None, reg=0, geometry=0, n=16, **kw):
    if geometry == 0:
        p = inputs.Problem(n=n, n_angles=12, n_det=24, geometry=0, levels=levels, probs=probs,
                           reg=reg, **kw)
    else:
        p = inputs.Problem(n=n, n_angles=12, n_det=24, geometry=1, angle_span=2 * math.pi,
                           levels=levels, probs=probs, reg=reg, **kw)
    return p


def _dense(o, ell):
    """Columns K_ell e_p, assembled from the oracle's operator."""
    n = o.n
    A = np.zeros((o.m, n * n))
    for p in range(n * n):
        e = np.zeros(n * n)
        e[p] = 1.0
        A[:, p] = o.K(ell, e).ravel()
    return A


def test_single_level_is_textbook_primal_dual(oracle_lib):
    # r = 1: xi = K^T y^k and zeta = K x^k, so Alg. 1 is the deterministic
    # iteration x+ = (x - s/mu K^T y)/(1 + s), y+ = (y + s K x - s b)/(1 + s).
    p = _tiny(levels=1, mu=0.5, sigma=0.2)
    o = Oracle(**p.params())
    A = _dense(o, -1)
    rng = np.random.default_rng(0)
    b = rng.standard_normal(o.m)
    x = np.zeros(o.n * o.n)
    y = np.zeros(o.m)
    s, mu = 0.2, 0.5
    for _ in range(15):
        x, y = (x - s / mu * (A.T @ y)) / (1 + s), (y + s * (A @ x) - s * b) / (1 + s)
    st, _ = o.run(b, seed=3, iters=15)
    np.testing.assert_allclose(st["x"], x, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(st["y"], y, rtol=1e-12, atol=1e-14)


def test_tables_hold_the_last_refresh(oracle_lib):
    # after the run, phi_l = K_l^T y and psi_l = K_l x at the last draw of l
    p = _tiny(levels=3, mu=1.0, sigma=0.1)
    o = Oracle(**p.params())
    rng = np.random.default_rng(1)
    b = rng.standard_normal(o.m)
    st = o.new_state()
    xs, ys = [], []
    lvls = []
    for _ in range(12):
        xs.append(st["x"].copy())
        ys.append(st["y"].copy())
        st, lv = o.run(b, seed=9, iters=1, state=st)
        lvls.append(int(lv[0]))
    np.testing.assert_array_equal(np.array(lvls), o.levels(9, 0, 12))
    d, m = o.n * o.n, o.m
    for ell in range(3):
        if ell not in lvls:
            continue
        k = max(i for i, v in enumerate(lvls) if v == ell)
        np.testing.assert_allclose(st["phi"][ell * d:(ell + 1) * d], o.KT(ell, ys[k]).ravel(),
                                   rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(st["psi"][ell * m:(ell + 1) * m], o.K(ell, xs[k]).ravel(),
                                   rtol=1e-13, atol=1e-15)


def test_resume_is_exact(oracle_lib):
    p = _tiny(levels=3, mu=1.0, sigma=0.1)
    o = Oracle(**p.params())
    b = np.random.default_rng(2).standard_normal(o.m)
    a, _ = o.run(b, 5, 20)
    s = o.new_state()
    s, _ = o.run(b, 5, 8, s)
    s, _ = o.run(b, 5, 12, s)
    for key in ("x", "y", "phi", "psi"):
        np.testing.assert_array_equal(a[key], s[key])


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_cg_fixed_point_equals_dense_solve(oracle_lib, levels):
    p = _tiny(levels=levels, mu=0.3)
    o = Oracle(**p.params())
    pr = o.probs()
    Kbar = sum(pr[l] * _dense(o, l) for l in range(levels))
    b = np.random.default_rng(3).standard_normal(o.m)
    xd = np.linalg.solve(Kbar.T @ Kbar + 0.3 * np.eye(o.n * o.n), Kbar.T @ b)
    xc, _ = o.solve_quadratic(b)
    np.testing.assert_allclose(xc.ravel(), xd, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("levels,geometry", [(2, 0), (4, 1)])
def test_iterates_converge_to_the_sketched_fixed_point(oracle_lib, levels, geometry):
    # Thm. 1: with the optimal step the iterates converge linearly to
    # x_nat = argmin 1/2 |sum p_i K_i x - b|^2 + mu/2 |x|^2 (eq. min_obj_new)
    p = _tiny(levels=levels, geometry=geometry, mu=0.0)
    o = Oracle(**p.params())
    nk = o.norm_K(200)
    mu = nk ** 2 / 2.46 ** 2
    o.set(mu=mu)
    L, Lb, Lp = o.constants(300)
    sigma, theta, _, _ = Oracle.optimal_step(L, Lb, Lp, o.probs().min())
    o.set(sigma=sigma)
    img = inputs.square_phantom(16, 1 << (levels - 1))
    b = o.K(-1, img).ravel()
    xn, _ = o.solve_quadratic(b)
    st, _ = o.run(b, seed=0, iters=3000)
    err = np.linalg.norm(st["x"] - xn.ravel()) / np.linalg.norm(xn)
    assert err < 1e-6, (err, sigma, theta)


def test_empirical_rate_respects_theorem_2(oracle_lib):
    # Thm. 2: E|z^k - z*|^2 <= theta^k C with z = (sqrt(mu) x, y) the normalised
    # variables of Sec. 3.3 and C = |z^0 - z*|^2 + b sum_i |B_i z*|^2 / p_i,
    # b = rho c / Lbar^2 at the optimum of Thm. 3 (B_i z* built from
    # A_i = p_i K_i: |B_i z*|^2 = p_i^2 (|K_i^T y*|^2 / mu + |K_i x*|^2)).
    # The mean over 16 seeds stands in for the expectation (slack 1.5).
    p = _tiny(levels=3, mu=0.0, n=8)
    p.n_angles, p.n_det = 8, 12
    o = Oracle(**p.params())
    mu = o.norm_K(200) ** 2 / 2.46 ** 2
    o.set(mu=mu)
    L, Lb, Lp = o.constants(300)
    sigma, theta, c, rho = Oracle.optimal_step(L, Lb, Lp, o.probs().min())
    o.set(sigma=sigma)
    b = np.random.default_rng(5).standard_normal(o.m)
    ref, _ = o.run(b, 0, 20000)           # the saddle point, to round-off
    xs, ys = ref["x"].copy(), ref["y"].copy()
    pr = o.probs()
    bb = rho * c / Lb ** 2
    gamma0 = sum(pr[i] * (np.sum(o.KT(i, ys) ** 2) / mu + np.sum(o.K(i, xs) ** 2))
                 for i in range(3))
    C = mu * np.sum(xs ** 2) + np.sum(ys ** 2) + bb * gamma0
    K = 400
    errs = np.zeros(K)
    for seed in range(16):
        st = o.new_state()
        for k in range(K):
            st, _ = o.run(b, 100 + seed, 1, st)
            errs[k] += mu * np.sum((st["x"] - xs) ** 2) + np.sum((st["y"] - ys) ** 2)
    errs /= 16
    bound = C * theta ** np.arange(1, K + 1)
    assert np.all(errs <= 1.5 * bound), np.max(errs / bound)
    # the contraction is real: the error falls by many orders over K steps
    assert errs[-1] < 1e-6 * errs[0]


def test_quadratic_prox_closed_form(oracle_lib):
    p = _tiny(mu=0.7)
    o = Oracle(**p.params())
    v = np.random.default_rng(6).standard_normal((16, 16))
    np.testing.assert_allclose(o.prox(0.3, v), v / (1 + 0.3 * 0.7), rtol=1e-15)


def test_tv_prox_without_tv_weight_is_quadratic(oracle_lib):
    # lambda = 0: one gradient step with 1/L_in already solves the quadratic
    # problem exactly and FISTA stays there
    p = _tiny(mu=0.7, reg=1, tv_lambda=0.0, tv_eps=1e-2, tv_inner=20)
    o = Oracle(**p.params())
    v = np.random.default_rng(7).standard_normal((16, 16))
    np.testing.assert_allclose(o.prox(0.3, v), v / (1 + 0.3 * 0.7), rtol=1e-14, atol=1e-15)


def test_tv_prox_satisfies_optimality(oracle_lib):
    # With many inner steps the prox output x minimises
    # F(x) = 1/2 |x - v|^2 + tau R(x): the finite-difference gradient of F,
    # built from the regulariser value alone, vanishes at x.
    n = 8
    p = _tiny(mu=1.0, reg=1, tv_lambda=0.1, tv_eps=0.05, tv_inner=3000, n=n)
    o = Oracle(**p.params())
    v = np.random.default_rng(8).standard_normal((n, n))
    tau = 0.5
    x = o.prox(tau, v)

    def F(z):
        return 0.5 * np.sum((z - v) ** 2) + tau * o.regulariser(z)

    g = np.zeros(n * n)
    hstep = 1e-6
    for k in range(n * n):
        e = np.zeros(n * n)
        e[k] = hstep
        g[k] = (F(x + e.reshape(n, n)) - F(x - e.reshape(n, n))) / (2 * hstep)
    assert np.max(np.abs(g)) < 1e-6
    # and it is a minimum
    rng = np.random.default_rng(9)
    for _ in range(5):
        assert F(x) <= F(x + 1e-3 * rng.standard_normal((n, n)))


def test_regulariser_tv_of_constant_and_ramp(oracle_lib):
    # TV_eps of a constant image is n^2 eps; of the ramp x[i, j] = j it is
    # n (n - 1) sqrt(1 + eps^2) + n eps (last column has zero difference).
    n, eps, lam = 8, 0.05, 0.3
    p = _tiny(mu=0.0, reg=1, tv_lambda=lam, tv_eps=eps, n=n)
    o = Oracle(**p.params())
    assert abs(o.regulariser(np.full((n, n), 2.0)) - lam * n * n * eps) < 1e-12
    ramp = np.tile(np.arange(n, dtype=float), (n, 1))
    expect = lam * (n * (n - 1) * math.sqrt(1 + eps * eps) + n * eps)
    assert abs(o.regulariser(ramp) - expect) < 1e-12


def test_objective_is_minimised_at_the_fixed_point(oracle_lib):
    # eq. min_obj_new with the quadratic regulariser: the CG fixed point is the
    # minimiser, so every perturbation raises the objective, quadratically
    p = _tiny(levels=2, mu=0.4)
    o = Oracle(**p.params())
    b = np.random.default_rng(10).standard_normal(o.m)
    xn, _ = o.solve_quadratic(b)
    f0 = o.objective(b, xn)
    rng = np.random.default_rng(11)
    for _ in range(5):
        dlt = rng.standard_normal(xn.shape)
        f1 = o.objective(b, xn + 1e-3 * dlt)
        f2 = o.objective(b, xn + 2e-3 * dlt)
        assert f1 > f0 and f2 > f1
        # quadratic growth: f(x + 2 e) - f0 = 4 (f(x + e) - f0)
        assert abs((f2 - f0) - 4 * (f1 - f0)) < 1e-6 * (f2 - f0)
