"""Pins of the oracle's Alg. 7 (ImaSk-Seq), the snapshot-table variant (remark
after Alg. 3) and the independent primal/dual level draws -- CPU only.

Each variant is pinned to something other than itself: a textbook iteration it
reduces to, a closed-form first iterate, the fixed point of eq. min_obj_new
(which none of the variants moves), or the pinned Alg. 1 / Alg. 7 runs that a
variant equals by linearity.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2412_10249_gb300 import inputs


def _tiny(levels=1, geometry=0, n=16, **kw):
    if geometry == 0:
        return inputs.Problem(n=n, n_angles=12, n_det=24, geometry=0, levels=levels, **kw)
    return inputs.Problem(n=n, n_angles=12, n_det=24, geometry=1, angle_span=2 * math.pi,
                          levels=levels, **kw)


def _dense(o, ell):
    n = o.n
    A = np.zeros((o.m, n * n))
    for p in range(n * n):
        e = np.zeros(n * n)
        e[p] = 1.0
        A[:, p] = o.K(ell, e).ravel()
    return A


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("theta", [1.0, 0.5, 0.0])
def test_seq_single_level_is_textbook_pdhg(oracle_lib, theta):
    # r = 1: every table refresh replaces the only entry, so zeta = K xbar and
    # xi = K^T y^{k+1}: the dual-first primal-dual hybrid gradient iteration
    # with extrapolation (Chambolle & Pock) on 1/2|Kx - b|^2 + mu/2|x|^2.
    s, mu = 0.2, 0.5
    o = Oracle(**_tiny(levels=1, mu=mu, sigma=s).params())
    A = _dense(o, -1)
    rng = np.random.default_rng(2)
    b = rng.standard_normal(o.m)
    x = np.zeros(o.n * o.n)
    xb = np.zeros_like(x)
    y = np.zeros(o.m)
    for _ in range(15):
        y = (y + s * (A @ xb - b)) / (1 + s)       # prox of s f*, f = 1/2|. - b|^2
        xn = (x - (s / mu) * (A.T @ y)) / (1 + s)  # prox of (s/mu) mu/2 |.|^2
        xb = xn + theta * (xn - x)
        x = xn
    st, _ = o.run_seq(b, seed=3, iters=15, theta=theta)
    np.testing.assert_allclose(st["x"], x, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(st["xbar"], xb, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(st["y"], y, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("theta", [1.0, 0.3])
def test_seq_first_iterate_closed_form(oracle_lib, theta):
    # from zeros: y^1 = -s b/(1+s), xi = K_l^T y^1, so
    # x^1 = s^2 / (mu (1+s)^2) K_l^T b and xbar^1 = (1 + theta) x^1
    # (Alg. 1 instead keeps x^1 = 0, because it back-projects y^0 = 0).
    s, mu = 0.07, 0.3
    o = Oracle(**_tiny(levels=3, geometry=1, mu=mu, sigma=s).params())
    b = np.random.default_rng(4).standard_normal(o.m)
    st, lv = o.run_seq(b, seed=9, iters=1, theta=theta)
    want = s * s / (mu * (1 + s) ** 2) * o.KT(int(lv[0]), b).ravel()
    np.testing.assert_allclose(st["x"], want, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(st["xbar"], (1 + theta) * want, rtol=1e-12, atol=1e-15)
    st1, _ = o.run(b, seed=9, iters=1)
    assert np.all(st1["x"] == 0.0)


def _fixed_point_case(levels, geometry, n=16):
    o = Oracle(**_tiny(levels=levels, geometry=geometry, n=n, mu=1.0, sigma=0.05).params())
    mu = o.norm_K(200) ** 2 / 2.46 ** 2
    o.set(mu=mu)
    img = inputs.square_phantom(n, 1 << (levels - 1))
    b = o.K(-1, img).ravel()
    xn, _ = o.solve_quadratic(b)
    return o, b, xn.ravel()


@pytest.mark.parametrize("variant", [
    dict(sequential=True),                              # Alg. 7, theta = 1, sigma = 0.05
    dict(sequential=True, snapshots=True),
    dict(independent=True),
    dict(sequential=True, independent=True, snapshots=True),
])
def test_variants_converge_to_the_sketched_fixed_point(oracle_lib, variant):
    # every variant keeps the fixed point of eq. min_obj_new: with
    # psi_i = K_i x and phi_i = K_i^T y the dual update gives y = Kbar x - b and
    # the primal prox gives mu x = -Kbar^T y, i.e. (Kbar^T Kbar + mu) x = Kbar^T b
    o, b, xn = _fixed_point_case(4, 1)
    st, _, _ = o.run_variant(b, seed=0, iters=900, **variant)
    assert _rel(st["x"], xn) < 1e-7


@pytest.mark.parametrize("sequential", [False, True])
@pytest.mark.parametrize("independent", [False, True])
@pytest.mark.parametrize("reg", [0, 1])
def test_snapshot_tables_equal_the_measurement_tables(oracle_lib, sequential, independent, reg):
    # remark after Alg. 3: K_l (u - u_old) = K_l u - K_l u_old by linearity, so
    # keeping the projector input of the last refresh instead of K_l u gives
    # the same iterates up to rounding
    kw = dict(mu=0.4, sigma=0.05)
    if reg == 1:
        kw.update(reg=1, tv_lambda=0.04, tv_eps=1e-2, tv_inner=5)
    o = Oracle(**_tiny(levels=3, geometry=1, **kw).params())
    b = np.random.default_rng(5).standard_normal(o.m)
    a, ld_a, lp_a = o.run_variant(b, 7, 40, sequential=sequential, independent=independent)
    c, ld_c, lp_c = o.run_variant(b, 7, 40, sequential=sequential, independent=independent,
                                  snapshots=True)
    assert np.array_equal(ld_a, ld_c) and np.array_equal(lp_a, lp_c)
    assert _rel(c["x"], a["x"]) < 1e-11
    assert _rel(c["y"], a["y"]) < 1e-11
    pr = o.probs()
    m = o.m
    psi_mean = sum(pr[l] * a["psi"][l * m:(l + 1) * m] for l in range(o.r))
    assert _rel(c["psi_mean"], psi_mean) < 1e-11


def test_variant_loop_reproduces_alg1_and_alg7(oracle_lib):
    # the shared loop with both options off is Alg. 1, with `sequential` Alg. 7
    o = Oracle(**_tiny(levels=4, geometry=1, mu=0.3, sigma=0.04).params())
    b = np.random.default_rng(6).standard_normal(o.m)
    a, la = o.run(b, 2, 30)
    v, ld, lp = o.run_variant(b, 2, 30)
    assert np.array_equal(la, ld) and np.array_equal(la, lp)
    assert np.array_equal(a["x"], v["x"]) and np.array_equal(a["y"], v["y"])
    s, ls = o.run_seq(b, 2, 30, theta=0.8)
    w, _, _ = o.run_variant(b, 2, 30, sequential=True, theta=0.8)
    assert np.array_equal(s["x"], w["x"]) and np.array_equal(s["xbar"], w["xbar"])


def test_independent_draws(oracle_lib):
    o = Oracle(**_tiny(levels=4, mu=0.3, sigma=0.04).params())
    # the primal stream's seed is the SplitMix64 finaliser of the seed, i.e.
    # the generator's first output from state seed - gamma
    gamma = 0x9E3779B97F4A7C15
    for seed in (0, 1, 12345, 2 ** 63 + 7):
        assert o.primal_seed(seed) == o.splitmix64_at((seed - gamma) % 2 ** 64, 0)
    b = np.random.default_rng(7).standard_normal(o.m)
    _, ld, lp = o.run_variant(b, 11, 60, independent=True)
    assert np.array_equal(ld, o.levels(11, 0, 60))
    assert np.array_equal(lp, o.levels(o.primal_seed(11), 0, 60))
    assert not np.array_equal(ld, lp)
    # the primal levels follow p as well (4 sigma band over 2e5 draws)
    pl = o.levels(o.primal_seed(11), 0, 200000)
    freq = np.bincount(pl, minlength=4) / pl.size
    assert np.all(np.abs(freq - 0.25) < 4 * math.sqrt(0.25 * 0.75 / pl.size))


def test_independent_draws_single_level_is_common(oracle_lib):
    o = Oracle(**_tiny(levels=1, mu=0.3, sigma=0.04).params())
    b = np.random.default_rng(8).standard_normal(o.m)
    a, _, _ = o.run_variant(b, 3, 20)
    c, _, _ = o.run_variant(b, 3, 20, independent=True)
    assert np.array_equal(a["x"], c["x"]) and np.array_equal(a["y"], c["y"])
