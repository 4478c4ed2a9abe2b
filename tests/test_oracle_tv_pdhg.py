"""Pins of the oracle's TV-with-nonnegativity prox (Sec. 4.5, FISTA on the
dual) and of its PDHG (Sec. 5 comparison method) -- CPU only."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2412_10249_gb300 import inputs


def _oracle(n=16, levels=1, **kw):
    p = inputs.Problem(n=n, n_angles=12, n_det=24, geometry=1, angle_span=2 * math.pi,
                       levels=levels)
    return Oracle(**dict(p.params(), **kw))


def _prox(o, v, tau):
    return o.prox(tau, v)


def test_tv_prox_without_tv_is_the_projection(oracle_lib):
    v = np.random.default_rng(0).standard_normal((16, 16))
    for kw in (dict(tv_lambda=0.0, tv_inner=20), dict(tv_lambda=0.3, tv_inner=0)):
        o = _oracle(reg=2, mu=1.0, **kw)
        np.testing.assert_array_equal(_prox(o, v, 0.7), np.maximum(v, 0.0))


def test_tv_prox_keeps_constant_images(oracle_lib):
    o = _oracle(reg=2, mu=1.0, tv_lambda=0.5, tv_inner=20)
    v = np.full((16, 16), 0.37)
    np.testing.assert_array_equal(_prox(o, v, 1.3), v)
    np.testing.assert_array_equal(_prox(o, -v, 1.3), np.zeros_like(v))


@pytest.mark.parametrize("a,b,k", [(1.0, 0.2, 5), (0.8, -0.3, 9), (0.5, 0.45, 8)])
def test_tv_prox_row_step_closed_form(oracle_lib, a, b, k):
    # v = a on rows [0, k), b on rows [k, N), constant along the rows.  With
    # alpha = tau lambda: TV_iso(x) >= sum over columns of the 1-D TV, with
    # equality for column-constant x, so the minimiser is the 1-D one
    # replicated: a' = a - alpha/k, b' = max(0, b + alpha/(N - k)) while the
    # jump stays open (a' > b').
    n, tau, lam = 16, 0.5, 0.2
    alpha = tau * lam
    o = _oracle(n=n, reg=2, mu=1.0, tv_lambda=lam, tv_inner=3000)
    v = np.full((n, n), b)
    v[:k] = a
    want = np.full((n, n), max(0.0, b + alpha / (n - k)))
    want[:k] = a - alpha / k
    assert want[0, 0] > want[-1, 0]
    np.testing.assert_allclose(_prox(o, v, tau), want, atol=2e-6)


def test_tv_prox_matches_an_independent_solver(oracle_lib):
    # the same convex problem min_{x>=0} 1/2|x - v|^2 + alpha |grad x|_{1,2}
    # solved by a plain primal-dual (Chambolle-Pock) loop on dense matrices
    n, tau, lam = 8, 0.4, 0.5
    alpha = tau * lam
    o = _oracle(n=n, reg=2, mu=1.0, tv_lambda=lam, tv_inner=4000)
    v = np.random.default_rng(1).uniform(-0.2, 1.0, (n, n))
    d = n * n
    D1 = np.zeros((d, d))
    D2 = np.zeros((d, d))
    for i in range(n):
        for j in range(n):
            p = i * n + j
            if i + 1 < n:
                D1[p, p + n], D1[p, p] = 1.0, -1.0
            if j + 1 < n:
                D2[p, p + 1], D2[p, p] = 1.0, -1.0
    D = np.vstack([D1, D2])
    vv = v.ravel()
    x = vv.copy()
    xb = x.copy()
    z = np.zeros(2 * d)
    s = t = 0.34          # s t |D|^2 < 1 with |D|^2 <= 8
    for _ in range(40000):
        z = z + s * (D @ xb)
        zz = z.reshape(2, d)
        nrm = np.maximum(1.0, np.hypot(zz[0], zz[1]) / alpha)
        z = (zz / nrm).ravel()   # projection onto |z_j| <= alpha
        xn = np.maximum(0.0, (x - t * (D.T @ z) + t * vv) / (1 + t))
        xb = 2 * xn - x
        x = xn
    np.testing.assert_allclose(_prox(o, v, tau).ravel(), x, atol=1e-6)


def test_pdhg_single_level_equals_alg7(oracle_lib):
    # the printed PDHG parameters have t = s/mu, so with r = 1 PDHG and Alg. 7
    # (sigma = s, same theta) are the same iteration
    o = _oracle(n=16, levels=1, mu=0.3, sigma=0.2)
    b = np.random.default_rng(2).standard_normal(o.m)
    s, t, th = Oracle.pdhg_params(o.norm_K(100), 0.3)
    assert abs(t - s / 0.3) <= 1e-15 * t
    pd = o.pdhg(b, 25, s, t, th)
    o.set(sigma=s)
    sq, _ = o.run_seq(b, 0, 25, theta=th)
    np.testing.assert_allclose(pd["x"], sq["x"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(pd["y"], sq["y"], rtol=1e-12, atol=1e-15)


def test_pdhg_converges_to_the_sketched_fixed_point(oracle_lib):
    # on Kbar = sum p_l K_l with the quadratic R, PDHG reaches the CG solution
    o = _oracle(n=16, levels=4, mu=1.0)
    nk = o.norm_K(200)
    mu = nk ** 2 / 2.46 ** 2
    o.set(mu=mu)
    b = o.K(-1, inputs.square_phantom(16, 8)).ravel()
    xn, _ = o.solve_quadratic(b)
    s, t, th = Oracle.pdhg_params(nk, mu)
    st = o.pdhg(b, 300, s, t, th)
    err = np.linalg.norm(st["x"] - xn.ravel()) / np.linalg.norm(xn)
    assert err < 1e-10


def test_imask_and_pdhg_agree_on_tv_nonneg(oracle_lib):
    # both methods minimise 1/2|Kbar x - b|^2 + lambda TV(x) over x >= 0
    o = _oracle(n=16, levels=2, mu=1.0)
    nk = o.norm_K(200)
    mu = nk ** 2 / 2.46 ** 2
    o.set(mu=mu, reg=2, tv_lambda=0.02 * mu, tv_inner=300, sigma=0.05)
    b = o.K(-1, inputs.square_phantom(16, 2)).ravel()
    s, t, th = Oracle.pdhg_params(nk, mu)
    pd = o.pdhg(b, 400, s, t, th)
    im, _, _ = o.run_variant(b, 0, 1200)
    assert np.all(pd["x"] >= 0.0) and np.all(im["x"] >= 0.0)
    err = np.linalg.norm(im["x"] - pd["x"]) / np.linalg.norm(pd["x"])
    assert err < 1e-6
    assert abs(o.objective(b, im["x"]) - o.objective(b, pd["x"])) < 1e-8
