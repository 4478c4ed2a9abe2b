"""Pins of the oracle's step-size constants and Thm. 3 solver -- CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import Oracle
from paper_2412_10249_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_remark_identical_operators(oracle_lib):
    # Remark after Lemma 1: uniform p and identical normalised operators
    # A~_i = C give L = Lbar_p = n |C| and Lbar = sqrt(n) |C|.  With A_i = p_i K_i
    # and mu = 1 this is K_i = C / p_i.
    rng = np.random.default_rng(0)
    C = rng.standard_normal((7, 5))
    nrm = np.linalg.norm(C, 2)
    for r in (1, 2, 4):
        p = np.full(r, 1.0 / r)
        mats = np.stack([C / p[i] for i in range(r)])
        L, Lb, Lp = Oracle.constants_dense(mats, p, 1.0, 500)
        assert abs(L - r * nrm) < 1e-9 * r * nrm
        assert abs(Lp - r * nrm) < 1e-9 * r * nrm
        assert abs(Lb - math.sqrt(r) * nrm) < 1e-9 * nrm


def test_constants_match_eigendecomposition(oracle_lib):
    # different operators and non-uniform p: compare with the dense spectra of
    # sum p_i^2 K_i^T K_i, sum p_i^2 K_i K_i^T, etc. (Sec. 3.4, eq. def_Lbar)
    rng = np.random.default_rng(1)
    r, dy, dx = 3, 6, 4
    mats = rng.standard_normal((r, dy, dx))
    p = np.array([0.5, 0.3, 0.2])
    mu = 0.7
    L, Lb, Lp = Oracle.constants_dense(mats, p, mu, 2000)
    Kbar = sum(p[i] * mats[i] for i in range(r))
    L_ref = np.linalg.norm(Kbar, 2) / math.sqrt(mu)
    lb = max(np.linalg.eigvalsh(sum(p[i] ** 2 * mats[i].T @ mats[i] for i in range(r)))[-1],
             np.linalg.eigvalsh(sum(p[i] ** 2 * mats[i] @ mats[i].T for i in range(r)))[-1])
    lp = max(np.linalg.eigvalsh(sum(p[i] * mats[i].T @ mats[i] for i in range(r)))[-1],
             np.linalg.eigvalsh(sum(p[i] * mats[i] @ mats[i].T for i in range(r)))[-1])
    assert abs(L - L_ref) < 1e-8 * L_ref
    assert abs(Lb - math.sqrt(lb / mu)) < 1e-8 * Lb
    assert abs(Lp - math.sqrt(lp / mu)) < 1e-8 * Lp


def _theta_thm2(sigma, a, b, L, Lb, Lp, pmin):
    # the convergence factor in the form of Thm. 2 (parameters a, b > 0)
    t1 = (1 + sigma ** 2 * (L ** 2 + (1 + a) * Lp ** 2)) / (1 + sigma) ** 2 + b * Lb ** 2
    t2 = (1 + 1 / a) * sigma ** 2 / (b * (1 + sigma) ** 2) + 1 - pmin
    return max(t1, t2)


@pytest.mark.parametrize("consts", [(2.46, 1.74, 1.23, 0.25), (2.46, 1.23, 2.46, 0.5),
                                    (1.0, 0.8, 0.9, 1.0 / 3)])
def test_reparametrisation_agrees_with_theorem_2(oracle_lib, consts):
    # eq. theta / phi_psi re-express Thm. 2 with eta = sigma/(1+sigma),
    # c = 1/(1 + L^2 + (1+a) Lbar_p^2) and b = rho c / Lbar^2.
    L, Lb, Lp, pmin = consts
    rng = np.random.default_rng(2)
    for _ in range(50):
        a = math.exp(rng.uniform(-3, 3))
        rho = rng.uniform(0.05, 0.95)
        sigma = math.exp(rng.uniform(-6, 0))
        c = 1.0 / (1 + L ** 2 + (1 + a) * Lp ** 2)
        b = rho * c / Lb ** 2
        eta = sigma / (1 + sigma)
        got = Oracle.theta(eta, c, rho, L, Lb, Lp, pmin)
        ref = _theta_thm2(sigma, a, b, L, Lb, Lp, pmin)
        assert abs(got - ref) < 1e-12 * ref


@pytest.mark.parametrize("consts", [(2.46, 1.74, 1.23, 0.25), (2.46, 2.46, 2.46, 1.0),
                                    (0.5, 0.3, 0.4, 0.5)])
def test_thm3_optimum_is_the_minimiser(oracle_lib, consts):
    # eta* of Thm. 3 minimises theta_{c,rho} over eta in (0, c]; in the
    # crossing case phi(eta*) = psi(eta*)
    L, Lb, Lp, pmin = consts
    cbar = 1.0 / (1 + L ** 2 + Lp ** 2)
    for c in (0.1 * cbar, 0.5 * cbar, 0.9 * cbar):
        for rho in (0.1, 0.5, 0.9):
            eta = Oracle.eta_opt(c, rho, L, Lb, Lp, pmin)
            th = Oracle.theta(eta, c, rho, L, Lb, Lp, pmin)
            grid = np.linspace(1e-9, c, 20001)
            brute = min(Oracle.theta(e, c, rho, L, Lb, Lp, pmin) for e in grid)
            assert th <= brute + 1e-12
            assert 0 < eta <= c + 1e-15


def test_optimal_step_is_admissible(oracle_lib):
    # Prop. 1: the reported eta lies in the admissible range and theta < 1
    for L, Lb, Lp, pmin in [(2.46, 1.74, 1.23, 0.5), (2.46, 1.23, 2.46, 0.25),
                            (2.46, 2.46, 2.46, 1.0)]:
        sigma, theta, c, rho = Oracle.optimal_step(L, Lb, Lp, pmin, 200)
        eta = sigma / (1 + sigma)
        assert 0 < theta < 1
        assert c - c * math.sqrt(1 - rho) < eta < c + c * math.sqrt(1 - rho)
        num = 1 - (1 + L ** 2) * c
        den = 1 - (1 + L ** 2 + Lp ** 2) * c
        alpha = 1.0 / (Lb ** 2 / (rho * c) * num / den)
        assert eta < math.sqrt(alpha * pmin)


def test_table1_inconsistent_with_lemma_opt(oracle_lib):
    # Recorded, not reproduced: Lemma 4 (lem:opt) bounds theta from below by
    # 1 - min{(1 - rho) c, p_min} >= 1 - cbar; with r = 1 (p = 1) and
    # L = Lbar_p = 2.46 this is 0.924, above the 0.914 that Table 1 prints.
    rows = []
    with open(os.path.join(GOLDEN, "table1_params.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    r, L, Lp, sig, th = rows[0]
    assert r == 1
    cbar = 1 / (1 + L ** 2 + Lp ** 2)
    assert 1 - cbar > th
    # the solver itself never goes below the lemma's bound
    sigma, theta, c, rho = Oracle.optimal_step(L, L / math.sqrt(1), Lp, 1.0, 200)
    assert theta >= 1 - cbar - 1e-12


def test_constants_on_a_projector_plan(oracle_lib):
    # Lbar <= L-ish sanity for the sketched CT operators and the single-level
    # case: with r = 1, L = Lbar = Lbar_p = |K| / sqrt(mu)
    p = inputs.Problem(n=16, n_angles=12, n_det=24, geometry=0, levels=1, mu=2.0)
    o = Oracle(**p.params())
    L, Lb, Lp = o.constants(400)
    nk = o.norm_K(400)
    for v in (L, Lb, Lp):
        assert abs(v - nk / math.sqrt(2.0)) < 1e-8 * v


def test_lemma1_saddle_operator_is_skew_with_norm_l(oracle_lib):
    # Lemma 1: B z = (A~^* y, -A~ x), A~ = sum_l p_l K_l / sqrt(mu), is
    # skew-symmetric (<z, B z> = 0: the projector pair is adjoint) and its
    # norm is L, attained at z = (v, 0) with v the top right singular vector
    p = inputs.Problem(n=16, n_angles=12, n_det=24, geometry=1, angle_span=2 * math.pi,
                       levels=3)
    mu = 0.6
    o = Oracle(**dict(p.params(), mu=mu, sigma=0.1))
    pr = o.probs()

    def A(x):
        return sum(pr[l] * o.K(l, x).ravel() for l in range(o.r)) / math.sqrt(mu)

    def At(y):
        return sum(pr[l] * o.KT(l, y).ravel() for l in range(o.r)) / math.sqrt(mu)

    L = o.constants(300)[0]
    rng = np.random.default_rng(3)
    for _ in range(4):
        x = rng.standard_normal(o.n * o.n)
        y = rng.standard_normal(o.m)
        bx, by = At(y), -A(x)
        nz = math.sqrt(x @ x + y @ y)
        nb = math.sqrt(bx @ bx + by @ by)
        assert abs(x @ bx + y @ by) <= 1e-13 * nz * nb
        assert nb <= L * nz * (1 + 1e-9)
    v = rng.standard_normal(o.n * o.n)
    for _ in range(400):
        v = At(A(v))
        v /= np.linalg.norm(v)
    assert abs(np.linalg.norm(A(v)) - L) <= 1e-6 * L
