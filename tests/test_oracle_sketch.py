"""Pins of the oracle's image-domain sketches (Sec. 4.1) -- CPU only."""
import math

import numpy as np
import pytest

from oracle import Oracle


def _o(n=16, levels=3, probs=None):
    return Oracle(n=n, n_angles=8, n_det=24, geometry=0, angle_span=math.pi, levels=levels,
                  probs=probs)


def test_block_mean_of_a_ramp(oracle_lib):
    # x[i, j] = i n + j: the mean over the block (I, J) of side b is
    # (I b + (b - 1)/2) n + J b + (b - 1)/2.
    n = 16
    x = (np.arange(n)[:, None] * n + np.arange(n)[None, :]).astype(np.float64)
    o = _o(n)
    for ell in (1, 2, 3):
        b = 1 << ell
        I = np.arange(n // b)[:, None]
        J = np.arange(n // b)[None, :]
        expect = (I * b + (b - 1) / 2) * n + J * b + (b - 1) / 2
        np.testing.assert_array_equal(o.block_mean(x, ell), expect)


def test_replicate_then_average_is_identity(oracle_lib):
    o = _o()
    rng = np.random.default_rng(0)
    for ell in (1, 2, 3):
        c = rng.standard_normal((16 >> ell, 16 >> ell))
        np.testing.assert_allclose(o.block_mean(o.replicate(c, ell), ell), c, rtol=0, atol=1e-15)


def test_projector_is_orthogonal_and_idempotent(oracle_lib):
    # S_ell = T_ell^* T_ell assembled densely: P^2 = P = P^T
    o = _o(8)
    for ell in (1, 2):
        P = np.zeros((64, 64))
        for p in range(64):
            e = np.zeros((8, 8))
            e.flat[p] = 1.0
            P[:, p] = o.replicate(o.block_mean(e, ell), ell).ravel()
        np.testing.assert_allclose(P @ P, P, atol=1e-15)
        np.testing.assert_allclose(P, P.T, atol=1e-15)
        # rank = number of blocks
        assert np.linalg.matrix_rank(P) == (8 >> ell) ** 2


def test_transpose_of_block_mean_is_scaled_replication(oracle_lib):
    o = _o()
    rng = np.random.default_rng(1)
    for ell in (1, 2, 3):
        a = rng.standard_normal((16, 16))
        c = rng.standard_normal((16 >> ell, 16 >> ell))
        lhs = np.vdot(o.block_mean(a, ell), c)
        rhs = np.vdot(a, o.replicate(c, ell) / 4 ** ell)
        assert abs(lhs - rhs) < 1e-12


@pytest.mark.parametrize("probs", [None, [0.2, 0.3, 0.3, 0.2], [0.1, 0.6, 0.2, 0.1]])
def test_sketches_average_to_identity(oracle_lib, probs):
    # eq. si: sum_i p_i S_i = I, with S_0 the compensation S_r
    o = _o(16, 4, probs)
    p = o.probs()
    rng = np.random.default_rng(2)
    x = rng.standard_normal((16, 16))
    acc = p[0] * o.compensate(x)
    for ell in (1, 2, 3):
        acc += p[ell] * o.replicate(o.block_mean(x, ell), ell)
    np.testing.assert_allclose(acc, x, rtol=0, atol=1e-13)


def test_compensation_is_symmetric(oracle_lib):
    o = _o(8, 3)
    S = np.zeros((64, 64))
    for p in range(64):
        e = np.zeros((8, 8))
        e.flat[p] = 1.0
        S[:, p] = o.compensate(e).ravel()
    np.testing.assert_allclose(S, S.T, atol=1e-14)


def test_single_level_is_the_plain_operator(oracle_lib):
    # r = 1: S_0 = I, so K_0 = K and Kbar = K
    o = _o(16, 1)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((16, 16))
    y = rng.standard_normal((8, 24))
    np.testing.assert_array_equal(o.K(0, x), o.K(-1, x))
    np.testing.assert_array_equal(o.KT(0, y), o.KT(-1, y))


def test_coarse_level_sees_only_block_means(oracle_lib):
    # K_ell = R_ell T_ell: images with equal block means give equal data, and
    # K_ell^T y is constant on every block
    o = _o(16, 3)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((16, 16))
    for ell in (1, 2):
        b = 1 << ell
        z = x - o.replicate(o.block_mean(x, ell), ell)   # zero block means
        np.testing.assert_allclose(o.K(ell, z), 0.0, atol=1e-13)
        g = o.KT(ell, rng.standard_normal((8, 24)))
        blocks = g.reshape(16 // b, b, 16 // b, b)
        np.testing.assert_allclose(blocks - blocks[:, :1, :, :1], 0.0, atol=1e-14)


def test_sketched_operator_is_close_to_k_on_smooth_images(oracle_lib):
    # Fig. 2(f): the sinogram of the sketched operator Kbar = sum_l p_l K_l
    # differs from K x by a discretisation error that shrinks as the image
    # gets smoother (Gaussian blobs of width w = 4, 8, 16 pixels, 64x64,
    # r = 4).  A coarse projector with the wrong pixel width or grid offset
    # misses by tens of percent.
    o = Oracle(n=64, n_angles=60, n_det=92, geometry=0, angle_span=math.pi, levels=4)
    pr = o.probs()
    yy, xx = np.mgrid[0:64, 0:64]
    errs = []
    for w in (4.0, 8.0, 16.0):
        img = np.exp(-((xx - 31.5) ** 2 + (yy - 31.5) ** 2) / (2 * w * w))
        kx = o.K(-1, img).ravel()
        kb = sum(pr[l] * o.K(l, img).ravel() for l in range(4))
        errs.append(np.linalg.norm(kx - kb) / np.linalg.norm(kx))
    assert errs[0] < 0.045 and errs[1] < 0.025 and errs[2] < 0.012
    assert errs[2] < errs[1] < errs[0]
