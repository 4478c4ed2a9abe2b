"""Pins of the oracle's Joseph projector and its transpose -- CPU only.

Each test checks the oracle against something other than itself: exact
column/row sums, the midpoint rule on affine images, analytic disk and
ellipse line integrals, per-view mass, the 90-degree rotation symmetry of the
square grid, and the transpose of an explicitly assembled matrix.
"""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2412_10249_gb300 import inputs


def _par(n, n_angles, n_det=None, **kw):
    return Oracle(n=n, n_angles=n_angles, n_det=n_det or n, geometry=0, fov=1.0,
                  angle_start=0.0, angle_span=math.pi, **kw)


def _fan(n, n_angles, n_det, **kw):
    return Oracle(n=n, n_angles=n_angles, n_det=n_det, geometry=1, fov=1.0,
                  angle_start=0.0, angle_span=2 * math.pi, src_dist=2.0, det_dist=1.0, **kw)


def test_axis_views_are_exact_column_and_row_sums(oracle_lib):
    # theta = 0: vertical rays through the column centres; theta = pi/2: horizontal
    # rays through the row centres.  Joseph reduces to h * (column / row sums).
    n = 16
    rng = np.random.default_rng(0)
    img = rng.random((n, n))
    o = _par(n, 2, n)  # views 0 and pi/2
    s = o.joseph_fp(img)
    h = 1.0 / n
    np.testing.assert_allclose(s[0], h * img.sum(axis=0), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(s[1], h * img.sum(axis=1), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("geometry", [0, 1])
def test_affine_image_is_integrated_exactly(oracle_lib, geometry):
    # For f(x, y) = a + b x + c y sampled at the pixel centres, linear
    # interpolation is exact and the column sum is the midpoint rule, exact for
    # affine integrands: a ray that stays between the first and last pixel
    # centres along its whole march integrates to (W / |cos|) f(0, y(0)).
    n = 32
    W, h = 1.0, 1.0 / 32
    xs = -W / 2 + (np.arange(n) + 0.5) * h
    A, B, C = 0.7, -0.3, 1.9
    img = A + B * xs[None, :] + C * xs[:, None]   # img[i, c] = f(x_c, y_i)
    if geometry == 0:
        o = _par(n, 40, 48)
    else:
        o = _fan(n, 40, 48)
    checked = 0
    for a in range(40):
        for j in range(48):
            p0, d = o.ray(a, j)
            xmaj = abs(d[0]) >= abs(d[1])
            if xmaj:
                t = d[1] / d[0]
                ys = p0[1] + (xs - p0[0]) * t
                if ys.min() < xs[0] or ys.max() > xs[-1]:
                    continue
                y0 = p0[1] + (0.0 - p0[0]) * t
                expect = W * math.hypot(d[0], d[1]) / abs(d[0]) * (A + B * 0.0 + C * y0)
            else:
                t = d[0] / d[1]
                xv = p0[0] + (xs - p0[1]) * t
                if xv.min() < xs[0] or xv.max() > xs[-1]:
                    continue
                x0 = p0[0] + (0.0 - p0[1]) * t
                expect = W * math.hypot(d[0], d[1]) / abs(d[1]) * (A + B * x0 + C * 0.0)
            got = o.joseph_ray(n, img, a, j)
            assert abs(got - expect) <= 1e-12 * max(1.0, abs(expect)), (a, j, got, expect)
            checked += 1
    assert checked > 100


def test_disk_line_integrals_converge(oracle_lib):
    # uniform disk of radius R at the origin: line integral 2 sqrt(R^2 - s^2).
    # The error near the tangent rays depends on how R falls on the pixel grid,
    # so it is not monotone at coarse grids; over a factor 8 in h it must fall
    # by at least a factor 4, and stay below 2% at 256^2.
    R = 0.3
    disk = np.array([[0.0, 0.0, R, R, 0.0, 1.0]])
    errs = {}
    for n in (64, 256, 512):
        o = _par(n, 16, int(1.5 * n))
        img = inputs.rasterize(disk, n, 1.0, supersample=8)
        s = o.joseph_fp(img)
        sj = (np.arange(o.p["n_det"]) - 0.5 * (o.p["n_det"] - 1)) * o.det_spacing()
        exact = 2.0 * np.sqrt(np.maximum(R * R - sj * sj, 0.0))
        errs[n] = np.linalg.norm(s - exact[None, :]) / np.linalg.norm(np.tile(exact, (16, 1)))
    assert errs[256] < 0.02, errs
    assert errs[512] < errs[64] / 4, errs


@pytest.mark.parametrize("geometry", [0, 1])
def test_ellipse_phantom_matches_analytic_sinogram(oracle_lib, geometry):
    errs = []
    for n in (64, 128, 256):
        if geometry == 0:
            p = inputs.Problem(n=n, n_angles=30, n_det=int(1.5 * n), geometry=0)
        else:
            p = inputs.Problem(n=n, n_angles=30, n_det=int(1.5 * n), geometry=1,
                               angle_span=2 * math.pi, src_dist=2.0, det_dist=1.0)
        o = Oracle(**p.params())
        e = inputs.random_ellipses(3, 10)
        img = inputs.rasterize(e, n, 1.0, supersample=8)
        exact = inputs.ellipse_sinogram(e, p)
        s = o.joseph_fp(img)
        errs.append(np.linalg.norm(s - exact) / np.linalg.norm(exact))
    assert errs[-1] < 0.02, errs
    assert errs[2] < errs[0] * 0.6, errs


def test_mass_per_view(oracle_lib):
    # sum_j p_j ds = sum_pixels x h^2: exact at 0 and pi/2, <= 1e-3 for a smooth
    # blob at the other views
    n = 64
    o = _par(n, 24, 96)
    h = 1.0 / n
    xs = -0.5 + (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xs, xs)
    blob = np.exp(-((X - 0.05) ** 2 + (Y + 0.03) ** 2) / (2 * 0.08 ** 2))
    s = o.joseph_fp(blob)
    mass = s.sum(axis=1) * o.det_spacing()
    total = blob.sum() * h * h
    assert abs(mass[0] - total) <= 1e-12 * total
    assert abs(mass[12] - total) <= 1e-12 * total
    assert np.max(np.abs(mass - total)) <= 1e-3 * total


def test_rotation_by_90_degrees_swaps_branches(oracle_lib):
    # Rotating the image by +90 degrees maps view theta to theta + pi/2 with the
    # same offsets; on the square grid this exchanges the x- and y-major branches.
    n = 24
    rng = np.random.default_rng(1)
    img = rng.random((n, n))
    rot = img[::-1, :].T.copy()   # rot(x, y) = img(y, -x)
    o = _par(n, 36, 40)           # 36 views over pi: view a + 18 is theta + pi/2
    s0 = o.joseph_fp(img)
    s1 = o.joseph_fp(rot)
    for a in range(18):
        if a in (9,):             # diagonal view: tie-break makes both x-major
            continue
        np.testing.assert_allclose(s1[a + 18], s0[a], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("geometry,nl", [(0, 16), (1, 16), (0, 8), (1, 8)])
def test_bp_is_transpose_of_assembled_matrix(oracle_lib, geometry, nl):
    if geometry == 0:
        o = _par(16, 12, 20)
    else:
        o = _fan(16, 12, 20)
    A = np.zeros((o.m, nl * nl))
    for p in range(nl * nl):
        e = np.zeros(nl * nl)
        e[p] = 1.0
        A[:, p] = o.joseph_fp(e.reshape(nl, nl)).ravel()
    rng = np.random.default_rng(2)
    y = rng.standard_normal(o.m)
    bp = o.joseph_bp(y.reshape(12, 20), nl).ravel()
    np.testing.assert_allclose(bp, A.T @ y, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("geometry", [0, 1])
@pytest.mark.parametrize("ell", [-1, 0, 1, 2])
def test_dot_test_all_levels(oracle_lib, geometry, ell):
    if geometry == 0:
        o = _par(32, 20, 48, levels=3)
    else:
        o = _fan(32, 20, 48, levels=3)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((32, 32))
    y = rng.standard_normal((20, 48))
    lhs = np.vdot(o.K(ell, x), y)
    rhs = np.vdot(x, o.KT(ell, y))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + abs(rhs))


def test_fan_central_ray_passes_through_origin(oracle_lib):
    o = _fan(16, 8, 21)  # odd bin count: bin 10 has u = 0
    for a in range(8):
        p0, d = o.ray(a, 10)
        # distance from the origin to the line through p0 with direction d
        dist = abs(p0[0] * d[1] - p0[1] * d[0]) / math.hypot(*d)
        assert dist < 1e-14
        # source at distance 2 and the detector at distance 1 on the other side
        assert abs(math.hypot(*p0) - 2.0) < 1e-14
        det = p0 + d
        assert abs(math.hypot(*det) - 1.0) < 1e-14
