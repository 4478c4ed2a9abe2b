"""The seeded input recipe shared by the oracle checks, the GPU tests and the
benchmark (CPU only): phantom parameters, raster mass, exact line integrals,
noise models and the request / slice mixes of the batched and served
workloads."""
import math

import numpy as np
import pytest

from paper_2412_10249_gb300 import inputs


def test_ellipse_recipe_ranges_and_seeding():
    for seed in range(20):
        e = inputs.random_ellipses(seed, 10)
        assert e.shape == (10, 6)
        cx, cy, a, b, al, rho = e.T
        assert np.all((a >= 0.03) & (a <= 0.25) & (b >= 0.03) & (b <= 0.25))
        assert np.all(np.hypot(cx, cy) <= 0.45 * (1.0 - np.maximum(a, b)) + 1e-12)
        assert np.all((al >= 0.0) & (al < math.pi) & (rho >= 0.0) & (rho <= 1.0))
        np.testing.assert_array_equal(e, inputs.random_ellipses(seed, 10))
    assert not np.array_equal(inputs.random_ellipses(0, 10), inputs.random_ellipses(1, 10))
    # 10 ellipses below N = 1024 (16 from there on)
    assert inputs.phantom(3, 64)[0].shape == (10, 6)


def test_raster_mass_is_the_ellipse_area():
    # ellipses well inside the square: mass = sum rho pi a b up to the 4x4
    # supersampling error of the boundary pixels
    e = np.array([[0.10, -0.05, 0.20, 0.12, 0.4, 0.7],
                  [-0.20, 0.15, 0.08, 0.15, 2.0, 0.3],
                  [0.05, 0.25, 0.10, 0.05, 1.0, 1.0]])
    n = 256
    img = inputs.rasterize(e, n)
    mass = img.sum() * (1.0 / n) ** 2
    want = float(np.sum(e[:, 5] * math.pi * e[:, 2] * e[:, 3]))
    assert abs(mass - want) < 2e-3 * want


@pytest.mark.parametrize("geometry", [0, 1])
def test_disk_sinogram_equals_the_chord_of_a_circle(geometry):
    # two independent routes to the same line integrals: the closed form of a
    # centred disk, and the quadratic chord of an ellipse with equal axes
    p = inputs.Problem(n=64, n_angles=24, n_det=96, geometry=geometry,
                       angle_span=2 * math.pi if geometry else math.pi)
    d = inputs.disk_sinogram(p, radius=0.3, density=0.8)
    c = inputs.ellipse_sinogram(np.array([[0.0, 0.0, 0.3, 0.3, 0.7, 0.8]]), p)
    np.testing.assert_allclose(d, c, atol=1e-12)
    assert d.max() == pytest.approx(2 * 0.8 * 0.3, rel=2e-3)   # a ray through the centre


def test_poisson_log_noise():
    b = np.full(200000, 0.7)
    y = inputs.poisson_log(b, 1e4, seed=5)
    # -log(counts / I0) with counts ~ Poisson(I0 e^-b): mean b to first order,
    # standard deviation 1 / sqrt(I0 e^-b)
    sd = 1.0 / math.sqrt(1e4 * math.exp(-0.7))
    assert abs(y.mean() - 0.7) < 5 * sd / math.sqrt(y.size) + sd ** 2
    assert y.std() == pytest.approx(sd, rel=0.02)
    # no photons: the zero-count clamp gives log(I0)
    assert np.all(inputs.poisson_log(np.full(10, 60.0), 1e4, seed=1) == pytest.approx(
        math.log(1e4)))


def test_gaussian_noise_scale():
    b = np.linspace(0.0, 3.0, 100000)
    y = inputs.gaussian_noise(b, 0.01, seed=2)
    assert (y - b).std() == pytest.approx(0.03, rel=0.02)
    assert abs((y - b).mean()) < 5 * 0.03 / math.sqrt(b.size)


def test_slice_mix_recipe():
    probs = inputs.slice_mix(200, seed=0)
    sides = {p.n for p in probs}
    views = {p.n_angles for p in probs}
    assert sides <= {256, 384, 512, 768, 1024} and len(sides) == 5
    assert views <= {180, 360, 720, 1080, 1440} and len(views) == 5
    for p in probs:
        assert p.n_det == 3 * p.n // 2 and p.geometry == 1 and p.levels == 4
        assert p.n % (1 << (p.levels - 1)) == 0


def test_serving_request_stream():
    dur, rate = 20.0, 200.0
    reqs = inputs.serving_requests(dur, rate, seed=0)
    # Poisson arrivals: the count is within 5 sigma of rate x duration
    assert abs(len(reqs) - rate * dur) < 5 * math.sqrt(rate * dur)
    ts = [t for t, _, _, _ in reqs]
    assert all(0 < t0 < t1 < dur for t0, t1 in zip(ts, ts[1:]))
    rs = set()
    for _, p, iters, seed in reqs:
        r = p.levels
        rs.add(r)
        assert 2 <= r <= 6 and p.n % (1 << (r - 1)) == 0
        assert (1 << (r - 1)) <= p.n <= 2048 and p.n >= 96
        assert 180 <= p.n_angles <= 2048 and p.n_det == 3 * p.n // 2
        assert 100 <= iters <= 1000 and 0 <= seed < 2 ** 31
    assert rs == {2, 3, 4, 5, 6}
    # log-uniform sides: about as many below sqrt(128 * 2048) = 512 as above
    below = sum(p.n < 512 for _, p, _, _ in reqs)
    assert abs(below / len(reqs) - 0.5) < 0.05
