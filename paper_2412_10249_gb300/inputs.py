"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds none of the method's arithmetic: it draws random-ellipse
phantoms, rasterises them by supersampling, computes their *analytic*
line integrals (the exact measurement model, not the discretised projector),
and adds measurement noise.  The ellipse phantoms stand in for the XCAT and
AAPM slices of the paper's experiments (Sec. 4), which are not available here.

Recipe (seed s; numpy PCG64 streams s for the phantom and s + 1 for the noise):
  * E ellipses (10, or 16 at N >= 1024); semi-axes uniform in [0.03, 0.25] W;
    centres uniform in the disk of radius 0.45 W (1 - max axis / W), so that the
    object stays inside the fan of the default fan geometry; rotation uniform
    in [0, pi); density uniform in [0, 1]; overlapping ellipses add.
  * Raster: the fraction of 4 x 4 sub-pixel centres inside each ellipse.
  * Data: the exact chord length of every ray through every ellipse times its
    density (no inverse crime).
  * Noise: Gaussian with std = rel * max|b|, or Poisson counts with I0 photons
    (counts ~ Poisson(I0 exp(-b)), b = -log(max(counts, 1) / I0)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np


@dataclass
class Problem:
    """Geometry and solver fields of one reconstruction problem."""
    n: int
    n_angles: int
    n_det: int
    geometry: int = 0            # 0 parallel, 1 fan (flat detector)
    fov: float = 1.0
    det_spacing: float = 0.0     # <= 0: default pitch
    angle_start: float = 0.0
    angle_span: float = math.pi
    src_dist: float = 2.0
    det_dist: float = 1.0
    levels: int = 1
    probs: list | None = None
    reg: int = 0                 # 0 quadratic, 1 quadratic + smoothed TV
    mu: float = 1.0
    tv_lambda: float = 0.0
    tv_eps: float = 1e-2
    tv_inner: int = 20
    sigma: float = 0.0

    def params(self) -> dict:
        return asdict(self)

    @property
    def m(self) -> int:
        return self.n_angles * self.n_det

    @property
    def d(self) -> int:
        return self.n * self.n

    def pitch(self) -> float:
        if self.det_spacing > 0:
            return self.det_spacing
        h = self.fov / self.n
        return h if self.geometry == 0 else h * (self.src_dist + self.det_dist) / self.src_dist


# The workloads.  "small" is the 64x64 parallel-beam case with two levels and
# the smoothed-TV regulariser; "fan512" is the 512x512 fan-beam case (720 views
# over 2 pi, 768 bins, source 2W / detector 1W from the centre, four levels,
# quadratic regulariser, 500 iterations) on which throughput is measured.
def small_problem(**kw) -> Problem:
    p = Problem(n=64, n_angles=60, n_det=92, geometry=0, angle_span=math.pi, levels=2,
                reg=1, mu=1.0, tv_lambda=0.1, tv_eps=1e-2, tv_inner=20)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def fan512_problem(**kw) -> Problem:
    p = Problem(n=512, n_angles=720, n_det=768, geometry=1, angle_span=2 * math.pi,
                src_dist=2.0, det_dist=1.0, levels=4, reg=0, mu=1.0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------------------------
# Phantoms
# ---------------------------------------------------------------------------------

def random_ellipses(seed: int, n_ellipses: int = 10, fov: float = 1.0) -> np.ndarray:
    """(E, 6) array of [cx, cy, a, b, alpha, rho]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.zeros((n_ellipses, 6))
    for e in range(n_ellipses):
        a, b = rng.uniform(0.03, 0.25, size=2) * fov
        rad = 0.45 * fov * (1.0 - max(a, b) / fov)
        # uniform in the disk
        rr = rad * math.sqrt(rng.uniform())
        ph = rng.uniform(0.0, 2 * math.pi)
        alpha = rng.uniform(0.0, math.pi)
        rho = rng.uniform(0.0, 1.0)
        out[e] = [rr * math.cos(ph), rr * math.sin(ph), a, b, alpha, rho]
    return out


def rasterize(ell: np.ndarray, n: int, fov: float = 1.0, supersample: int = 4) -> np.ndarray:
    """Row-major (n, n) image; pixel (i, c) centred at (-W/2+(c+1/2)h, -W/2+(i+1/2)h)."""
    h = fov / n
    img = np.zeros((n, n))
    sub = (np.arange(supersample) + 0.5) / supersample
    centres = -0.5 * fov + np.arange(n) * h
    for row_block in range(0, n, 64):
        rows = np.arange(row_block, min(n, row_block + 64))
        ys = (centres[rows][:, None] + sub[None, :] * h).reshape(-1)      # (R*S,)
        xs = (centres[:, None] + sub[None, :] * h).reshape(-1)            # (n*S,)
        X, Y = np.meshgrid(xs, ys)                                         # (R*S, n*S)
        acc = np.zeros_like(X)
        for cx, cy, a, b, al, rho in ell:
            ca, sa = math.cos(al), math.sin(al)
            u = (X - cx) * ca + (Y - cy) * sa
            v = -(X - cx) * sa + (Y - cy) * ca
            acc += rho * ((u / a) ** 2 + (v / b) ** 2 <= 1.0)
        acc = acc.reshape(len(rows), supersample, n, supersample).mean(axis=(1, 3))
        img[rows] = acc
    return img


def phantom(seed: int, n: int, fov: float = 1.0, n_ellipses: int | None = None):
    if n_ellipses is None:
        n_ellipses = 16 if n >= 1024 else 10
    e = random_ellipses(seed, n_ellipses, fov)
    return e, rasterize(e, n, fov)


def square_phantom(n: int, block: int, value: float = 1.0) -> np.ndarray:
    """A centred square insert whose edges lie on multiples of ``block`` pixels."""
    img = np.zeros((n, n))
    lo = (n // 4) // block * block
    hi = (3 * n // 4 + block - 1) // block * block
    img[lo:hi, lo:hi] = value
    return img


# ---------------------------------------------------------------------------------
# Exact line integrals of ellipse phantoms
# ---------------------------------------------------------------------------------

def ray_endpoints(p: Problem):
    """Per ray (a, j): a point on the ray and its unit direction, shapes (m, 2)."""
    a = np.arange(p.n_angles)[:, None].astype(np.float64)
    j = np.arange(p.n_det)[None, :].astype(np.float64)
    ang = p.angle_start + p.angle_span * a / p.n_angles
    s = (j - 0.5 * (p.n_det - 1)) * p.pitch()
    ca, sa = np.cos(ang), np.sin(ang)
    if p.geometry == 0:
        px, py = s * ca, s * sa
        dx, dy = -sa + 0 * s, ca + 0 * s
    else:
        sx, sy = p.src_dist * ca, p.src_dist * sa
        qx = -p.det_dist * ca - s * sa
        qy = -p.det_dist * sa + s * ca
        px, py = sx + 0 * s, sy + 0 * s
        dx, dy = qx - sx, qy - sy
    nrm = np.hypot(dx, dy)
    P = np.stack([px.ravel(), py.ravel()], axis=1)
    D = np.stack([(dx / nrm).ravel(), (dy / nrm).ravel()], axis=1)
    return P, D


def ellipse_sinogram(ell: np.ndarray, p: Problem) -> np.ndarray:
    """Exact line integrals, shape (n_angles, n_det)."""
    P, D = ray_endpoints(p)
    out = np.zeros(P.shape[0])
    for cx, cy, a, b, al, rho in ell:
        ca, sa = math.cos(al), math.sin(al)
        # ellipse frame, scaled to the unit circle
        ox, oy = P[:, 0] - cx, P[:, 1] - cy
        q0x = (ox * ca + oy * sa) / a
        q0y = (-ox * sa + oy * ca) / b
        qdx = (D[:, 0] * ca + D[:, 1] * sa) / a
        qdy = (-D[:, 0] * sa + D[:, 1] * ca) / b
        A = qdx * qdx + qdy * qdy
        B = 2.0 * (q0x * qdx + q0y * qdy)
        C = q0x * q0x + q0y * q0y - 1.0
        disc = B * B - 4.0 * A * C
        chord = np.where(disc > 0.0, np.sqrt(np.maximum(disc, 0.0)) / A, 0.0)
        out += rho * chord
    return out.reshape(p.n_angles, p.n_det)


# ---------------------------------------------------------------------------------
# Noise
# ---------------------------------------------------------------------------------

def gaussian_noise(b: np.ndarray, rel: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return b + rng.normal(0.0, rel * float(np.abs(b).max()), size=b.shape)


def poisson_log(b: np.ndarray, i0: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.poisson(i0 * np.exp(-b))
    return -np.log(np.maximum(counts, 1) / i0)


def sinogram(p: Problem, seed: int, noise: str = "auto") -> np.ndarray:
    """The noisy sinogram of ``measurements`` without rasterising the phantom."""
    n_e = 16 if p.n >= 1024 else 10
    clean = ellipse_sinogram(random_ellipses(seed, n_e, p.fov), p)
    if noise == "auto":
        noise = "gauss" if p.geometry == 0 else "poisson"
    if noise == "gauss":
        return gaussian_noise(clean, 0.01, seed + 1)
    if noise == "poisson":
        return poisson_log(clean, 1e4, seed + 1)
    return clean


def slice_mix(n_slices: int, seed: int):
    """Mixed-size fan-beam slices: side from {256, 384, 512, 768, 1024}, view
    count from {180, 360, 720, 1080, 1440} (uniform draws), 1.5 x side bins,
    geometry as the 512x512 workload (source 2W, detector 1W, 2 pi), 4 levels."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sides = [256, 384, 512, 768, 1024]
    views = [180, 360, 720, 1080, 1440]
    out = []
    for _ in range(n_slices):
        n = int(sides[rng.integers(len(sides))])
        na = int(views[rng.integers(len(views))])
        out.append(Problem(n=n, n_angles=na, n_det=3 * n // 2, geometry=1,
                           angle_span=2 * math.pi, src_dist=2.0, det_dist=1.0, levels=4))
    return out


def disk_sinogram(p: Problem, radius: float = 0.3, density: float = 1.0) -> np.ndarray:
    """Exact line integrals of a centred uniform disk: 2 rho sqrt(R^2 - s^2),
    s the distance of the ray from the centre (cheap for very large m)."""
    P, D = ray_endpoints(p)
    s = P[:, 0] * D[:, 1] - P[:, 1] * D[:, 0]
    return (2.0 * density * np.sqrt(np.maximum(radius * radius - s * s, 0.0))).reshape(
        p.n_angles, p.n_det)


def _serving_geometry(rng, max_side: int) -> Problem:
    r = int(rng.integers(2, 7))
    blk = 1 << (r - 1)
    n = int(round(math.exp(rng.uniform(math.log(128), math.log(max_side))) / blk)) * blk
    n = max(blk, min(n, max_side))
    na = int(rng.integers(180, 2049))
    return Problem(n=n, n_angles=na, n_det=3 * n // 2, geometry=1, angle_span=2 * math.pi,
                   src_dist=2.0, det_dist=1.0, levels=r)


def serving_requests(duration: float, rate: float, seed: int, max_side: int = 2048,
                     n_geometries: int = 0):
    """Poisson arrivals (mean `rate` per second) over `duration` seconds; per
    request: levels r uniform in {2..6}, side N log-uniform in [128, max_side]
    rounded to a multiple of 2^(r-1), views uniform in [180, 2048], bins 1.5 N,
    fan beam as the 512x512 workload, iterations uniform in [100, 1000], a
    seed.  With n_geometries > 0, that many geometries are drawn first (same
    distribution) and every request takes one of them uniformly (a scanner
    fleet with a few protocols); else every request draws its own.  Returns a
    list of (arrival, Problem, iters, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fleet = [_serving_geometry(rng, max_side) for _ in range(n_geometries)]
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        p = fleet[int(rng.integers(0, len(fleet)))] if fleet else _serving_geometry(rng, max_side)
        out.append((t, p, int(rng.integers(100, 1001)), int(rng.integers(0, 2 ** 31))))


def measurements(p: Problem, seed: int, noise: str = "auto"):
    """(phantom image, noisy sinogram b, clean sinogram) for problem ``p``."""
    e, img = phantom(seed, p.n, p.fov)
    clean = ellipse_sinogram(e, p)
    if noise == "auto":
        noise = "gauss" if p.geometry == 0 else "poisson"
    if noise == "gauss":
        b = gaussian_noise(clean, 0.01, seed + 1)
    elif noise == "poisson":
        b = poisson_log(clean, 1e4, seed + 1)
    else:
        b = clean.copy()
    return img, b, clean
