"""Pins of the oracle's 16-bit table storage: the rounding against library
conversions and its defining properties, and the effect of rounded tables on
the iteration (bounded offset of the fixed point, removed by continuing with
full-precision tables) -- CPU only."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_2412_10249_gb300 import inputs


def _values(seed, n=20000):
    rng = np.random.default_rng(seed)
    mags = 10.0 ** rng.uniform(-9, 4, n)
    return mags * rng.choice([-1.0, 1.0], n)


def test_binary16_rounding_matches_numpy(oracle_lib):
    v = _values(0)
    got = np.array([Oracle.round_format(x, 2) for x in v])
    want = v.astype(np.float16).astype(np.float64)
    np.testing.assert_array_equal(got, want)


def test_bfloat16_rounding_matches_torch(oracle_lib):
    torch = pytest.importorskip("torch")
    v = _values(1).astype(np.float32)          # torch converts from float32
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([Oracle.round_format(float(x), 1) for x in v])
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("fmt,bits,emin", [(1, 8, -126), (2, 11, -14)])
def test_rounding_is_nearest_even(oracle_lib, fmt, bits, emin):
    for x in _values(2, 3000):
        r = Oracle.round_format(x, fmt)
        ex = max(math.floor(math.log2(abs(x))), emin)
        q = 2.0 ** (ex - bits + 1)
        k = r / q
        assert k == round(k)                      # representable
        assert abs(x - r) <= 0.5 * q              # nearest
        if abs(abs(x - r) - 0.5 * q) == 0.0:      # a tie goes to the even multiple
            assert int(k) % 2 == 0
    # exact ties
    q1 = 2.0 ** (-bits + 1)
    assert Oracle.round_format(1.0 + 0.5 * q1, fmt) == 1.0
    assert Oracle.round_format(1.0 + 1.5 * q1, fmt) == 1.0 + 2 * q1


def _case():
    p = inputs.Problem(n=16, n_angles=12, n_det=24, geometry=1, angle_span=2 * math.pi,
                       levels=4)
    o = Oracle(**dict(p.params(), mu=1.0, sigma=0.05))
    mu = o.norm_K(200) ** 2 / 2.46 ** 2
    o.set(mu=mu)
    b = o.K(-1, inputs.square_phantom(16, 8)).ravel()
    xn, _ = o.solve_quadratic(b)
    return o, b, xn.ravel()


def test_full_precision_storage_is_alg1(oracle_lib):
    o, b, _ = _case()
    a, _ = o.run(b, 3, 40)
    v, _, _ = o.run_variant(b, 3, 40, storage=0)
    assert np.array_equal(a["x"], v["x"])


@pytest.mark.parametrize("fmt,bound", [(1, 2e-2), (2, 3e-3)])
def test_rounded_tables_offset_then_refinement(oracle_lib, fmt, bound):
    # with rounded tables the iteration settles near x_nat, offset by about
    # the format's relative precision; continuing with full-precision tables
    # (the refinement sweep) reaches x_nat
    o, b, xn = _case()
    st, _, _ = o.run_variant(b, 0, 900, storage=fmt)
    e16 = np.linalg.norm(st["x"] - xn) / np.linalg.norm(xn)
    assert 1e-7 < e16 < bound
    st, _, _ = o.run_variant(b, 0, 900, storage=0, state=st)
    e32 = np.linalg.norm(st["x"] - xn) / np.linalg.norm(xn)
    assert e32 < 1e-8
