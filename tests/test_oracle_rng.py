"""Pins of the oracle's level draw (Alg. 1, sampling step) -- CPU only."""
import os

import numpy as np
import pytest

from oracle import Oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_splitmix():
    out = []
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out.append((int(k), int(v, 16)))
    return out


def test_splitmix64_published_outputs(oracle_lib):
    o = Oracle(n=8, n_angles=1, n_det=1)
    for k, v in _golden_splitmix():
        assert o.splitmix64_at(0, k) == v


def test_thresholds_uniform_exact(oracle_lib):
    # uniform p: thresholds are (l + 1) / r of 2^64 where that is exact in 53 bits
    o = Oracle(n=8, n_angles=1, n_det=1, levels=2)
    assert list(o.thresholds()) == [1 << 63]
    o = Oracle(n=8, n_angles=1, n_det=1, levels=4)
    assert list(o.thresholds()) == [1 << 62, 2 << 62, 3 << 62]


@pytest.mark.parametrize("probs", [None, [0.2, 0.3, 0.3, 0.2], [0.5, 0.25, 0.125, 0.125]])
def test_level_frequencies_within_4_sigma(oracle_lib, probs):
    o = Oracle(n=8, n_angles=1, n_det=1, levels=4, probs=probs)
    n = 1_000_000
    lv = o.levels(12345, 0, n)
    p = o.probs()
    cnt = np.bincount(lv, minlength=4)
    sd = np.sqrt(n * p * (1 - p))
    assert np.all(np.abs(cnt - n * p) <= 4 * sd), (cnt, n * p)


def test_level_stream_is_counter_based(oracle_lib):
    # resuming at position k gives the same draws as running from 0
    o = Oracle(n=8, n_angles=1, n_det=1, levels=3)
    full = o.levels(7, 0, 1000)
    part = o.levels(7, 600, 400)
    assert np.array_equal(full[600:], part)
    # a different seed gives a different stream
    assert not np.array_equal(full, o.levels(8, 0, 1000))


def test_single_level_always_zero(oracle_lib):
    o = Oracle(n=8, n_angles=1, n_det=1, levels=1)
    assert np.all(o.levels(3, 0, 1000) == 0)
