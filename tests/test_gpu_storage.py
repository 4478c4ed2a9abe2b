"""16-bit SAGA tables (bfloat16 / binary16, measurement- and image-side)
against the oracle's rounded-table iteration, the refinement sweep to fp32 tables, and the memory
they save.

Tolerances (relative L2 of the iterates): binary16 1e-4 as for fp32; bfloat16
2e-3.  The GPU rounds its FP32 projector value and the oracle its FP64 value;
they straddle a bfloat16 rounding boundary with probability about
2e-6 / 2^-8 = 5e-4 per stored entry, and each such entry then differs by one
bfloat16 ulp (2^-8 relative) -- about 3e-4 relative L2 over the 30 iterations
here, so 2e-3 leaves a margin.  For binary16 both factors are 8 times smaller.
"""
import math

import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2412_10249_gb300 import build as pkg_build
from paper_2412_10249_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-4, 1: 2e-3, 2: 1e-4}


@pytest.fixture(scope="module")
def imask():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pkg_build.build()
    from paper_2412_10249_gb300 import imask as m
    m.lib()
    return m


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


FAN64 = inputs.Problem(n=64, n_angles=90, n_det=96, geometry=1, angle_span=2 * math.pi,
                       levels=4)
FAN48 = inputs.Problem(n=48, n_angles=37, n_det=75, geometry=1, angle_span=2 * math.pi,
                       angle_start=0.3, levels=4, probs=[0.3, 0.3, 0.2, 0.2])


@pytest.mark.parametrize("fmt", [1, 2])
@pytest.mark.parametrize("prob,seq", [(FAN64, False), (FAN48, True)], ids=["fan64", "fan48_seq"])
def test_16bit_tables_match_oracle(imask, fmt, prob, seq):
    params = dict(prob.params(), mu=0.1, sigma=0.04)
    _, b, _ = inputs.measurements(prob, seed=1, noise="none")
    o = Oracle(**params)
    st, _, _ = o.run_variant(b.ravel(), 5, 30, sequential=seq, storage=fmt)
    plan = imask.Plan(dict(params, storage=fmt, variant=int(seq), theta=1.0))
    s = plan.state(torch.as_tensor(b.ravel().astype(np.float32), device="cuda"), 5)
    s.step(30)
    ex = rel(s.get(s.X).double().cpu().numpy(), st["x"])
    ey = rel(s.get(s.Y).double().cpu().numpy(), st["y"])
    assert ex <= TOL[fmt] and ey <= TOL[fmt], (ex, ey)


@pytest.mark.parametrize("fmt", [1, 2])
def test_refinement_sweep(imask, fmt):
    prob = FAN64
    params = dict(prob.params(), mu=0.1, sigma=0.04)
    _, b, _ = inputs.measurements(prob, seed=2, noise="none")
    o = Oracle(**params)
    st, _, _ = o.run_variant(b.ravel(), 9, 20, storage=fmt)
    st, _, _ = o.run_variant(b.ravel(), 9, 20, storage=0, state=st)
    plan = imask.Plan(dict(params, storage=fmt))
    s = plan.state(torch.as_tensor(b.ravel().astype(np.float32), device="cuda"), 9)
    s.step(20)
    s.set_storage(0)
    s.step(20)
    ex = rel(s.get(s.X).double().cpu().numpy(), st["x"])
    assert ex <= TOL[fmt], ex
    # the running mean is the p-weighted sum of the (now fp32) tables
    pr = o.probs()
    m = o.m
    psi_mean = sum(pr[l] * st["psi"][l * m:(l + 1) * m] for l in range(o.r))
    assert rel(s.get(s.PSI_MEAN).double().cpu().numpy(), psi_mean) <= TOL[fmt]
    # and so is the image-side running mean of the image-side tables
    d = o.n * o.n
    phi_mean = sum(pr[l] * st["phi"][l * d:(l + 1) * d] for l in range(o.r))
    assert rel(s.get(s.PHI_MEAN).double().cpu().numpy(), phi_mean) <= TOL[fmt]


def test_16bit_tables_save_memory(imask):
    base = dict(FAN64.params(), mu=0.1, sigma=0.04)
    b32 = imask.Plan(base).info["state_bytes"]
    b16 = imask.Plan(dict(base, storage=1)).info["state_bytes"]
    m, r = FAN64.n_angles * FAN64.n_det, FAN64.levels
    # both table families in half the bytes: r m measurement-side entries and
    # n^2 + sum_{l>=1} (n / 2^l)^2 image-side entries
    d_tab = sum((FAN64.n >> l) ** 2 for l in range(r))
    assert b32 - b16 >= 2 * m * r + 2 * d_tab - 256
