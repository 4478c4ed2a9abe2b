"""Failure detection without a GPU fault: a bounded device-side wait that runs
out is reported through the plan's error flag, and non-finite data is caught
by the FP64 reductions."""
import math

import numpy as np
import pytest
import torch

from oracle import Oracle
from paper_2412_10249_gb300 import build as pkg_build
from paper_2412_10249_gb300 import inputs

pytestmark = pytest.mark.gpu

FAN64 = inputs.Problem(n=64, n_angles=90, n_det=96, geometry=1, angle_span=2 * math.pi,
                       levels=4)


@pytest.fixture(scope="module")
def imask():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pkg_build.build()
    from paper_2412_10249_gb300 import imask as m
    m.lib()
    return m


def test_projector_wait_that_runs_out_is_reported(imask):
    params = dict(FAN64.params(), mu=0.1, sigma=0.04)
    plan = imask.Plan(params)
    plan.check()                       # clean to start with
    plan.selftest_timeout()
    with pytest.raises(imask.ImaskError) as ei:
        plan.check()
    assert ei.value.status == 5        # IMASK_ERR_TIMEOUT
    plan.check()                       # the flag was cleared
    # and the plan still computes correctly
    o = Oracle(**params)
    img = inputs.square_phantom(64, 8)
    got = plan.project(0, torch.as_tensor(img.ravel().astype(np.float32), device="cuda"))
    ref = o.K(0, img).ravel()
    assert np.linalg.norm(got.double().cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5


def test_non_finite_data_is_caught(imask):
    plan = imask.Plan(dict(FAN64.params(), mu=0.1, sigma=0.04))
    _, b, _ = inputs.measurements(FAN64, seed=1, noise="none")
    b = b.ravel().astype(np.float32)
    b[123] = np.nan                    # a poisoned measurement
    bt = torch.as_tensor(b, device="cuda")
    x = plan.solve(bt, 0, 10)
    assert torch.isnan(x).any()
    with pytest.raises(imask.ImaskError) as ei:
        plan.objective(x, bt)
    assert ei.value.status == 6        # IMASK_ERR_NONFINITE
    with pytest.raises(imask.ImaskError) as ei:
        imask.imask_rel_distance(x, torch.ones_like(x))
    assert ei.value.status == 6
