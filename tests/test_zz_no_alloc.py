"""The allocation-free back-projection entry point (imask_backproject_noalloc).

It is for callers that cannot allocate device memory while they run; it must
give the same image as imask_backproject.  Two calls in a row with different
sinograms check that the shared fixed array carries nothing from one call
into the next.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest
import torch

from paper_2412_10249_gb300 import build as pkg_build
from paper_2412_10249_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_OP = 1e-5


@pytest.fixture(scope="module")
def imask():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pkg_build.build()
    from paper_2412_10249_gb300 import imask as m
    m.lib()
    return m


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("params", [
    inputs.Problem(n=48, n_angles=37, n_det=75, geometry=1, angle_span=2 * math.pi,
                   angle_start=0.3, levels=4, mu=1.0, sigma=0.1).params(),
    inputs.fan512_problem(mu=0.25, sigma=0.03).params(),
])
def test_noalloc_matches_backproject_twice(imask, params):
    plan = imask.Plan(params)
    n, m = plan.n, plan.m
    gen = torch.Generator(device="cuda").manual_seed(7)
    for call in range(2):
        y = torch.randn(m, device="cuda", generator=gen)
        for level in range(-1, params["levels"]):
            ref = plan.backproject(level, y)
            out = torch.full((n * n,), float("nan"), device="cuda")
            imask.imask_backproject_noalloc(plan.handle, level, y, out, n, m)
            torch.cuda.synchronize()
            assert torch.isfinite(out).all()
            assert _rel(out, ref) <= TOL_OP, (call, level, _rel(out, ref))
    plan.check()
