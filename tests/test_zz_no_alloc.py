"""The allocation-free back-projection entry point (imask_backproject_noalloc).

It is for callers that cannot allocate device memory while they run; it must
give the same image as imask_backproject, bit for bit (the same kernels run
in the same order, only the partial sums live in a fixed array instead of a
buffer from cudaMallocAsync).  Two calls in a row with different sinograms
check that the shared fixed array carries nothing from one call into the
next.  A second test reads the device's default memory pool (the pool that
cudaMallocAsync draws from) through the driver API and checks that a run of
calls leaves its high-water mark where it was, while imask_backproject, the
allocating entry point, does raise it.  This file is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_2412_10249_gb300 import build as pkg_build
from paper_2412_10249_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_OP = 1e-5
# CUmemPool_attribute values (cuda.h)
ATTR_USED_MEM_CURRENT = 7
ATTR_USED_MEM_HIGH = 8


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
            assert torch.equal(out, ref), (call, level, _rel(out, ref))
    plan.check()


class _DefaultPool:
    """The current device's default memory pool, read through libcuda."""

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int(0)
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        # setting the high-water mark to 0 resets it to the current use
        v = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, ATTR_USED_MEM_HIGH, ctypes.byref(v)) == 0


def test_noalloc_draws_nothing_from_the_memory_pool(imask):
    p = inputs.Problem(n=64, n_angles=90, n_det=96, geometry=1, angle_span=2 * math.pi,
                       levels=3, mu=1.0, sigma=0.1)
    plan = imask.Plan(p.params())
    n, m = plan.n, plan.m
    y = torch.randn(m, device="cuda")
    out = torch.empty(n * n, device="cuda")
    # the first call on the device looks up the array's address
    imask.imask_backproject_noalloc(plan.handle, 0, y, out, n, m)
    torch.cuda.synchronize()
    pool = _DefaultPool()
    pool.reset_high()
    used0 = pool.get(ATTR_USED_MEM_CURRENT)
    assert pool.get(ATTR_USED_MEM_HIGH) == used0
    for _ in range(3):
        for level in range(-1, p.levels):
            imask.imask_backproject_noalloc(plan.handle, level, y, out, n, m)
    torch.cuda.synchronize()
    assert pool.get(ATTR_USED_MEM_HIGH) == used0
    assert pool.get(ATTR_USED_MEM_CURRENT) == used0
    # the allocating entry point does move the high-water mark: the check sees it
    plan.backproject(1, y)
    torch.cuda.synchronize()
    assert pool.get(ATTR_USED_MEM_HIGH) > used0
    plan.check()
