"""State checkpoints: a state restored from a checkpoint continues exactly as
the saved one would have (bit-identical iterates), through eager and
graph-replayed steps, for every iteration form; checkpoints of another plan
or corrupted ones are refused."""
import math

import numpy as np
import pytest
import torch

from paper_2412_10249_gb300 import build as pkg_build
from paper_2412_10249_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def imask():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pkg_build.build()
    from paper_2412_10249_gb300 import imask as m
    m.lib()
    return m


def _setup(imask, n=64, **kw):
    p = inputs.Problem(n=n, n_angles=90, n_det=3 * n // 2, geometry=1,
                       angle_span=2 * math.pi, levels=3)
    plan = imask.Plan(dict(p.params(), mu=0.3, sigma=0.03, **kw))
    b = torch.as_tensor(inputs.sinogram(p, 3).ravel().astype(np.float32), device="cuda")
    return plan, b


@pytest.mark.parametrize("kw", [dict(), dict(variant=1), dict(dual_tables=1), dict(storage=1),
                                dict(draws=1), dict(reg=1, tv_lambda=0.03)])
def test_resume_from_a_checkpoint_is_exact(imask, kw):
    plan, b = _setup(imask, **kw)
    a = plan.state(b, 5)
    a.step(13)                     # eager iterations
    a.step(8)                      # graph replays
    ck = a.save()
    c = plan.state(torch.zeros_like(b), 99)
    c.step(3)
    c.load(ck)
    assert c.k == a.k == 21
    a.step(17)
    c.step(17)
    torch.cuda.synchronize()
    assert torch.equal(a.get(a.X), c.get(c.X))
    assert torch.equal(a.get(a.Y), c.get(c.Y))
    assert torch.equal(a.get(a.PSI_MEAN), c.get(c.PSI_MEAN))
    # loading the same checkpoint again rewinds to iteration 21
    c.load(ck)
    assert c.k == 21
    c.step(17)
    torch.cuda.synchronize()
    assert torch.equal(a.get(a.X), c.get(c.X))
    a.close()
    c.close()
    plan.check()


def test_foreign_or_corrupt_checkpoints_are_refused(imask):
    plan, b = _setup(imask)
    a = plan.state(b, 1)
    a.step(5)
    ck = a.save()
    plan2, b2 = _setup(imask, n=32)
    s2 = plan2.state(b2, 1)
    with pytest.raises(ValueError):
        s2.load(ck)                # another plan: the sizes differ
    bad = ck.clone()
    bad[:8] = 0                    # no checkpoint header
    c = plan.state(b, 2)
    with pytest.raises(imask.ImaskError):
        c.load(bad)
    assert c.k == 0
    for s in (a, s2, c):
        s.close()


def test_save_on_a_side_stream_then_step_at_once(imask):
    """A save enqueued on a second stream is ordered before the state's next
    step on the first: the checkpoint is the state at the save, not a torn mix
    of it and the later iterations."""
    plan, b = _setup(imask, n=128)
    a = plan.state(b, 11)
    a.step(10)
    side = torch.cuda.Stream()
    ck = a.save(stream=side)
    a.step(40)                      # on the current stream, enqueued at once
    c = plan.state(torch.zeros_like(b), 12)
    c.load(ck)
    assert c.k == 10
    c.step(40)
    torch.cuda.synchronize()
    assert torch.equal(a.get(a.X), c.get(c.X))
    assert torch.equal(a.get(a.Y), c.get(c.Y))
    for s in (a, c):
        s.close()


def test_checkpoint_of_a_plan_of_the_same_size_is_refused(imask):
    """Two plans whose states have the same size but another mu (hence another
    step size): the plan fingerprint in the header refuses the load."""
    plan, b = _setup(imask)
    a = plan.state(b, 1)
    a.step(5)
    ck = a.save()
    p = inputs.Problem(n=64, n_angles=90, n_det=96, geometry=1, angle_span=2 * math.pi, levels=3)
    other = imask.Plan(dict(p.params(), mu=0.31, sigma=0.03))
    s2 = other.state(b, 1)
    assert int(imask.lib().imask_state_checkpoint_bytes(s2.handle)) == ck.numel()
    with pytest.raises(imask.ImaskError):
        s2.load(ck)
    assert s2.k == 0
    for s in (a, s2):
        s.close()
