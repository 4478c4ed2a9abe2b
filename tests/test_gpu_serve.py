"""The continuous-batching loop: every result equals the same solve run alone;
admission respects the device-memory budget; oversize requests are rejected."""
import math

import numpy as np
import pytest
import torch

from paper_2412_10249_gb300 import build as pkg_build
from paper_2412_10249_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    pkg_build.build()
    from paper_2412_10249_gb300 import imask, serve
    imask.lib()
    return imask, serve


def _requests(serve):
    specs = [(64, 90, 2, 40, 0.0), (96, 120, 3, 60, 0.0), (128, 200, 4, 30, 0.0),
             (64, 90, 2, 50, 0.02), (160, 150, 2, 40, 0.05), (96, 120, 3, 20, 0.05)]
    out = []
    for i, (n, na, r, iters, t) in enumerate(specs):
        p = inputs.Problem(n=n, n_angles=na, n_det=3 * n // 2, geometry=1,
                           angle_span=2 * math.pi, levels=r)
        b = inputs.sinogram(p, 50 + i).ravel().astype(np.float32)
        out.append(serve.Request(rid=i, params=p.params(), b=b, iters=iters, seed=7 + i,
                                 arrival=t))
    return out


def _alone(imask, serve, req):
    plan = imask.Plan(dict(req.params, mu=0.0, sigma=serve.normalised_sigma(req.params["levels"]),
                           power_iters=20))
    x = plan.solve(torch.as_tensor(req.b, device="cuda"), req.seed, req.iters)
    return x.cpu()


def test_results_equal_solves_alone(mods):
    imask, serve = mods
    reqs = _requests(serve)
    srv = serve.Server(budget_bytes=8 << 30, max_active=4, quantum=7)
    st = srv.run(reqs)
    srv.close()
    assert st.completed == len(reqs) and st.max_active >= 2
    for r in reqs:
        assert r.status == "done"
        assert torch.equal(r.x, _alone(imask, serve, r)), r.rid


def test_admission_respects_the_budget(mods):
    imask, serve = mods
    reqs = _requests(serve)
    # room for the plans and about two states at a time
    infos = []
    for r in reqs:
        plan = imask.Plan(dict(r.params, mu=0.3, sigma=0.03))
        infos.append((plan.info["plan_bytes"], plan.info["state_bytes"]))
        plan.close()
    budget = sum(pb for pb, _ in set(infos)) + 2 * max(sb for _, sb in infos) + (4 << 20)
    srv = serve.Server(budget_bytes=budget, max_active=6, quantum=5)
    st = srv.run(reqs)
    srv.close()
    assert st.completed == len(reqs)
    assert st.peak_bytes <= budget
    assert st.max_active <= 3


def test_oversize_request_is_rejected(mods):
    imask, serve = mods
    reqs = _requests(serve)[:2]
    srv = serve.Server(budget_bytes=1 << 20, max_active=2)
    st = srv.run(reqs)
    srv.close()
    assert st.rejected_too_large == 2 and st.completed == 0


def test_cancelled_solve_frees_its_state(mods):
    imask, serve = mods
    reqs = _requests(serve)[:3]
    for r in reqs:
        r.arrival = 0.0
        r.iters = 400               # long enough to still be running when withdrawn
    srv = serve.Server(budget_bytes=8 << 30, max_active=2, quantum=5)
    for r in reqs:
        srv.offer(r)
    for _ in range(100000):
        srv.poll()
        if reqs[0].status == "active" and reqs[1].status == "active":
            break
    assert reqs[0].status == "active" and reqs[2].status == "queued"
    assert srv.cancel(reqs[0].rid)
    st = srv.run([])
    assert reqs[0].status == "cancelled" and reqs[0].x is None
    assert [r.status for r in reqs[1:]] == ["done", "done"]
    assert st.cancelled == 1 and st.completed == 2
    assert srv.used == sum(pb for _, pb, _ in srv.plans.values())
    srv.close()
    for r in reqs[1:]:
        assert torch.equal(r.x, _alone(imask, serve, r)), r.rid


def test_plan_bytes_estimate_bounds_the_plan(mods):
    # the loop reserves the estimate while a plan is being built
    imask, serve = mods
    for r in _requests(serve):
        plan = imask.Plan(dict(r.params, mu=0.3, sigma=0.03))
        assert serve.Server.plan_bytes_estimate(r.params) >= plan.info["plan_bytes"]
        plan.close()


def test_served_results_match_the_oracle(mods):
    # two requests served together (sharing the GPU in the loop), each against
    # the FP64 oracle run with the plan's own mu and sigma on the same seed
    from oracle import Oracle
    imask, serve = mods
    reqs = _requests(serve)[:2]
    srv = serve.Server(budget_bytes=8 << 30, max_active=2, quantum=7)
    st = srv.run(reqs)
    srv.close()
    assert st.completed == 2
    for r in reqs:
        plan = imask.Plan(dict(r.params, mu=0.0, sigma=serve.normalised_sigma(r.params["levels"]),
                               power_iters=20))
        info = plan.info
        plan.close()
        o = Oracle(**dict(r.params, mu=info["mu"], sigma=info["sigma"]))
        ref, _ = o.run(r.b.astype(np.float64), r.seed, r.iters)
        got = r.x.double().numpy()
        err = np.linalg.norm(got - ref["x"]) / np.linalg.norm(ref["x"])
        assert err <= 1e-4, (r.rid, err)
