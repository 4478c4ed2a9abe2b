"""Host-side logic of the continuous-batching loop, on the CPU with a fake
device backend: every admitted solve advances exactly its iteration count,
the memory budget and slot limit hold, full queues and oversize requests are
rejected, failed plan builds fail only their own requests, and a plan is never
closed while one of its solves runs."""
import numpy as np
import pytest

from paper_2412_10249_gb300 import serve


class _Marker:
    def __init__(self, polls):
        self.left = polls

    def query(self):
        self.left -= 1
        return self.left <= 0


class FakeBackend:
    """Plans cost 1000 n bytes, states 100 n^2; a marker completes after two polls."""

    def __init__(self):
        self.running = {}          # id(plan) -> running solves
        self.closed = []
        self.max_running = 0

    def build_plan(self, params):
        if params["n"] == 99:
            raise serve.PlanBuildError("unsupported size")
        plan = {"n": params["n"]}
        return plan, 1000 * params["n"], 100 * params["n"] ** 2

    def host_sinogram(self, b):
        return np.asarray(b, dtype=np.float32)

    def start(self, plan, host, seed):
        assert all(plan is not c for c in self.closed), "solve started on a closed plan"
        self.running[id(plan)] = self.running.get(id(plan), 0) + 1
        self.max_running = max(self.max_running, sum(self.running.values()))
        return {"plan": plan, "k": 0, "seed": seed}

    def step(self, solve, n):
        solve["k"] += n

    def fetch(self, solve):
        return np.array([solve["k"], solve["seed"]])

    def mark(self, solve):
        return _Marker(2)

    @staticmethod
    def done(marker):
        return marker.query()

    def finish(self, solve):
        self.running[id(solve["plan"])] -= 1

    def close_plan(self, plan):
        assert self.running.get(id(plan), 0) == 0, "plan closed while a solve runs"
        self.closed.append(plan)

    def check_plan(self, plan):
        pass

    def synchronize(self):
        pass


def _req(rid, n, iters, t=0.0, na=4, nd=6):
    params = dict(n=n, n_angles=na, n_det=nd, geometry=1, levels=2)
    return serve.Request(rid=rid, params=params, b=np.zeros(na * nd), iters=iters,
                         seed=100 + rid, arrival=t)


def test_every_solve_runs_its_iterations():
    be = FakeBackend()
    reqs = [_req(i, 8 + 8 * (i % 3), 5 + 7 * i) for i in range(10)]
    srv = serve.Server(budget_bytes=10 ** 9, max_active=3, quantum=4, backend=be)
    st = srv.run(reqs)
    srv.close()
    assert st.completed == 10 and st.max_active <= 3
    for r in reqs:
        assert r.status == "done"
        assert list(r.x) == [r.iters, r.seed]


def test_memory_budget_bounds_concurrency():
    be = FakeBackend()
    reqs = [_req(i, 16, 9) for i in range(6)]
    # one plan (16 000 B) and two states (25 600 B each, plus 4 m bytes of b)
    budget = 16000 + 2 * (25600 + 4 * 24) + 10
    srv = serve.Server(budget_bytes=budget, max_active=6, quantum=3, backend=be)
    st = srv.run(reqs)
    srv.close()
    assert st.completed == 6
    assert st.peak_bytes <= budget and be.max_running <= 2


def test_full_queue_and_oversize_requests_are_rejected():
    be = FakeBackend()
    reqs = [_req(i, 8, 50) for i in range(8)] + [_req(100, 64, 5)]
    srv = serve.Server(budget_bytes=200000, max_active=1, max_queue=4, quantum=10, backend=be)
    for r in reqs:
        srv.offer(r)
    st = srv.run([])
    srv.close()
    assert st.rejected_queue_full == 5          # 4 queued, the rest (and the big one) refused
    assert sum(r.status == "done" for r in reqs) == 4
    srv2 = serve.Server(budget_bytes=200000, max_active=1, quantum=10, backend=FakeBackend())
    st2 = srv2.run([_req(7, 64, 5)])             # state 409 600 B > budget
    srv2.close()
    assert st2.rejected_too_large == 1 and st2.completed == 0


def test_failed_plan_build_fails_only_its_requests():
    be = FakeBackend()
    reqs = [_req(0, 99, 5), _req(1, 8, 5), _req(2, 99, 5), _req(3, 16, 5)]
    srv = serve.Server(budget_bytes=10 ** 9, max_active=2, quantum=5, backend=be)
    st = srv.run(reqs)
    srv.close()
    assert [r.status for r in reqs] == ["failed", "done", "failed", "done"]
    assert st.failed == 2 and len(st.failed_plans) == 1


def test_idle_plans_are_evicted_under_pressure():
    be = FakeBackend()
    # three geometries whose plans do not all fit beside a running state
    reqs = [_req(i, n, 6, t=0.001 * i) for i, n in enumerate([32, 40, 48, 32, 40, 48])]
    budget = 48000 + 100 * 48 ** 2 + 4 * 24 + 40000
    srv = serve.Server(budget_bytes=budget, max_active=1, quantum=3, backend=be)
    st = srv.run(reqs)
    srv.close()
    assert st.completed == 6
    assert st.peak_bytes <= budget
    assert st.plans_built > 3                    # some plans were rebuilt after eviction


def test_cancelled_requests_free_their_slots():
    be = FakeBackend()
    reqs = [_req(i, 8, 40) for i in range(4)]
    srv = serve.Server(budget_bytes=10 ** 9, max_active=2, quantum=4, backend=be)
    for r in reqs:
        srv.offer(r)
    for _ in range(1000):
        srv.poll()
        if reqs[0].status == "active" and reqs[1].status == "active":
            break
    assert reqs[0].status == "active" and reqs[3].status == "queued"
    assert srv.cancel(reqs[3].rid)          # queued: leaves at once
    assert reqs[3].status == "cancelled"
    assert srv.cancel(reqs[0].rid)          # active: stops after its quantum
    assert not srv.cancel(reqs[0].rid)      # already withdrawn
    assert not srv.cancel(12345)            # unknown
    st = srv.run([])
    assert reqs[0].status == "cancelled" and reqs[0].x is None
    assert [r.status for r in reqs[1:3]] == ["done", "done"]
    assert [list(r.x) for r in reqs[1:3]] == [[40, 101], [40, 102]]
    assert st.completed == 2 and st.cancelled == 2
    # only the plan still holds memory; no solve is left running
    assert srv.used == sum(pb for _, pb, _ in srv.plans.values())
    assert sum(be.running.values()) == 0
    srv.close()
