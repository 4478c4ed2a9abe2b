"""Continuous-batching request loop over the C ABI.

Requests (one ImaSk solve each: geometry, levels, iteration count, seed and a
sinogram) arrive over time.  A queued request is first prepared on a worker
thread (its plan, cached per geometry, and its sinogram if it comes as a
callable); the library's calls release the interpreter lock, so preparation
overlaps with the device work.  The loop admits prepared requests while a slot
is free and the device-memory budget holds the request's state (plans count
against the budget too; idle plans are evicted least recently used).  Every
admitted solve runs on its own CUDA stream, so solves that arrive while others
are on the device overlap with them.  A solve advances in quanta of iterations;
after the last quantum its iterate is copied to pinned host memory and its
state is freed.  Latency is measured from arrival to that host copy.  A
request can be withdrawn while it waits or runs (Server.cancel): a running
solve stops at the end of its quantum in flight and frees its state.

All arithmetic runs in the library's kernels; this module only schedules.
The device operations sit behind a backend object (CudaBackend by default),
so that the scheduling itself can be exercised without a GPU.
mu comes from the plan's power method; sigma is the Thm. 3 step for the
normalised constants of r uniform levels (L = 2.46, Lbar = L / sqrt(r),
Lbar_p = L), which the mu normalisation makes common to all geometries.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import math
import threading
import time
from dataclasses import dataclass, field
from typing import Callable

import numpy as np


@dataclass
class Request:
    rid: int
    params: dict                      # imask descriptor fields (geometry, levels, ...)
    b: np.ndarray | Callable          # float32 sinogram (n_angles * n_det), or a maker
    iters: int
    seed: int
    arrival: float = 0.0              # seconds after the start of the run
    # filled by the server
    admitted: float = math.nan
    finished: float = math.nan
    x: object = None                  # host copy of the result (pinned tensor on CUDA)
    status: str = "pending"           # pending, queued, active, done, rejected, failed,
                                      # cancelled


@dataclass
class _Active:
    req: Request
    plan_key: tuple
    solve: object          # the backend's handle of one running solve
    remaining: int
    bytes: int
    event: object = None   # the backend's completion marker of the last work
    finishing: bool = False
    cancelled: bool = False


def geometry_key(params: dict) -> tuple:
    keys = ("n", "n_angles", "n_det", "geometry", "fov", "det_spacing", "angle_start",
            "angle_span", "src_dist", "det_dist", "levels", "reg")
    return tuple(params.get(k) for k in keys)


_SIGMA_CACHE: dict = {}


def normalised_sigma(levels: int) -> float:
    if levels not in _SIGMA_CACHE:
        from . import imask
        L = 2.46
        _SIGMA_CACHE[levels] = imask.imask_optimal_step(L, L / math.sqrt(levels), L,
                                                        1.0 / levels)[0]
    return _SIGMA_CACHE[levels]


class PlanBuildError(RuntimeError):
    """A plan could not be built; the requests of its geometry fail."""


class CudaBackend:
    """Device side of the loop: plans, states and streams of the library."""

    def __init__(self, power_iters: int = 20):
        import torch
        from . import imask
        self.torch, self.imask = torch, imask
        self.power_iters = power_iters
        self.device = torch.cuda.current_device()

    def build_plan(self, params: dict):
        """(plan, plan bytes, state bytes); runs on a worker thread."""
        self.torch.cuda.set_device(self.device)
        try:
            plan = self.imask.Plan(dict(params, mu=0.0, sigma=normalised_sigma(params["levels"]),
                                        power_iters=self.power_iters))
        except self.imask.ImaskError as e:
            raise PlanBuildError(str(e)) from e
        info = plan.info
        return plan, int(info["plan_bytes"]), int(info["state_bytes"])

    def host_sinogram(self, b):
        return self.torch.from_numpy(np.ascontiguousarray(b, dtype=np.float32).ravel()).pin_memory()

    def start(self, plan, host, seed: int):
        torch = self.torch
        stream = torch.cuda.Stream()
        b_dev = torch.empty(host.numel(), device="cuda", dtype=torch.float32)
        with torch.cuda.stream(stream):
            b_dev.copy_(host, non_blocking=True)
            state = plan.state(b_dev, seed, stream=stream)
        return (stream, state, b_dev)

    def step(self, solve, n: int):
        stream, state, _ = solve
        with self.torch.cuda.stream(stream):
            state.step(n, stream=stream)

    def fetch(self, solve):
        """Starts the copy of the iterate to host memory; returns the host buffer."""
        torch = self.torch
        stream, state, _ = solve
        with torch.cuda.stream(stream):
            x_dev = state.get(state.X, stream=stream)
            host = torch.empty(x_dev.numel(), dtype=torch.float32, pin_memory=True)
            host.copy_(x_dev, non_blocking=True)
        return host

    def mark(self, solve):
        ev = self.torch.cuda.Event()
        ev.record(solve[0])
        return ev

    @staticmethod
    def done(marker) -> bool:
        return marker.query()

    def finish(self, solve):
        solve[1].close()

    def close_plan(self, plan):
        plan.close()

    def check_plan(self, plan):
        plan.check()

    def synchronize(self):
        self.torch.cuda.synchronize()


@dataclass
class ServerStats:
    admitted: int = 0
    rejected_queue_full: int = 0
    rejected_too_large: int = 0
    completed: int = 0
    max_active: int = 0
    peak_bytes: int = 0
    plans_built: int = 0
    plan_seconds: float = 0.0
    failed: int = 0
    cancelled: int = 0
    failed_plans: list = field(default_factory=list)
    latencies: list = field(default_factory=list)
    waits: list = field(default_factory=list)


class Server:
    def __init__(self, budget_bytes: int, max_active: int = 16, max_queue: int = 64,
                 quantum: int = 10, power_iters: int = 20, workers: int = 2, backend=None):
        self.budget = int(budget_bytes)
        self.max_active = max_active
        self.max_queue = max_queue
        self.quantum = quantum
        self.backend = backend if backend is not None else CudaBackend(power_iters)
        self.plans: collections.OrderedDict = collections.OrderedDict()   # key -> (plan, bytes)
        self.plan_users: collections.Counter = collections.Counter()
        self.building: dict = {}          # key -> future of the plan
        self.reserved: dict = {}          # key -> bytes reserved for a plan being built
        self.prepared: dict = {}          # rid -> future of the host sinogram
        self.queue: list = []
        self.active: list[_Active] = []
        self.used = 0
        self.stats = ServerStats()
        self.lock = threading.Lock()
        self.pool = cf.ThreadPoolExecutor(max_workers=workers)
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # -- preparation (worker threads) ----------------------------------------------
    def _build_plan(self, params: dict):
        t = time.perf_counter()
        out = self.backend.build_plan(params)
        with self.lock:
            self.stats.plan_seconds += time.perf_counter() - t
            self.stats.plans_built += 1
        return out

    def _make_b(self, req: Request):
        b = req.b() if callable(req.b) else req.b
        return self.backend.host_sinogram(b)

    @staticmethod
    def plan_bytes_estimate(params: dict) -> int:
        # the plan's device tables: 24 bytes per ray, 32 per view, an error
        # flag, the back-projector's tile order (under 4 x 2 n^2/512 bytes),
        # its per-axis view lists and the view-group bounds of every level
        na = int(params["n_angles"])
        m = na * int(params["n_det"])
        n = int(params["n"])
        groups = 8 * na + 8 * (int(params.get("levels", 1)) + 1) * (na + 1)
        return 24 * m + 32 * na + 4 + 16 * (n // 16 + 1) * (n // 32 + 1) + groups

    def _prepare(self, req: Request) -> bool:
        """Starts the plan build (memory permitting) and the sinogram; False
        when the request can never fit."""
        key = geometry_key(req.params)
        if key not in self.plans and key not in self.building:
            est = self.plan_bytes_estimate(req.params)
            if est > self.budget:
                return False
            if self.used + est > self.budget:
                self._evict_idle_plans(est, None)
            if self.used + est > self.budget:
                return True   # wait for memory
            self.used += est
            self.reserved[key] = est
            self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)
            self.building[key] = self.pool.submit(self._build_plan, req.params)
        if req.rid not in self.prepared:
            self.prepared[req.rid] = self.pool.submit(self._make_b, req)
        return True

    def _collect_plans(self):
        for key, fut in list(self.building.items()):
            if fut.done():
                del self.building[key]
                est = self.reserved.pop(key)
                try:
                    plan, pb, sb = fut.result()
                except PlanBuildError as e:
                    # the requests of this geometry fail; the loop carries on
                    self.used -= est
                    self.stats.failed_plans.append((key, str(e)))
                    for req in [r for r in self.queue if geometry_key(r.params) == key]:
                        self.queue.remove(req)
                        self.prepared.pop(req.rid, None)
                        req.status = "failed"
                        self.stats.failed += 1
                    continue
                self.plans[key] = (plan, pb, sb)
                self.used += pb - est
                self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)

    def _evict_idle_plans(self, need: int, keep: tuple):
        for key in list(self.plans.keys()):
            if self.used + need <= self.budget:
                return
            if key != keep and self.plan_users[key] == 0:
                plan, pb, _ = self.plans.pop(key)
                self.backend.close_plan(plan)
                self.used -= pb

    # -- scheduling ----------------------------------------------------------------
    def offer(self, req: Request) -> bool:
        if len(self.queue) >= self.max_queue:
            req.status = "rejected"
            self.stats.rejected_queue_full += 1
            return False
        req.status = "queued"
        self.queue.append(req)
        return True

    def cancel(self, rid: int) -> bool:
        """Withdraws request `rid` (call from the thread that polls).  A queued
        request leaves the queue; an active solve stops at the end of the
        quantum in flight, without a result, and its state is freed.  False if
        the request is not queued or active, or its result is already being
        copied out."""
        for req in self.queue:
            if req.rid == rid:
                self.queue.remove(req)
                self.prepared.pop(rid, None)
                req.status = "cancelled"
                self.stats.cancelled += 1
                return True
        for a in self.active:
            if a.req.rid == rid and not a.cancelled and not a.finishing:
                a.cancelled = True
                return True
        return False

    def _admit(self):
        self._collect_plans()
        for req in list(self.queue[: 2 * self.max_active]):
            if not self._prepare(req):
                self.queue.remove(req)
                req.status = "rejected"
                self.stats.rejected_too_large += 1
        remaining = []
        blocked = False
        for req in self.queue:
            key = geometry_key(req.params)
            fut_b = self.prepared.get(req.rid)
            if blocked or len(self.active) >= self.max_active or key not in self.plans \
                    or fut_b is None or not fut_b.done():
                remaining.append(req)
                continue
            plan, pb, sb = self.plans[key]
            m = int(req.params["n_angles"]) * int(req.params["n_det"])
            need = sb + 4 * m
            if pb + need > self.budget:
                req.status = "rejected"
                self.stats.rejected_too_large += 1
                self.prepared.pop(req.rid, None)
                continue
            if self.used + need > self.budget:
                self._evict_idle_plans(need, key)
            if self.used + need > self.budget:
                blocked = True   # first in line that does not fit: wait for memory
                remaining.append(req)
                continue
            self.plans.move_to_end(key)
            host = self.prepared.pop(req.rid).result()
            solve = self.backend.start(plan, host, req.seed)
            self.plan_users[key] += 1
            self.used += need
            self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)
            req.admitted = self.now()
            req.status = "active"
            self.active.append(_Active(req, key, solve, req.iters, need))
            self.stats.admitted += 1
            self.stats.max_active = max(self.stats.max_active, len(self.active))
        self.queue = remaining

    def _advance(self):
        be = self.backend
        for a in self.active:
            if a.finishing or (a.event is not None and not be.done(a.event)):
                continue
            if a.cancelled:
                a.finishing = True   # nothing more is launched; no result is read
            elif a.remaining > 0:
                q = min(self.quantum, a.remaining)
                be.step(a.solve, q)
                a.remaining -= q
            else:
                a.req.x = be.fetch(a.solve)
                a.finishing = True
            a.event = be.mark(a.solve)

    def _retire(self):
        keep = []
        for a in self.active:
            if a.finishing and self.backend.done(a.event):
                a.req.finished = self.now()
                if a.cancelled:
                    a.req.status = "cancelled"
                    self.stats.cancelled += 1
                else:
                    a.req.status = "done"
                    self.stats.completed += 1
                    self.stats.latencies.append(a.req.finished - a.req.arrival)
                    self.stats.waits.append(a.req.admitted - a.req.arrival)
                self.backend.finish(a.solve)
                self.plan_users[a.plan_key] -= 1
                self.used -= a.bytes
            else:
                keep.append(a)
        self.active = keep

    def poll(self):
        self._admit()
        self._advance()
        self._retire()

    def idle(self) -> bool:
        return not self.queue and not self.active

    def run(self, requests, duration: float | None = None, drain: bool = True):
        """Offers `requests` at their arrival times (seconds after the start) and
        serves until every offered request is done or rejected; with
        drain=False, stops once `duration` has passed.  Returns the stats."""
        pending = sorted(requests, key=lambda r: r.arrival)
        i = 0
        self.t0 = time.perf_counter()
        while True:
            t = self.now()
            while i < len(pending) and pending[i].arrival <= t:
                self.offer(pending[i])
                i += 1
            self.poll()
            if i >= len(pending) and self.idle():
                break
            if not drain and duration is not None and t >= duration:
                break
            if not self.active and not self.queue and i < len(pending):
                time.sleep(max(0.0, min(0.001, pending[i].arrival - t)))
        self.backend.synchronize()
        for plan, _, _ in self.plans.values():
            self.backend.check_plan(plan)
        return self.stats

    def close(self):
        self.backend.synchronize()
        for a in self.active:
            self.backend.finish(a.solve)
        self.active = []
        for fut in self.building.values():
            try:
                plan, _, _ = fut.result()
            except PlanBuildError:
                continue
            self.backend.close_plan(plan)
        self.building.clear()
        self.pool.shutdown(wait=True)
        for plan, _, _ in self.plans.values():
            self.backend.close_plan(plan)
        self.plans.clear()
