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
state is freed.  Latency is measured from arrival to that host copy.

All arithmetic runs in the library's kernels; this module only schedules.
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
import torch

from . import imask


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
    x: torch.Tensor | None = None     # pinned host copy of the result
    status: str = "pending"           # pending, queued, active, done, rejected, failed


@dataclass
class _Active:
    req: Request
    plan_key: tuple
    stream: torch.cuda.Stream
    state: imask.State
    b_dev: torch.Tensor
    remaining: int
    bytes: int
    event: torch.cuda.Event | None = None
    finishing: bool = False


def geometry_key(params: dict) -> tuple:
    keys = ("n", "n_angles", "n_det", "geometry", "fov", "det_spacing", "angle_start",
            "angle_span", "src_dist", "det_dist", "levels", "reg")
    return tuple(params.get(k) for k in keys)


_SIGMA_CACHE: dict = {}


def normalised_sigma(levels: int) -> float:
    if levels not in _SIGMA_CACHE:
        L = 2.46
        _SIGMA_CACHE[levels] = imask.imask_optimal_step(L, L / math.sqrt(levels), L,
                                                        1.0 / levels)[0]
    return _SIGMA_CACHE[levels]


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
    failed_plans: list = field(default_factory=list)
    latencies: list = field(default_factory=list)
    waits: list = field(default_factory=list)


class Server:
    def __init__(self, budget_bytes: int, max_active: int = 16, max_queue: int = 64,
                 quantum: int = 10, power_iters: int = 20, workers: int = 2):
        self.budget = int(budget_bytes)
        self.max_active = max_active
        self.max_queue = max_queue
        self.quantum = quantum
        self.power_iters = power_iters
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
        self.device = torch.cuda.current_device()
        self.t0 = time.perf_counter()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    # -- preparation (worker threads) ----------------------------------------------
    def _build_plan(self, params: dict):
        torch.cuda.set_device(self.device)
        t = time.perf_counter()
        plan = imask.Plan(dict(params, mu=0.0, sigma=normalised_sigma(params["levels"]),
                               power_iters=self.power_iters))
        info = plan.info
        with self.lock:
            self.stats.plan_seconds += time.perf_counter() - t
            self.stats.plans_built += 1
        return plan, int(info["plan_bytes"]), int(info["state_bytes"])

    @staticmethod
    def _make_b(req: Request):
        b = req.b() if callable(req.b) else req.b
        return torch.from_numpy(np.ascontiguousarray(b, dtype=np.float32).ravel()).pin_memory()

    @staticmethod
    def plan_bytes_estimate(params: dict) -> int:
        # the plan's device tables: 24 bytes per ray, 32 per view, an error
        # flag, and the back-projector's tile order (under 4 x 2 n^2/512 bytes)
        m = int(params["n_angles"]) * int(params["n_det"])
        n = int(params["n"])
        return 24 * m + 32 * int(params["n_angles"]) + 4 + 16 * (n // 16 + 1) * (n // 32 + 1)

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
                except imask.ImaskError as e:
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
                plan.close()
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
            stream = torch.cuda.Stream()
            b_dev = torch.empty(m, device="cuda", dtype=torch.float32)
            with torch.cuda.stream(stream):
                b_dev.copy_(host, non_blocking=True)
                state = plan.state(b_dev, req.seed, stream=stream)
            self.plan_users[key] += 1
            self.used += need
            self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)
            req.admitted = self.now()
            req.status = "active"
            self.active.append(_Active(req, key, stream, state, b_dev, req.iters, need))
            self.stats.admitted += 1
            self.stats.max_active = max(self.stats.max_active, len(self.active))
        self.queue = remaining

    def _advance(self):
        for a in self.active:
            if a.finishing or (a.event is not None and not a.event.query()):
                continue
            with torch.cuda.stream(a.stream):
                if a.remaining > 0:
                    q = min(self.quantum, a.remaining)
                    a.state.step(q, stream=a.stream)
                    a.remaining -= q
                else:
                    x_dev = a.state.get(a.state.X, stream=a.stream)
                    a.req.x = torch.empty(x_dev.numel(), dtype=torch.float32, pin_memory=True)
                    a.req.x.copy_(x_dev, non_blocking=True)
                    a.finishing = True
                a.event = torch.cuda.Event()
                a.event.record(a.stream)

    def _retire(self):
        keep = []
        for a in self.active:
            if a.finishing and a.event.query():
                a.req.finished = self.now()
                a.req.status = "done"
                self.stats.completed += 1
                self.stats.latencies.append(a.req.finished - a.req.arrival)
                self.stats.waits.append(a.req.admitted - a.req.arrival)
                a.state.close()
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
        torch.cuda.synchronize()
        for plan, _, _ in self.plans.values():
            plan.check()
        return self.stats

    def close(self):
        torch.cuda.synchronize()
        for a in self.active:
            a.state.close()
        self.active = []
        for fut in self.building.values():
            plan, _, _ = fut.result()
            plan.close()
        self.building.clear()
        self.pool.shutdown(wait=True)
        for plan, _, _ in self.plans.values():
            plan.close()
        self.plans.clear()
