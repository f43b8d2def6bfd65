"""Continuous-batching step server over device-resident scenes.

Requests ``(scene_id, n_steps)`` arrive over time.  Each resident scene is one library
scene with its own CUDA stream and its state kept on the device between requests.  Every
``pump()`` polls the steps in flight and admits newly arrived requests. A scene becomes
resident when its device memory fits the HBM budget; idle scenes are evicted least recently
used first, their state kept on the host. ``pump()`` then launches one step (one CUDA-graph
launch) for every resident scene that has pending work and no step in flight. Steps of
different scenes therefore overlap on the GPU, and a request that arrives while others run
joins at the next pump instead of waiting for them to finish.

Latency of a step: from the moment it became eligible (the request's arrival for its first
step, the completion of its previous step otherwise) to the host observing its completion
event.  Each scene's arithmetic is independent of the others, so its result is the same
alone and in the mix.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Callable

import numpy as np


@dataclass
class Request:
    rid: int
    scene_id: int
    n_steps: int
    t_arrival: float
    steps_done: int = 0
    t_eligible: float = 0.0       # when the next step became launchable
    t_done: float | None = None
    step_latency: list = field(default_factory=list)


class _Resident:
    def __init__(self, scene, stream, nbytes, n_bodies):
        self.scene = scene
        self.stream = stream
        self.bytes = nbytes
        self.n_bodies = n_bodies
        self.queue = collections.deque()
        self.inflight = None          # (request, t_eligible, event)
        self.last_use = 0.0


class Server:
    """make_scene(scene_id) -> scenes.Scene describes a scene the first time it is needed."""

    def __init__(self, make_scene: Callable[[int], object], hbm_budget: int = 32 << 30, device: int = 0,
                 clock=time.perf_counter):
        import torch
        import paper_2609_02675_gb300 as P
        self._torch = torch
        self._P = P
        self.make_scene = make_scene
        self.budget = int(hbm_budget)
        self.device = device
        self.clock = clock
        self.resident: dict[int, _Resident] = {}
        self.evicted: dict[int, tuple] = {}      # scene_id -> (state rows, step index, n_bodies)
        self.waiting = collections.deque()       # requests whose scene is not resident yet
        self.requests: list[Request] = []
        self.bytes_used = 0
        self.bytes_per_body = None
        self.steps_completed = 0
        self.evictions = 0
        self.admissions = 0
        self.over_budget = 0         # scenes admitted alone although larger than the budget

    # -- admission -----------------------------------------------------------------------
    def _estimate(self, n_bodies: int) -> int:
        if self.bytes_per_body is None:
            return 0
        return int(self.bytes_per_body * n_bodies) + (1 << 20)

    def _evict_one(self) -> bool:
        idle = [(r.last_use, sid) for sid, r in self.resident.items() if r.inflight is None and not r.queue]
        if not idle:
            return False
        _, sid = min(idle)
        r = self.resident.pop(sid)
        st = r.scene.state()
        self.evicted[sid] = (st, r.scene.info()["step_index"], r.n_bodies)
        self.bytes_used -= r.bytes
        r.scene.close()
        self.evictions += 1
        return True

    def _admit(self, scene_id: int) -> bool:
        desc = self.make_scene(scene_id)
        n = desc.n_bodies
        need = self._estimate(n)
        while self.bytes_used + need > self.budget:
            if not self._evict_one():
                if self.resident:
                    return False
                break                # alone it may exceed the budget: run it rather than wait forever
        if self.bytes_used + need > self.budget:
            self.over_budget += 1
        stream = self._torch.cuda.Stream(self.device)
        sc = self._P.Scene(desc, device=self.device, stream=stream)
        if scene_id in self.evicted:
            st, k, _ = self.evicted.pop(scene_id)
            sc.set_state(st)
            sc.set_step_index(k)
        nbytes = sc.info()["device_bytes"]
        if self.bytes_per_body is None:
            self.bytes_per_body = nbytes / max(n, 1)
        self.resident[scene_id] = _Resident(sc, stream, nbytes, n)
        self.bytes_used += nbytes
        self.admissions += 1
        return True

    # -- requests ------------------------------------------------------------------------
    def submit(self, scene_id: int, n_steps: int, t_arrival: float | None = None) -> Request:
        t = self.clock() if t_arrival is None else t_arrival
        req = Request(len(self.requests), scene_id, n_steps, t, t_eligible=t)
        self.requests.append(req)
        self.waiting.append(req)
        return req

    def _route_waiting(self):
        still = collections.deque()
        while self.waiting:
            req = self.waiting.popleft()
            r = self.resident.get(req.scene_id)
            if r is None and self._admit(req.scene_id):
                r = self.resident[req.scene_id]
            if r is None:
                still.append(req)
            else:
                r.queue.append(req)
        self.waiting = still

    def pump(self) -> int:
        """Poll completions, admit and launch; returns the number of steps launched."""
        now = self.clock()
        for r in self.resident.values():
            if r.inflight is not None and r.inflight[2].query():
                req, t_elig, _ = r.inflight
                t = self.clock()
                req.step_latency.append(t - t_elig)
                req.steps_done += 1
                self.steps_completed += 1
                r.inflight = None
                r.last_use = t
                if req.steps_done == req.n_steps:
                    req.t_done = t
                    r.queue.popleft()
                else:
                    req.t_eligible = t
        self._route_waiting()
        launched = 0
        for r in self.resident.values():
            if r.inflight is None and r.queue:
                req = r.queue[0]
                t_elig = req.t_eligible if req.steps_done else max(req.t_arrival, req.t_eligible)
                r.scene.step(1)
                ev = self._torch.cuda.Event()
                ev.record(r.stream)
                r.inflight = (req, t_elig, ev)
                r.last_use = now
                launched += 1
        return launched

    def busy(self) -> bool:
        return bool(self.waiting) or any(r.inflight is not None or r.queue for r in self.resident.values())

    def drain(self, timeout: float = 600.0):
        t0 = self.clock()
        while self.busy() and self.clock() - t0 < timeout:
            self.pump()

    def close(self):
        for r in self.resident.values():
            r.scene.close()
        self.resident.clear()

    # -- results ---------------------------------------------------------------------------
    def stats(self, t_start: float, t_end: float) -> dict:
        lat = np.array([x for q in self.requests for x in q.step_latency]) * 1e3
        done = [q for q in self.requests if q.t_done is not None]
        rl = np.array([q.t_done - q.t_arrival for q in done]) * 1e3
        return {
            "requests": len(self.requests), "requests_done": len(done), "steps": int(lat.size),
            "steps_per_s": lat.size / max(t_end - t_start, 1e-9),
            "step_latency_ms": {"p50": float(np.percentile(lat, 50)) if lat.size else None,
                                "p99": float(np.percentile(lat, 99)) if lat.size else None},
            "request_latency_ms": {"p50": float(np.percentile(rl, 50)) if rl.size else None,
                                   "p99": float(np.percentile(rl, 99)) if rl.size else None},
            "admissions": self.admissions, "evictions": self.evictions, "over_budget": self.over_budget,
            "resident_bytes": self.bytes_used,
        }


def replay(server: Server, reqs, duration: float | None = None, drain_timeout: float = 120.0):
    """Feed (t, scene_id, n_steps) requests at their arrival times (seconds from start) in
    real time, pumping the server in between, until every request is done or drain_timeout
    seconds after the last arrival; returns (t_start, t_end)."""
    t0 = server.clock()
    k = 0
    reqs = sorted(reqs)
    last = reqs[-1][0] if reqs else 0.0
    limit = (duration if duration is not None else last) + drain_timeout
    while k < len(reqs) or server.busy():
        now = server.clock() - t0
        while k < len(reqs) and reqs[k][0] <= now:
            t, sid, n = reqs[k]
            server.submit(sid, n, t0 + t)
            k += 1
        server.pump()
        if now > limit:
            break
    return t0, server.clock()
