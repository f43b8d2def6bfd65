"""Continuous-batching step server over device-resident scenes.

Requests ``(scene_id, n_steps)`` arrive over time; every scene's state stays on the device
between requests.  Every ``pump()`` polls the steps in flight, admits newly arrived requests
and launches the next steps, so a request that arrives while others run joins at the next
pump instead of waiting for them to finish.

Two kinds of resident scene:

* **Packed** (scenes of at most ``pool_max_bodies`` bodies without drives or augmented
  Lagrangian bonds): such scenes are the groups of one library scene, a *pool*.  One graph
  launch steps every member that has work; the members without work are held still for that
  step (``pabd_set_group_hold``).  A group's step depends only on its own bodies and bonds, and
  a pool holds scenes that use the same lane count alone (the library's choice for the scene's
  size: 16 up to 8192 bodies, 8 up to 16384, ...) and runs with it, so each member's result is
  bit for bit the one it reaches alone.  Small and mid-size scenes are bound by launches and
  latency rather than by the GPU's throughput, so stepping many in one set of launches raises
  the steps served per second.  A newly
  admitted small scene first runs on its own (below) and joins a pool at the next rebuild,
  which happens between steps, at most every ``rebuild_interval`` seconds: the pool's
  members' states are read back, a new pool is built with the newcomers as extra groups, and
  the states are written into it.
* **Alone**: every other scene is its own library scene on its own CUDA stream; one graph
  launch per step, overlapping with the other scenes' steps on the device.

Every scene (and pool) keeps up to ``depth`` steps enqueued on the device, so its next step
never waits for the host to observe the last one.  Packed and small scenes run on
high-priority streams: when the device is oversubscribed, the GPU's scheduler takes their
short kernels before the large scenes' ones, which keeps small steps fast and raises the
steps served per second, at the expense of the large scenes' latency.

Admission by HBM budget: a scene becomes resident when its estimated device memory fits;
idle scenes running alone are evicted least recently used first, their state kept on the
host.  Packing needs room for the new pool next to the old one while it is rebuilt; when
that does not fit, small scenes stay alone.

Latency of a step: from the moment it became eligible (the request's arrival for its first
step, the completion of its previous step otherwise) to the host observing its completion.
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
    launched: int = 0             # steps enqueued on the device so far
    t_eligible: float = 0.0       # when the next step became launchable
    t_done: float | None = None
    step_latency: list = field(default_factory=list)


class _Resident:
    """A scene alone in its own library scene and stream."""

    def __init__(self, scene, stream, nbytes, n_bodies, desc):
        self.scene = scene
        self.stream = stream
        self.bytes = nbytes
        self.n_bodies = n_bodies
        self.desc = desc
        self.queue = collections.deque()
        self.inflight = collections.deque()   # (request, event) per enqueued step, in order
        self.last_use = 0.0


class _Pool:
    """Small scenes packed as the groups of one library scene."""

    def __init__(self, scene, stream, nbytes, members, offsets):
        self.scene = scene
        self.stream = stream
        self.bytes = nbytes
        self.members = members        # scene ids, group order
        self.offsets = offsets        # body offsets of the groups (len(members) + 1)
        self.queues = {sid: collections.deque() for sid in members}
        self.last_use = {sid: 0.0 for sid in members}
        self.inflight = collections.deque()   # ([(scene id, request)], event) per enqueued step
        self.hold = None              # last hold mask sent
        self.key = None               # the members' scene parameters


def _pkey(desc):
    return tuple(sorted((k, repr(v)) for k, v in desc.params.items()))


def _pack(descs):
    """One scenes.Scene whose groups are the given scenes (same parameters), in order."""
    import scenes as S
    bodies, bonds, off = [], [], [0]
    for g, d in enumerate(descs):
        b = d.bodies.copy()
        b["group"] = g
        bo = d.bonds.copy()
        bo["i"] += off[-1]
        bo["j"] = np.where(bo["j"] >= 0, bo["j"] + off[-1], -1)
        bodies.append(b)
        bonds.append(bo)
        off.append(off[-1] + d.n_bodies)
    sc = S.Scene("pool", dict(descs[0].params), np.concatenate(bodies),
                 np.concatenate(bonds) if bonds else np.zeros(0, dtype=S.BOND_DTYPE), 1)
    return sc, np.asarray(off)


class Server:
    """make_scene(scene_id) -> scenes.Scene describes a scene the first time it is needed."""

    def __init__(self, make_scene: Callable[[int], object], hbm_budget: int = 32 << 30, device: int = 0,
                 clock=time.perf_counter, pack: bool = True, pool_max_bodies: int = 8192,
                 pool_capacity: int = 65536, rebuild_interval: float = 0.1, depth: int = 4):
        import torch
        import paper_2609_02675_gb300 as P
        self._torch = torch
        self._P = P
        self.make_scene = make_scene
        self.budget = int(hbm_budget)
        self.device = device
        self.clock = clock
        self.pack = pack
        self.pool_max_bodies = pool_max_bodies
        self.pool_capacity = pool_capacity
        self.rebuild_interval = rebuild_interval
        self.depth = depth
        self.resident: dict[int, _Resident] = {}
        self.pools: list[_Pool] = []
        self.pooled: dict[int, _Pool] = {}       # scene_id -> its pool
        self.descs: dict[int, object] = {}       # scene descriptions of packed scenes
        self.evicted: dict[int, tuple] = {}      # scene_id -> (state rows, step index, n_bodies)
        self.waiting = collections.deque()       # requests whose scene is not resident yet
        self.requests: list[Request] = []
        self.bytes_used = 0
        self.bytes_per_body = None
        self.steps_completed = 0
        self.evictions = 0
        self.admissions = 0
        self.over_budget = 0         # scenes admitted alone although larger than the budget
        self.rebuilds = 0
        self.pool_launches = 0
        self.last_rebuild = -1e30
        self.pending = None          # (key, pool, scene ids) of a rebuild waiting for their steps to drain

    # -- admission -----------------------------------------------------------------------
    def _estimate(self, n_bodies: int) -> int:
        if self.bytes_per_body is None:
            return 0
        return int(self.bytes_per_body * n_bodies) + (1 << 20)

    def _evict_one(self) -> bool:
        """Evict the least recently used idle scene running alone, or idle pool (all its
        members without work), keeping the states on the host."""
        idle = [(r.last_use, 0, sid) for sid, r in self.resident.items() if not r.inflight and not r.queue]
        idle += [(max(p.last_use.values()), 1, k) for k, p in enumerate(self.pools)
                 if not p.inflight and not any(p.queues[s] for s in p.members)]
        if not idle:
            return False
        _, kind, key = min(idle)
        if kind == 0:
            r = self.resident.pop(key)
            st = r.scene.state()
            self.evicted[key] = (st, r.scene.info()["step_index"], r.n_bodies)
            self.bytes_used -= r.bytes
            r.scene.close()
        else:
            p = self.pools.pop(key)
            st = p.scene.state()
            step = p.scene.info()["step_index"]
            for k, sid in enumerate(p.members):
                self.evicted[sid] = (st[p.offsets[k]:p.offsets[k + 1]], step, int(p.offsets[k + 1] - p.offsets[k]))
                del self.pooled[sid]
            self.bytes_used -= p.bytes
            p.scene.close()
        self.evictions += 1
        return True

    def _packable(self, desc) -> bool:
        b = desc.bonds
        return (self.pack and desc.n_bodies <= self.pool_max_bodies and desc.n_groups <= 1
                and not np.isin(b["type"], (4, 5)).any())  # no DRIVE, no AL_DISTANCE

    def _admit(self, scene_id: int) -> bool:
        desc = self.make_scene(scene_id)
        n = desc.n_bodies
        need = self._estimate(n)
        while self.bytes_used + need > self.budget:
            if not self._evict_one():
                if self.resident or self.pools:
                    return False
                break                # alone it may exceed the budget: run it rather than wait forever
        if self.bytes_used + need > self.budget:
            self.over_budget += 1
        # (small scenes keep the launch shape of the pools they will join; large ones are tuned)
        small = self._packable(desc)
        stream = self._torch.cuda.Stream(self.device, priority=-1 if small else 0)
        sc = self._P.Scene(desc, device=self.device, stream=stream, sweep_mode=2 if small else 0,
                           light_order=1 if small else 0)
        if scene_id in self.evicted:
            st, k, _ = self.evicted.pop(scene_id)
            sc.set_state(st)
            sc.set_step_index(k)
        info = sc.info()
        nbytes = info["device_bytes"]
        if self.bytes_per_body is None:
            self.bytes_per_body = nbytes / max(n, 1)
        self.resident[scene_id] = _Resident(sc, stream, nbytes, n, desc)
        self.resident[scene_id].lanes = info["sweep_lanes"]
        self.bytes_used += nbytes
        self.admissions += 1
        return True

    # -- packing -------------------------------------------------------------------------
    def _rebuild(self):
        """Absorb small scenes running alone into a pool, between steps: once a rebuild is
        due, the chosen scenes and the pool they join stop enqueueing steps; when their
        enqueued steps have completed the pool is rebuilt with them."""
        now = self.clock()
        if self.pending is None:
            if now - self.last_rebuild < self.rebuild_interval:
                return
            cand = [sid for sid, r in self.resident.items() if self._packable(r.desc)]
            if not cand:
                return

            # one pool holds scenes of the same parameters (time step, sweeps, ground, ...)
            # and the same lane count alone
            def key_of(sid):
                r = self.resident[sid]
                return _pkey(r.desc), r.lanes

            key = key_of(cand[0])
            cand = [sid for sid in cand if key_of(sid) == key]
            # a pool is only as large as the library keeps the members' lane count for (it
            # halves the lanes above 2^17 lanes x bodies)
            cap = min(self.pool_capacity, (1 << 17) // key[1])
            first = self.resident[cand[0]].n_bodies
            size = {p: sum(self.descs[s].n_bodies for s in p.members) for p in self.pools}
            pool = next((p for p in self.pools if p.key == key and size[p] + first <= cap), None)
            total = size[pool] if pool else 0
            new = []
            for sid in cand:
                n = self.resident[sid].n_bodies
                if total + n > cap:
                    continue
                new.append(sid)
                total += n
            # room for the new pool beside the old one while the states move across
            if not new or self.bytes_used + self._estimate(total) > self.budget:
                self.last_rebuild = now
                return
            self.pending = (key, pool, new)
        key, pool, new = self.pending
        if pool is not None and pool not in self.pools:
            pool = None              # evicted meanwhile: the newcomers start a pool of their own
        new = [sid for sid in new if sid in self.resident]
        if (pool is not None and pool.inflight) or any(self.resident[sid].inflight for sid in new):
            return                   # their enqueued steps are still running
        self.pending = None
        if not new:
            return
        old = list(pool.members) if pool else []
        self.last_rebuild = now
        members = old + new
        descs = [self.descs[s] if s in self.descs else self.resident[s].desc for s in members]
        rows = []
        if pool:
            st = pool.scene.state()
            rows += [st[pool.offsets[k]:pool.offsets[k + 1]] for k in range(len(old))]
        rows += [self.resident[s].scene.state() for s in new]
        sc_desc, off = _pack(descs)
        stream = self._torch.cuda.Stream(self.device, priority=-1)
        lib = self._P.Scene(sc_desc, device=self.device, stream=stream, sweep_lanes=key[1], sweep_mode=2,
                            light_order=1)
        lib.set_state(np.concatenate(rows))
        nbytes = lib.info()["device_bytes"]
        p = _Pool(lib, stream, nbytes, members, off)
        p.key = key
        if pool:
            for s in old:
                p.queues[s] = pool.queues[s]
                p.last_use[s] = pool.last_use[s]
            pool.scene.close()
            self.bytes_used -= pool.bytes
            self.pools.remove(pool)
        for s in new:
            r = self.resident.pop(s)
            p.queues[s] = r.queue
            p.last_use[s] = r.last_use
            self.descs[s] = r.desc
            r.scene.close()
            self.bytes_used -= r.bytes
        for s in members:
            self.pooled[s] = p
        self.pools.append(p)
        self.bytes_used += nbytes
        self.rebuilds += 1

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
            p = self.pooled.get(req.scene_id)
            if p is not None:
                p.queues[req.scene_id].append(req)
                continue
            r = self.resident.get(req.scene_id)
            if r is None and self._admit(req.scene_id):
                r = self.resident[req.scene_id]
            if r is None:
                still.append(req)
            else:
                r.queue.append(req)
        self.waiting = still

    def _complete(self, req, queue, t):
        """One step of req observed complete at t."""
        req.step_latency.append(t - req.t_eligible)
        req.steps_done += 1
        self.steps_completed += 1
        if req.steps_done == req.n_steps:
            req.t_done = t
            queue.popleft()
        else:
            req.t_eligible = t

    @staticmethod
    def _next(queue):
        """The first request of a queue with steps not yet enqueued (requests run in order)."""
        for req in queue:
            if req.launched < req.n_steps:
                return req
        return None

    def pump(self) -> int:
        """Poll completions, admit, pack and launch; returns the number of steps launched.
        Each scene (and each pool) keeps up to `depth` steps enqueued on the device, so it
        never waits for the host to observe a step before the next one starts."""
        for p in self.pools:
            while p.inflight and p.inflight[0][1].query():
                members, _ = p.inflight.popleft()
                t = self.clock()
                for sid, req in members:
                    self._complete(req, p.queues[sid], t)
                    p.last_use[sid] = t
        for r in self.resident.values():
            while r.inflight and r.inflight[0][1].query():
                req, _ = r.inflight.popleft()
                t = self.clock()
                self._complete(req, r.queue, t)
                r.last_use = t
        self._route_waiting()
        if self.pack:
            self._rebuild()
        launched = 0
        draining = set(self.pending[2]) if self.pending else set()
        drain_pool = self.pending[1] if self.pending else None
        for p in self.pools:
            if p is drain_pool:
                continue
            idx = None
            while len(p.inflight) < self.depth:
                active = [(sid, self._next(p.queues[sid])) for sid in p.members]
                active = [(sid, req) for sid, req in active if req is not None]
                if not active:
                    break
                if idx is None:
                    idx = {sid: k for k, sid in enumerate(p.members)}
                hold = np.ones(len(p.members), dtype=np.uint8)
                for sid, _ in active:
                    hold[idx[sid]] = 0
                if p.hold is None or not np.array_equal(hold, p.hold):
                    p.scene.set_group_hold(hold)
                    p.hold = hold
                p.scene.step(1)
                ev = self._torch.cuda.Event()
                ev.record(p.stream)
                for _, req in active:
                    req.launched += 1
                p.inflight.append((active, ev))
                self.pool_launches += 1
                launched += len(active)
        now = self.clock()
        for sid, r in self.resident.items():
            if sid in draining:
                continue
            while len(r.inflight) < self.depth:
                req = self._next(r.queue)
                if req is None:
                    break
                r.scene.step(1)
                ev = self._torch.cuda.Event()
                ev.record(r.stream)
                req.launched += 1
                r.inflight.append((req, ev))
                r.last_use = now
                launched += 1
        return launched

    def busy(self) -> bool:
        return (bool(self.waiting) or any(r.inflight or r.queue for r in self.resident.values())
                or any(p.inflight or any(p.queues[s] for s in p.members) for p in self.pools))

    def drain(self, timeout: float = 600.0):
        t0 = self.clock()
        while self.busy() and self.clock() - t0 < timeout:
            self.pump()

    def state(self, scene_id: int) -> np.ndarray:
        """The scene's current state rows (resident alone, packed or evicted)."""
        p = self.pooled.get(scene_id)
        if p is not None:
            k = p.members.index(scene_id)
            return p.scene.state()[p.offsets[k]:p.offsets[k + 1]]
        r = self.resident.get(scene_id)
        if r is not None:
            return r.scene.state()
        return self.evicted[scene_id][0]

    def close(self):
        for r in self.resident.values():
            r.scene.close()
        for p in self.pools:
            p.scene.close()
        self.resident.clear()
        self.pools.clear()
        self.pooled.clear()

    def _n_bodies(self, scene_id: int) -> int:
        if scene_id in self.descs:
            return self.descs[scene_id].n_bodies
        r = self.resident.get(scene_id)
        if r is not None:
            return r.n_bodies
        e = self.evicted.get(scene_id)
        return e[2] if e is not None else 0

    # -- results ---------------------------------------------------------------------------
    def stats(self, t_start: float, t_end: float) -> dict:
        lat = np.array([x for q in self.requests for x in q.step_latency]) * 1e3
        body_steps = sum(self._n_bodies(q.scene_id) * q.steps_done for q in self.requests)
        done = [q for q in self.requests if q.t_done is not None]
        rl = np.array([q.t_done - q.t_arrival for q in done]) * 1e3
        return {
            "requests": len(self.requests), "requests_done": len(done), "steps": int(lat.size),
            "steps_per_s": lat.size / max(t_end - t_start, 1e-9),
            "body_steps_per_s": body_steps / max(t_end - t_start, 1e-9),
            "step_latency_ms": {"p50": float(np.percentile(lat, 50)) if lat.size else None,
                                "p99": float(np.percentile(lat, 99)) if lat.size else None},
            "request_latency_ms": {"p50": float(np.percentile(rl, 50)) if rl.size else None,
                                   "p99": float(np.percentile(rl, 99)) if rl.size else None},
            "admissions": self.admissions, "evictions": self.evictions, "over_budget": self.over_budget,
            "resident_bytes": self.bytes_used, "packed_scenes": len(self.pooled), "pool_rebuilds": self.rebuilds,
            "pool_launches": self.pool_launches,
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
